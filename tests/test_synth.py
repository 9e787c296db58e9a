"""The seeded input generator (no GPU): array invariants that the library's
ingest checks, determinism, and the workload recipe (sizes and variation
rates) that the inputs are built to."""
import numpy as np
import pytest

from synth import CONFIGS, make_custom, make_graph, make_linear_path


@pytest.fixture(scope="module", params=["tiny", "mid"])
def graph(request):
    return request.param, make_graph(request.param)


def test_arrays_satisfy_the_ingest_rules(graph):
    _, g = graph
    assert g.node_len.dtype == np.uint32 and g.path_off.dtype == np.uint64
    assert g.step_node.dtype == np.uint32 and g.step_rev.dtype == np.uint8 and g.step_pos.dtype == np.int64
    assert g.node_len.min() >= 1
    off = g.path_off.astype(np.int64)
    assert off[0] == 0 and np.all(np.diff(off) >= 0) and off[-1] == len(g.step_node)
    assert g.step_node.max() < g.n_nodes and set(np.unique(g.step_rev)) <= {0, 1}
    # a path starts at position 0 and advances by the length of the node it leaves
    nl = g.node_len[g.step_node].astype(np.int64)
    first = np.zeros(len(g.step_node), bool)
    first[off[:-1][np.diff(off) > 0]] = True
    assert np.all(g.step_pos[first] == 0)
    nxt = ~first[1:]
    np.testing.assert_array_equal(g.step_pos[1:][nxt], (g.step_pos[:-1] + nl[:-1])[nxt])
    # the initial layout is FP32-representable, finite, one segment per node
    assert g.init_xy.shape == (g.n_nodes, 4) and np.all(np.isfinite(g.init_xy))
    np.testing.assert_array_equal(g.init_xy.astype(np.float32).astype(np.float64), g.init_xy)


def test_generation_is_deterministic_per_seed():
    a, b, c = make_graph("tiny"), make_graph("tiny"), make_graph("tiny", gen_seed=99)
    for f in ("node_len", "path_off", "step_node", "step_rev", "step_pos", "init_xy"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert len(c.step_node) != len(a.step_node) or not np.array_equal(c.step_node, a.step_node)


def test_sizes_of_the_configurations(graph):
    name, g = graph
    cfg = CONFIGS[name]
    B = cfg["backbone"]
    assert g.n_paths == cfg["paths"] and g.n_nodes == B + g.meta["sites"]
    assert g.n_steps == {"tiny": 15_855, "mid": 6_963_896}[name]
    # alternative nodes copy their site's length
    assert abs(g.meta["sites"] / B - cfg["p_site"]) < 4 * np.sqrt(cfg["p_site"] / B) + 1e-3
    # backbone lengths: geometric on 1, 2, ... with the configured mean
    assert abs(g.node_len[:B].mean() / cfg["len_mean"] - 1) < 0.05


def test_variation_rates_follow_the_recipe():
    g = make_graph("mid")
    cfg = CONFIGS["mid"]
    B = cfg["backbone"]
    # a path takes the alternative at a site with probability p_alt: p_site * p_alt of its steps
    alt = np.mean(g.step_node >= B)
    assert abs(alt - cfg["p_site"] * cfg["p_alt"]) < 0.003
    # reversed steps come from inversions: p_inv per node x mean run length (27.5), less overlaps
    rev = g.step_rev.mean()
    assert 0.8 * cfg["p_inv"] * 27.5 < rev < 1.05 * cfg["p_inv"] * 27.5
    # a path visits about B nodes: deletions remove 1 %, duplications add p_dup x mean run (105)
    per_path = np.diff(g.path_off.astype(np.int64)).mean()
    expect = B * (1 + cfg["p_dup"] * 105) * (1 - cfg["p_del"])
    assert abs(per_path / expect - 1) < 0.02


def test_alternative_nodes_sit_at_a_backbone_site_of_their_length():
    g = make_graph("tiny")
    B = CONFIGS["tiny"]["backbone"]
    assert np.any(g.step_node >= B)
    back_pos = np.concatenate([[0], np.cumsum(g.node_len[:B].astype(np.int64))[:-1]])
    # initial x of an alternative node = its site's backbone position + N(0, 1) jitter, and it has the
    # site's length: some backbone node of that length starts within 5 sigma of it
    for a in range(B, g.n_nodes):
        near = np.abs(back_pos - g.init_xy[a, 0]) < 5
        assert np.any(near & (g.node_len[:B] == g.node_len[a])), a
    seg = g.init_xy[:, 2] - g.init_xy[:, 0]
    assert np.all(np.abs(seg - g.node_len) < 10)  # two N(0, 1) draws apart


def test_custom_and_linear_graphs():
    g = make_custom([4, 5, 6], [[(0, 0), (2, 1)], [], [(1, 0)]])
    np.testing.assert_array_equal(g.path_off, [0, 2, 2, 3])
    np.testing.assert_array_equal(g.step_pos, [0, 4, 0])
    np.testing.assert_array_equal(g.step_rev, [0, 1, 0])
    lin = make_linear_path(100, seed=3, jitter=0.0)
    x = np.concatenate([[0], np.cumsum(lin.node_len.astype(np.int64))[:-1]])
    np.testing.assert_array_equal(lin.init_xy[:, 0], x)
    np.testing.assert_array_equal(lin.init_xy[:, 2], x + lin.node_len)
    np.testing.assert_array_equal(lin.step_pos, x)
