"""Hogwild! layouts on the GPU against the oracle's layouts (stress level).

GPU and oracle apply the same draws in different orders (lock-free threads
vs the oracle's loop), so their layouts differ; parity is judged on the
sampled path stress (Eq. 2) of the results under the same stress seed. The
oracle's numbers for the two larger graphs come from
tests/golden/make_oracle_layouts.py.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from synth import make_graph, make_linear_path

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_layouts.json")
T = 30


@pytest.fixture(scope="module")
def pg():
    import paper_2409_00876_gb300 as pg
    pg.load_library()
    return pg


def _gold(name):
    if not os.path.exists(GOLD):
        pytest.skip("no oracle layout record")
    data = json.load(open(GOLD))
    if name not in data or not data[name]["runs"]:
        pytest.skip(f"no oracle layout record for {name}")
    return data[name]


def _layout_stress(pg, g, seed, per_step, sseed, **opts):
    G = pg.Graph.from_synth(g)
    for k, v in opts.items():
        G.set_option(k, v)
    G.set_coords(g.init_xy)
    G.layout(T, theta=0.99, seed=seed)
    return G.stress(per_step, seed=sseed), G


def test_linear_path_converges_on_gpu(pg):
    g = make_linear_path(3000, len_mean=8, seed=4, jitter=3.0)
    st, _ = _layout_stress(pg, g, 3, 100, 2)
    assert st["mean"] < 1e-3


def test_tiny_layout_quality_matches_oracle_within_1_percent(pg):
    """The 1 % target resolved: 64 layout seeds on each side (the oracle
    sequential, the GPU lock-free, each seed's draws the same on both), so
    that two standard errors of the difference of the means, from the
    measured seed-to-seed spreads, come below 1 % of the oracle's mean; the
    bar is then 1 %. (With 40 seeds 2 SE came to 0.90-0.95 %, too close to
    the 1 % it must stay under for a sample variance of 40 lock-free runs;
    64 seeds put it near 0.7 %.)"""
    g = make_graph("tiny")
    ref = []
    got = []
    for seed in range(1, 65):
        xy, _ = O.layout(g, g.init_xy, T=T, theta=0.99, seed=seed)
        ref.append(O.sampled_stress(g, xy, seed=7)["mean"])
        got.append(_layout_stress(pg, g, seed, 100, 7)[0]["mean"])
    ref, got = np.array(ref), np.array(got)
    se = np.sqrt(ref.var(ddof=1) / len(ref) + got.var(ddof=1) / len(got))
    print("tiny", got.mean(), ref.mean(), (got.mean() - ref.mean()) / ref.mean(), 2 * se / ref.mean())
    assert 2 * se <= 0.01 * ref.mean(), (se, ref.mean())  # the comparison resolves 1 %
    assert abs(got.mean() - ref.mean()) <= 0.01 * ref.mean(), (got.mean(), ref.mean())


@pytest.mark.parametrize("name", ["mid", "mid_1000", "chrom"])
def test_layout_stress_matches_oracle(pg, name):
    """The GPU's lock-free layout reaches the oracle's quality (the 1 % target
    on the sampled path stress, Eq. 2, under the same layout and stress
    seeds; reading R28). Every variance in the bar is measured, none assumed:

    - records over several layout seeds (mid: 6 seeds at 100 samples per
      step; mid_1000: 16 seeds at 1000): the GPU lays the graph out once per
      seed, and the comparison is paired by seed, since a seed's draws are the
      same on both sides and fix most of its layout's stress (the per-seed
      stresses of the two sides correlate at 0.96 on mid_1000): the mean
      difference over seeds, SE from the spread of the per-seed differences;
      bar max(1 %, 2 SE). mid_1000 must resolve the target (2 SE <= 1 %);
      at 100 samples per step the heavy-tailed sample set makes most of the
      spread (reading R29);
    - the chromosome graph (one seed, each oracle run takes hours): five GPU
      repeats against the oracle's repeats of the same seed; SE from the
      measured run-to-run spreads of both; bar max(1 %, 2 SE), and it must
      resolve the target (2 SE <= 1 %). It needs two oracle runs at least,
      else the oracle's spread is unknown and the test skips."""
    gold = _gold(name)
    g = make_graph(gold.get("graph", name))
    fp = gold["fingerprint"]
    assert (g.n_nodes, g.n_paths, g.n_steps) == (fp["n_nodes"], fp["n_paths"], fp["n_steps"])
    per, sseed = gold["stress_samples_per_step"], gold["stress_seed"]
    ref = np.array([r["stress"] for r in gold["runs"]])
    seeds = [r["seed"] for r in gold["runs"]]
    if len(set(seeds)) > 1:
        assert len(set(seeds)) == len(seeds)
        got = np.array([_layout_stress(pg, g, sd, per, sseed)[0]["mean"] for sd in seeds])
        d = got - ref
        se = d.std(ddof=1) / np.sqrt(len(d))
    else:
        if len(ref) < 2:
            pytest.skip(f"{name}: one oracle run; its run-to-run spread is not measured")
        got = np.array([_layout_stress(pg, g, seeds[0], per, sseed)[0]["mean"] for _ in range(5)])
        se = np.sqrt(got.var(ddof=1) / len(got) + ref.var(ddof=1) / len(ref))
    bar = max(0.01 * ref.mean(), 2 * se)
    print(name, got, ref, (got.mean() - ref.mean()) / ref.mean(), 2 * se / ref.mean())
    if name in ("mid_1000", "chrom"):  # these records resolve the target: the bar is the 1 % itself
        assert 2 * se <= 0.01 * ref.mean(), (se, ref.mean())
    assert abs(got.mean() - ref.mean()) <= bar, (got, ref, bar)
    assert got.max() < 0.5 * gold["init_stress"]


def test_small_graphs_laid_out_alone_match_the_oracle(pg):
    """The concurrency cap on small graphs (reading R17): each of the 12
    graphs of the small batch workload (1-12 k nodes, 4-12 paths) laid out
    alone by the single-graph kernel, under the first 48 layout seeds of the
    oracle's record for these graphs, compared paired by seed as the batch
    test does: the pooled relative difference within max(1 %, 2 SE), the
    comparison resolving 1 % (2 SE <= 1 %). With 2048 updates in flight on
    these graphs the GPU came out 3.4 % above the oracle."""
    from synth import make_batch
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_batch_small.json")))
    n_seeds = 48  # one graph folds on some seeds: enough seeds to dilute a fold on one side only
    gs = make_batch("batch_small")
    rel = []
    for k, g in enumerate(gs):
        rec = gold["graphs"][k]
        assert (g.n_nodes, g.n_steps) == (rec["n_nodes"], rec["n_steps"])
        ref = np.array(rec["stress"][:n_seeds])
        G = pg.Graph.from_synth(g)
        got = []
        for s in gold["seeds"][:n_seeds]:
            G.set_coords(g.init_xy)
            G.layout(gold["iterations"], theta=gold["theta"], seed=s)
            got.append(G.stress(gold["stress_samples_per_step"], seed=gold["stress_seed"])["mean"])
        G.close()
        rel.append((np.array(got) - ref) / ref.mean())
    rel = np.array(rel)                                      # [G, seeds]
    per_graph = rel.mean(axis=1)
    se = np.sqrt(np.sum(rel.var(axis=1, ddof=1) / n_seeds)) / len(per_graph)
    print("alone: per-graph differences", np.round(per_graph, 4), "pooled", per_graph.mean(), "2 SE", 2 * se)
    assert 2 * se <= 0.01, se
    assert abs(per_graph.mean()) <= max(0.01, 2 * se), (per_graph, se)


def test_resume_in_two_calls_matches_one_call_quality(pg):
    g = make_graph("mid")
    G = pg.Graph.from_synth(g)
    G.set_coords(g.init_xy)
    G.layout(T, theta=0.99, seed=5, iter_end=12)
    G.layout(T, theta=0.99, seed=5, iter_begin=12)
    two = G.stress(20, seed=7)["mean"]
    ones = [_layout_stress(pg, g, 5, 20, 7)[0]["mean"] for _ in range(2)]
    # lock-free runs differ from run to run; the split run must sit in that spread
    spread = max(abs(ones[0] - ones[1]), 0.1 * ones[0])
    assert abs(two - np.mean(ones)) <= 2 * spread, (two, ones)


def _adjacent_stress(g, xy):
    """Mean stress of the start points of consecutive steps of a forward path
    (reference distance = the first node's length): the layout's local detail."""
    a, b = g.step_node[:-1], g.step_node[1:]
    d = g.node_len[a].astype(np.float64)
    mag = np.hypot(xy[a, 0] - xy[b, 0], xy[a, 1] - xy[b, 1])
    return float(np.mean(((mag - d) / d) ** 2))


def test_plain_fp32_coordinates_lose_resolution_at_chromosome_scale(pg):
    # A single forward path far from the origin: its zero-stress layout exists.
    # At 1.5e8 an FP32 value is a multiple of 16 nt, so plain FP32 cannot place
    # 8-nt neighbours; the anchored form keeps sub-nucleotide resolution.
    g = make_linear_path(20_000, len_mean=8, seed=4, jitter=3.0)
    xy = g.init_xy.copy()
    xy[:, [0, 2]] += 1.5e8
    res = {}
    for mode in (0, 1):
        G = pg.Graph.from_synth(g)
        G.set_option("coord_mode", mode)
        G.set_coords(xy)
        G.layout(T, theta=0.99, seed=1)
        res[mode] = _adjacent_stress(g, G.get_coords())
    assert res[0] < 0.05 and res[1] > 10 * res[0], res


def test_create_rejects_inconsistent_graphs(pg):
    from paper_2409_00876_gb300 import PgsgdError
    g = make_graph("tiny")
    bad_node = g.step_node.copy()
    bad_node[100] = g.n_nodes
    with pytest.raises(PgsgdError, match="node id"):
        pg.Graph(g.node_len, g.path_off, bad_node, g.step_rev, g.step_pos)
    bad_pos = g.step_pos.copy()
    bad_pos[200] += 1
    with pytest.raises(PgsgdError, match="positions"):
        pg.Graph(g.node_len, g.path_off, g.step_node, g.step_rev, bad_pos)
    bad_rev = g.step_rev.copy()
    bad_rev[5] = 2
    with pytest.raises(PgsgdError, match="orientation"):
        pg.Graph(g.node_len, g.path_off, g.step_node, bad_rev, g.step_pos)
    zero = g.node_len.copy()
    zero[0] = 0
    with pytest.raises(PgsgdError):
        pg.Graph(zero, g.path_off, g.step_node, g.step_rev, g.step_pos)
    G = pg.Graph.from_synth(g)
    with pytest.raises(PgsgdError, match="set_coords"):
        G.layout(T)
    far = g.init_xy.copy()
    far[3, 0] = 2.0 ** 31
    with pytest.raises(PgsgdError, match="2\\^30"):
        G.set_coords(far)
    with pytest.raises(PgsgdError, match="theta"):
        G.set_coords(g.init_xy)
        G.layout(T, theta=5.0)


def test_layout_rejects_bad_learning_rates_before_any_move(pg):
    """A negative or NaN rate would move pairs apart or poison both nodes:
    the call refuses it before the first launch, so the layout is unchanged."""
    from paper_2409_00876_gb300 import PgsgdError
    g = make_graph("tiny")
    G = pg.Graph.from_synth(g)
    G.set_coords(g.init_xy)
    before = G.get_coords()
    good = np.geomspace(100.0, 0.01, T)
    for t, v in [(0, np.nan), (T - 1, -1e-3), (7, np.inf)]:
        eta = good.copy()
        eta[t] = v
        with pytest.raises(PgsgdError, match="learning rate"):
            G.layout(T, eta=eta, seed=3)
    with pytest.raises(PgsgdError, match="learning rate"):
        G.layout(T, eta_max=np.inf, seed=3)
    np.testing.assert_array_equal(G.get_coords(), before)
    eta = good.copy()
    eta[-5:] = 0.0  # a zero rate is a valid no-op iteration
    G.layout(T, eta=eta, seed=3)
    assert not np.array_equal(G.get_coords(), before)
