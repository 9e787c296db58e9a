"""Batched layout on the GPU against the oracle, graph by graph.

Every graph of a batch must draw exactly the pairs the oracle draws for that
graph alone under its seed (bit-exact), its sampled stress must be the
oracle's statistic of the same layout, and the three schedules (per-iteration
launches, one persistent launch, one launch per graph) must reach the
oracle's layout quality (tests/golden/make_batch_goldens.py). The persistent
kernel's bounded waits are made to expire on purpose (a queue that never
opens) and must end in PGSGD_ETIMEOUT with the context still usable.
"""
import json
import os
import time

import numpy as np
import pytest

import oracle as O
from synth import concat, make_batch, make_custom, make_graph

pytestmark = pytest.mark.gpu

T = 30
THETA = 0.99
GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_batch_small.json")
HIGHPATH = os.path.join(os.path.dirname(__file__), "golden", "oracle_batch_highpath.json")
FIELDS = ["g", "i", "j", "d_ref", "path", "cooling", "e_i", "e_j", "skip"]


@pytest.fixture(scope="module")
def small():
    from paper_2409_00876_gb300.batch import Batch
    gs = make_batch("batch_small")
    arr = concat(gs)
    B = Batch.from_arrays(arr)
    B.set_coords(arr.init_xy)
    return gs, arr, B


def _same(a, b):
    for f in FIELDS:
        np.testing.assert_array_equal(a[f], b[f], err_msg=f)


@pytest.mark.parametrize("t", [0, 14, 29])
def test_draws_bit_exact_per_graph(small, t):
    gs, _, B = small
    for k in (0, 3, 7, 11):
        seed = 1000 + k
        got = B.debug_sample(k, t, T, THETA, seed, 777, 30_000)
        want = O.sample(gs[k], T, t, THETA, seed, 777, 30_000)
        _same(got, want)


def test_draws_match_the_single_graph_kernel(small):
    import paper_2409_00876_gb300 as pg
    gs, _, B = small
    for k in (1, 9):
        G = pg.Graph.from_synth(gs[k])
        for t in (3, 20):
            _same(B.debug_sample(k, t, T, 0.5, 42, 0, 50_000), G.debug_sample(t, T, 0.5, 42, 0, 50_000))


def test_stress_per_graph_is_the_oracle_statistic(small):
    gs, arr, B = small
    B.set_option("mode", 0)
    B.set_coords(arr.init_xy)
    B.layout(T, seeds=np.arange(1, len(gs) + 1), theta=THETA)
    xy = B.get_coords()
    st = B.stress(100, seed=7)
    for k, g in enumerate(gs):
        want = O.sampled_stress(g, arr.graph_xy(xy, k), per_step=100, seed=7)
        assert st[k]["n_valid"] == want["n_valid"]
        assert st[k]["n_skipped"] == want["n_skipped"]
        assert abs(st[k]["mean"] - want["mean"]) <= 1e-4 * want["mean"], (k, st[k], want)


def test_stress_per_graph_equals_single_graph_stress(small):
    import paper_2409_00876_gb300 as pg
    gs, arr, B = small
    B.set_coords(arr.init_xy)
    B.layout(T, seeds=5, theta=THETA, iter_end=3)
    xy = B.get_coords()
    st = B.stress(20, seed=9)
    for k in (0, 5, 10):
        G = pg.Graph.from_synth(gs[k])
        G.set_coords(arr.graph_xy(xy, k))
        one = G.stress(20, seed=9)
        assert st[k]["n_valid"] == one["n_valid"]
        # same pairs; the one-graph handle re-anchors x on upload, which
        # changes FP32 rounding of the differences only
        assert abs(st[k]["mean"] - one["mean"]) <= 1e-6 * one["mean"]


def _gold():
    if not os.path.exists(GOLD):
        pytest.skip("no oracle batch record")
    return json.load(open(GOLD))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_layout_quality_matches_oracle(small, mode):
    """Per graph and layout seed, the GPU batch's sampled stress against the
    oracle's for that graph alone under the same seed (the same draws on both
    sides; reading R28). Single layouts of these 1 k - 12 k-node graphs vary by
    tens of percent from seed to seed (some seeds fold a graph into a layout
    of several times the typical stress), so the record holds 128 seeds per
    graph and the comparison is paired by seed: per graph the mean of the
    per-seed differences relative to the oracle's mean, pooled over the 12
    graphs with SE from the measured spread of the per-seed differences. The
    pooled difference must lie within max(1 %, 2 SE), the comparison must
    resolve the 1 % target (2 SE <= 1 %), and no graph may be far off. Every
    schedule runs the first 64 seeds: one graph (5 k nodes) folds on about
    one seed in ten into a layout of three times the typical stress, and a
    seed that folds on one side only moves its mean by several percent, which
    16 seeds did not dilute enough (2 SE 1.2 % in two runs)."""
    gold = _gold()
    gs, arr, B = small
    for k, g in enumerate(gs):
        rec = gold["graphs"][k]
        assert (g.n_nodes, g.n_paths, g.n_steps) == (rec["n_nodes"], rec["n_paths"], rec["n_steps"])
    B.set_option("mode", mode)
    n_seeds = 64
    runs = []
    for s in gold["seeds"][:n_seeds]:
        B.set_coords(arr.init_xy)
        B.layout(gold["iterations"], seeds=s, theta=gold["theta"])
        runs.append([r["mean"] for r in B.stress(gold["stress_samples_per_step"], gold["stress_seed"])])
    got = np.array(runs).T                                   # [G, seeds]
    ref = np.array([r["stress"][:n_seeds] for r in gold["graphs"]])  # [G, seeds]
    n = got.shape[1]
    rel = (got - ref) / ref.mean(axis=1, keepdims=True)      # paired, relative to the oracle's mean
    per_graph = rel.mean(axis=1)
    se_graph = rel.std(axis=1, ddof=1) / np.sqrt(n)
    pooled = per_graph.mean()
    se = np.sqrt(np.sum(se_graph ** 2)) / len(per_graph)
    corr = [np.corrcoef(got[k], ref[k])[0, 1] for k in range(len(gs))]
    print("mode", mode, "per-graph differences", np.round(per_graph, 4), "2 SE", np.round(2 * se_graph, 4),
          "seed correlation", np.round(corr, 2), "pooled", pooled, "2 SE", 2 * se)
    assert 2 * se <= 0.01, se                                # the comparison resolves 1 %
    assert abs(pooled) <= max(0.01, 2 * se), (pooled, se)
    # a graph the schedule broke would sit far from the oracle or near its initial stress
    assert np.all(np.abs(per_graph) <= np.maximum(0.15, 4 * se_graph)), (per_graph, se_graph)
    init = np.array([r["init_stress"] for r in gold["graphs"]])
    assert np.all(got.mean(axis=1) < init)


def test_many_paths_per_node_quality_matches_oracle():
    """Small graphs with many paths per node (1.1-3.9 k nodes, 65-88 paths,
    from the 256-subgraph workload): each node receives hundreds of moves per
    iteration, and the cap's N / 5120 term lets more updates run at once
    than n_nodes / 16 would. Laid out together in one batch (mode 0) under
    16 layout seeds, paired by seed with the oracle's layouts of each graph
    alone: the pooled relative difference within max(1 %, 2 SE), the
    comparison resolving 1 % (2 SE <= 1 %). With 2048 updates in flight
    these graphs came out 1.95 % above the oracle."""
    from paper_2409_00876_gb300.batch import Batch
    gold = json.load(open(HIGHPATH))
    gs = make_batch(gold["source_workload"], indices=[r["index"] for r in gold["graphs"]])
    for g, rec in zip(gs, gold["graphs"]):
        assert (g.n_nodes, g.n_paths, g.n_steps) == (rec["n_nodes"], rec["n_paths"], rec["n_steps"])
    arr = concat(gs)
    B = Batch.from_arrays(arr)
    runs = []
    for s in gold["seeds"]:
        B.set_coords(arr.init_xy)
        B.layout(gold["iterations"], seeds=s, theta=gold["theta"])
        runs.append([r["mean"] for r in B.stress(gold["stress_samples_per_step"], gold["stress_seed"])])
    B.close()
    got = np.array(runs).T
    ref = np.array([r["stress"] for r in gold["graphs"]])
    rel = (got - ref) / ref.mean(axis=1, keepdims=True)
    per_graph = rel.mean(axis=1)
    se = np.sqrt(np.sum(rel.var(axis=1, ddof=1) / rel.shape[1])) / len(per_graph)
    print("many paths: per-graph differences", np.round(per_graph, 4), "pooled", per_graph.mean(), "2 SE", 2 * se)
    assert 2 * se <= 0.01, se
    assert abs(per_graph.mean()) <= max(0.01, 2 * se), (per_graph, se)


def test_modes_launch_counts_and_graph_replay(small):
    gs, arr, B = small
    B.set_coords(arr.init_xy)
    B.set_option("mode", 0)
    B.set_option("cuda_graph", 1)
    for _ in range(2):
        B.layout(T, seeds=3, theta=THETA)
        assert B.info()["last_launches"] == T
    B.set_option("mode", 2)
    B.layout(T, seeds=3, theta=THETA)
    assert B.info()["last_launches"] == T * len(gs)
    B.set_option("cuda_graph", 0)
    B.layout(T, seeds=3, theta=THETA, iter_end=2)
    assert B.info()["last_launches"] == 2 * len(gs)
    B.set_option("mode", 1)
    B.layout(T, seeds=3, theta=THETA)
    info = B.info()
    assert info["last_launches"] == 1 and info["last_grid"] > 0
    B.set_option("mode", 0)
    B.set_option("cuda_graph", 1)
    st = B.stress(10, 7)
    assert all(np.isfinite(r["mean"]) for r in st)


def test_persistent_split_run_reaches_the_same_quality(small):
    gs, arr, B = small
    B.set_option("mode", 1)
    one = []
    for _ in range(2):
        B.set_coords(arr.init_xy)
        B.layout(T, seeds=4, theta=THETA)
        one.append(np.mean([r["mean"] for r in B.stress(20, 7)]))
    B.set_coords(arr.init_xy)
    B.layout(T, seeds=4, theta=THETA, iter_end=11)
    B.layout(T, seeds=4, theta=THETA, iter_begin=11)
    two = np.mean([r["mean"] for r in B.stress(20, 7)])
    spread = max(abs(one[0] - one[1]), 0.05 * np.mean(one))
    assert abs(two - np.mean(one)) <= 2 * spread, (two, one)
    B.set_option("mode", 0)


def test_persistent_wait_expires_with_etimeout_and_context_survives(small):
    from paper_2409_00876_gb300 import PgsgdError
    from paper_2409_00876_gb300._native import PGSGD_ETIMEOUT
    gs, arr, B = small
    B.set_option("mode", 1)
    B.set_option("timeout_ms", 200)
    B.set_option("stall_test", 1)
    B.set_coords(arr.init_xy)
    t0 = time.time()
    with pytest.raises(PgsgdError) as ei:
        B.layout(T, seeds=1, theta=THETA)
    assert ei.value.status == PGSGD_ETIMEOUT
    assert time.time() - t0 < 30
    B.set_option("stall_test", 0)
    B.set_option("timeout_ms", 10000)
    # the context is usable: a full persistent layout runs to the end and
    # reaches the oracle's quality on every graph
    gold = _gold()
    B.set_coords(arr.init_xy)
    B.layout(T, seeds=1, theta=THETA)
    st = np.array([r["mean"] for r in B.stress(gold["stress_samples_per_step"], gold["stress_seed"])])
    ref = np.array([np.mean(r["stress"]) for r in gold["graphs"]])
    # one run per graph varies by tens of percent on the smallest graphs:
    # judge the pooled ratio, and only gross failure graph by graph
    ratio = st / ref
    assert np.all(np.isfinite(st)) and 0.8 < ratio.mean() < 1.25 and np.all(ratio < 2.5), (st, ref)
    B.set_option("mode", 0)


def test_graphs_without_moves_or_work_device_inputs_and_mixed_sizes():
    import torch
    from paper_2409_00876_gb300.batch import Batch
    one_step = make_custom([5, 7], [[(0, 0)], []])   # updates drawn, all skipped (no path of two steps)
    empty = make_custom([3], [[]])                    # no steps: no updates, no queue work
    gs = [make_graph("tiny"), one_step, empty, make_graph("tiny", gen_seed=9, backbone=500, paths=3)]
    arr = concat(gs)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for mode in (0, 1, 2):
        B = Batch(arr.graph_node_off, arr.graph_path_off, dev(arr.node_len), dev(arr.path_off),
                  dev(arr.step_node), dev(arr.step_rev), dev(arr.step_pos))
        B.set_option("mode", mode)
        B.set_coords(arr.init_xy)
        init = B.stress(50, 7)
        B.layout(T, seeds=[1, 2, 3, 4], theta=THETA)
        xy = B.get_coords()
        for k in (1, 2):
            np.testing.assert_array_equal(arr.graph_xy(xy, k), arr.graph_xy(arr.init_xy, k))
        st = B.stress(50, 7)
        assert st[1]["n_valid"] == 0 and st[2]["n_valid"] == 0
        assert st[0]["mean"] < 0.5 * init[0]["mean"] and st[3]["mean"] < init[3]["mean"], (st, init)


def test_create_rejects_a_node_outside_its_graph():
    import torch
    from paper_2409_00876_gb300 import PgsgdError
    from paper_2409_00876_gb300.batch import Batch
    gs = [make_graph("tiny"), make_graph("tiny", gen_seed=4, backbone=300, paths=2)]
    arr = concat(gs)
    bad = arr.step_node.copy()
    s = int(arr.path_off[arr.graph_path_off[1]]) + 10   # a step of graph 1
    bad[s] = gs[1].n_nodes                               # valid globally, not in graph 1
    with pytest.raises(PgsgdError, match="outside"):
        Batch(arr.graph_node_off, arr.graph_path_off, arr.node_len, arr.path_off, bad, arr.step_rev, arr.step_pos)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with pytest.raises(PgsgdError, match="outside"):
        Batch(arr.graph_node_off, arr.graph_path_off, dev(arr.node_len), dev(arr.path_off), dev(bad),
              dev(arr.step_rev), dev(arr.step_pos))
    with pytest.raises(PgsgdError):
        Batch(arr.graph_node_off[::-1].copy(), arr.graph_path_off, arr.node_len, arr.path_off, arr.step_node,
              arr.step_rev, arr.step_pos)


def test_batch_layout_rejects_bad_learning_rates_before_any_move():
    from paper_2409_00876_gb300 import PgsgdError
    from paper_2409_00876_gb300.batch import Batch
    gs = [make_graph("tiny"), make_graph("tiny", gen_seed=4, backbone=300, paths=2)]
    arr = concat(gs)
    B = Batch.from_arrays(arr)
    B.set_coords(arr.init_xy)
    before = B.get_coords()
    eta = np.tile(np.geomspace(100.0, 0.01, T), (2, 1))
    for v in [np.nan, -1.0, np.inf]:
        bad = eta.copy()
        bad[1, 4] = v
        with pytest.raises(PgsgdError, match="learning rate"):
            B.layout(T, seeds=[1, 2], eta=bad)
    np.testing.assert_array_equal(B.get_coords(), before)
    B.layout(T, seeds=[1, 2], eta=eta)
    assert not np.array_equal(B.get_coords(), before)


def test_full_batch_in_the_benchmarked_schedule():
    """The 256-graph workload in the autotuned schedule the benchmark times:
    draws of the largest, a middle and the smallest graph are bit-exact with
    the oracle, and after the layout the per-graph stress of those graphs is
    the oracle's statistic of the GPU layout."""
    import torch
    from paper_2409_00876_gb300.batch import Batch, autotune
    gs = make_batch("batch256")
    arr = concat(gs)
    B = Batch.from_arrays(arr)
    xy0 = torch.from_numpy(arr.init_xy).cuda()
    seeds = np.arange(1, len(gs) + 1, dtype=np.uint64)
    autotune(B, xy0, seeds=seeds, iter_max=T, theta=THETA)
    steps = np.array([g.n_steps for g in gs])
    picks = [int(np.argmax(steps)), int(np.argsort(steps)[len(gs) // 2]), int(np.argmin(steps))]
    for k in picks:
        for t in (0, T - 1):
            u0 = int(10 * gs[k].n_steps) - 20_000  # the iteration's last draws
            _same(B.debug_sample(k, t, T, THETA, int(seeds[k]), u0, 20_000),
                  O.sample(gs[k], T, t, THETA, int(seeds[k]), u0, 20_000))
    B.set_coords(xy0)
    init = B.stress(1, 7)
    B.layout(T, seeds=seeds, theta=THETA)
    xy = B.get_coords()
    st = B.stress(1, 7)
    for k in picks:
        want = O.sampled_stress(gs[k], arr.graph_xy(xy, k), per_step=1, seed=7)
        assert st[k]["n_valid"] == want["n_valid"]
        assert abs(st[k]["mean"] - want["mean"]) <= 1e-4 * want["mean"], (k, st[k], want)
    # the generator's initial layouts are already near the backbone order, so
    # PG-SGD (which first scrambles them at a large learning rate) ends near
    # them, not far below: only a blow-up is a failure here; quality against
    # the oracle is checked on the small batch
    m = np.array([r["mean"] for r in st])
    m0 = np.array([r["mean"] for r in init])
    assert np.all(np.isfinite(m)) and np.median(m / m0) < 1.5 and np.all(m < 10 * m0.max())


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_per_graph_learning_rates_reach_their_graphs(mode):
    """Graphs are scheduled in rank order (longest lanes first); the caller's
    per-graph eta rows must still reach the right graphs: a graph given
    eta = 0 in every iteration keeps its layout exactly, the others move."""
    from paper_2409_00876_gb300.batch import Batch
    gs = [make_graph("tiny", gen_seed=s, backbone=b, paths=p) for s, b, p in [(3, 400, 3), (4, 2500, 6), (5, 1200, 4)]]
    arr = concat(gs)
    B = Batch.from_arrays(arr)
    B.set_option("mode", mode)
    eta = np.stack([O.eta_schedule(T, O.default_eta_max(g)) for g in gs])
    for frozen in range(len(gs)):
        e = eta.copy()
        e[frozen] = 0.0
        B.set_coords(arr.init_xy)
        B.layout(T, seeds=[7, 8, 9], eta=e, theta=THETA)
        xy = B.get_coords()
        for k in range(len(gs)):
            same = np.array_equal(arr.graph_xy(xy, k), arr.graph_xy(arr.init_xy, k))
            assert same == (k == frozen), (mode, frozen, k)
