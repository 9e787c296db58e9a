"""Host-side logic of the batched layout (no GPU): the batch generator, its
concatenation, and the schedule plan the library computes on the host."""
import numpy as np
import pytest

from synth import batch_shapes, concat, make_batch, make_graph


def test_batch_shapes_follow_the_workload_ranges():
    sh = batch_shapes(256, (1_000, 200_000), (4, 90), 11)
    v = np.array([a for a, _, _ in sh])
    p = np.array([b for _, b, _ in sh])
    assert len(sh) == 256
    assert v.min() >= 1_000 and v.max() <= 200_000
    assert p.min() >= 4 and p.max() <= 90
    # log-uniform: about half the graphs below the geometric midpoint
    mid = np.sqrt(1_000 * 200_000)
    assert 0.4 < np.mean(v < mid) < 0.6
    assert len({s for _, _, s in sh}) == 256


def test_concat_keeps_every_graph_intact():
    gs = make_batch("batch_small")
    b = concat(gs)
    assert b.n_graphs == len(gs)
    for k, g in enumerate(gs):
        n0, n1 = int(b.graph_node_off[k]), int(b.graph_node_off[k + 1])
        p0, p1 = int(b.graph_path_off[k]), int(b.graph_path_off[k + 1])
        assert n1 - n0 == g.n_nodes and p1 - p0 == g.n_paths
        s0, s1 = int(b.path_off[p0]), int(b.path_off[p1])
        np.testing.assert_array_equal(b.path_off[p0:p1 + 1] - b.path_off[p0], g.path_off)
        np.testing.assert_array_equal(b.step_node[s0:s1], g.step_node)
        np.testing.assert_array_equal(b.step_pos[s0:s1], g.step_pos)
        np.testing.assert_array_equal(b.node_len[n0:n1], g.node_len)
        np.testing.assert_array_equal(b.graph_xy(b.init_xy, k), g.init_xy)
    # node counts near the requested ones (backbone plus about 10 % bubble nodes)
    want = [v for v, _, _ in batch_shapes(12, (1_000, 12_000), (4, 12), 5)]
    got = [g.n_nodes for g in gs]
    assert np.all(np.abs(np.array(got) / np.array(want) - 1) < 0.05)


def _plan(*a, **k):
    from paper_2409_00876_gb300.batch import plan
    return plan(*a, **k)


def test_plan_orders_by_work_and_caps_lanes():
    nu = np.array([100, 0, 5000, 5000, 70000], np.uint64)
    nn = np.array([10, 5, 4000, 100000, 3000], np.uint64)
    r2g, nch, lanes, thr = _plan(nu, nn, block=256, updates_per_thread=2, chunk=1000)
    # longest lanes first (rounds 547, 27, then 2 and 2 broken by most updates, then 0)
    assert list(r2g) == [4, 2, 3, 0, 1]
    np.testing.assert_array_equal(nch, [1, 0, 5, 5, 70])
    # cap = max(64, V / 16, N / 5120) updates in flight = cap // 512 chunks, at most the chunks there are
    cap = np.maximum(64, np.maximum(nn // 16, nu // 5120))
    np.testing.assert_array_equal(lanes, np.where(nch == 0, 0, np.minimum(np.maximum(cap // 512, 1), nch)))
    # a cap below one block's worth (512 updates) runs on whole warps: max(32, cap / 2) rounded down to 32
    np.testing.assert_array_equal(thr, np.where(cap < 512, np.maximum(32, cap // 2 // 32 * 32), 256))
    assert list(thr) == [32, 32, 96, 256, 64]


def test_plan_starts_the_longest_lanes_first():
    # a small graph with many paths per node runs one lane of 5,209 rounds
    # (cap 1 M / 5120 = 195 updates: 96 threads x 2); the large graph 122
    # lanes of 160 rounds: the small graph ranks first despite fewer updates
    r2g, nch, lanes, thr = _plan(np.array([10_000_000, 1_000_000], np.uint64),
                                 np.array([1_000_000, 1_000], np.uint64))
    assert list(lanes) == [122, 1] and list(thr) == [256, 96]
    assert list(r2g) == [1, 0]


def test_plan_options_change_lanes():
    nu = np.array([10_000_000], np.uint64)
    nn = np.array([200_000], np.uint64)
    _, nch, lanes, thr = _plan(nu, nn, block=128, updates_per_thread=4, chunk=4096)
    assert nch[0] == -(-10_000_000 // 4096)
    assert lanes[0] == 12_500 // 512 and thr[0] == 128  # cap V / 16 = 12,500 updates over 128 x 4 per lane
    _, _, lanes0, thr0 = _plan(nu, nn, chunk=4096, max_concurrent=0)
    assert lanes0[0] == nch[0] and thr0[0] == 256  # no cap: every chunk may run at once on whole blocks
    _, _, lanes1, thr1 = _plan(nu, nn, chunk=4096, max_concurrent=100)
    assert lanes1[0] == 1 and thr1[0] == 32  # 100 updates at 2 per thread: one warp
    # many updates per node: the N / 5120 term sets the cap (10 M / 5120 = 1953 > 1000 / 16)
    _, _, lanes2, thr2 = _plan(nu, [1000], chunk=4096)
    assert lanes2[0] == 1953 // 512 and thr2[0] == 256


@pytest.mark.parametrize("kw", [dict(block=48), dict(block=288), dict(updates_per_thread=3), dict(chunk=0),
                                dict(max_concurrent=-2)])
def test_plan_rejects_bad_options(kw):
    from paper_2409_00876_gb300 import PgsgdError
    with pytest.raises(PgsgdError):
        _plan([10], [10], **kw)


def test_batch_of_one_graph_matches_its_arrays():
    g = make_graph("tiny")
    b = concat([g])
    np.testing.assert_array_equal(b.path_off, g.path_off)
    assert list(b.graph_node_off) == [0, g.n_nodes]


class _FakeBatch:
    """Stands in for a Batch on the CPU: the time of a layout is a made-up
    function of the options, so the autotuner's search can be checked."""

    def __init__(self, landscape, start):
        self.opts = dict(start, timing=0)
        self.landscape = landscape
        self.calls = 0
        self._ms = 0.0

    def get_option(self, k):
        return self.opts[k]

    def set_option(self, k, v):
        self.opts[k] = v

    def set_coords(self, xy):
        pass

    def layout(self, *a, **k):
        self.calls += 1
        self._ms = self.landscape(self.opts)

    def timing_read(self, reset=True):
        ms, self._ms = self._ms, 0.0
        return ms, 1, 1


def test_autotune_descends_to_the_best_schedule_and_leaves_it_set():
    from paper_2409_00876_gb300.batch import autotune
    space = dict(mode=[0, 1], pipeline=[0, 1], updates_per_thread=[2, 1, 4], block=[256, 128],
                 chunk=[16384, 4096, 65536])
    best = dict(mode=1, pipeline=0, updates_per_thread=4, block=128, chunk=65536)
    cost = dict(mode=3.0, pipeline=1.0, updates_per_thread=2.0, block=0.5, chunk=0.25)

    def landscape(o):  # separable: every coordinate off its best value adds its own penalty
        return 100.0 + sum(0.0 if o[k] == best[k] else cost[k] for k in space)

    b = _FakeBatch(landscape, dict(mode=0, pipeline=0, updates_per_thread=2, block=256, chunk=16384))
    got, table = autotune(b, None, space=space)
    assert got == best
    assert {k: b.opts[k] for k in space} == best
    assert b.opts["timing"] == 0
    # every trial timed once after one untimed run; no trial repeated
    assert len(table) == len(set(table))
    assert b.calls == 2 * len(table)
