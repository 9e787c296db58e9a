"""Warp merging and warp-level data reuse on the GPU against the oracle's
mirrors: bit-exact draws, the kernels' updates against the oracle's on
sparse iterations (where no two updates share a node, order cannot matter),
and layout quality under the same seeds."""
import numpy as np
import pytest

import oracle as O
from synth import make_graph

pytestmark = pytest.mark.gpu

T = 30
FIELDS = ["g", "i", "j", "d_ref", "path", "cooling", "e_i", "e_j", "skip"]


@pytest.fixture(scope="module")
def pg():
    import paper_2409_00876_gb300 as pg
    pg.load_library()
    return pg


@pytest.fixture(scope="module")
def mid():
    return make_graph("mid")


def _same(a, b):
    for f in FIELDS:
        np.testing.assert_array_equal(a[f], b[f], err_msg=f)


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_warp_merged_draws_are_bit_exact(pg, name):
    g = make_graph(name)
    G = pg.Graph.from_synth(g)
    G.set_option("warp_merge", 1)
    for t, u0 in [(0, 0), (7, 32 * 1000), (14, 12345), (20, 999)]:
        _same(G.debug_sample(t, T, 0.99, 5, u0, 40_000), O.sample_wm(g, T, t, 0.99, 5, u0, 40_000, wm=1))


@pytest.mark.parametrize("drf,srf,wm", [(2, 1, 0), (4, 3, 1), (8, 8, 0)])
def test_reuse_draws_are_bit_exact(pg, mid, drf, srf, wm):
    G = pg.Graph.from_synth(mid)
    G.set_option("drf", drf)
    G.set_option("srf", srf)
    G.set_option("warp_merge", wm)
    n_sel = O.n_selections(mid, 10, srf)
    for t, q0, count in [(2, 0, 8192), (16, 32 * 777 + 5, 5000), (29, n_sel - 3000, 3000 + 40)]:
        got = G.debug_sample_reuse(t, T, 0.99, 9, q0, count)
        want = O.sample_reuse(mid, T, t, 0.99, 9, drf, n_sel, q0, count, wm=wm)
        _same(got.ravel(), want.ravel())


def _sparse_iteration(pg, g, drf, wm, srf, t=10, seed=3, **opts):
    """One iteration with so few updates that nodes rarely meet twice: GPU
    kernel vs the oracle's sequential mirror from the same layout."""
    G = pg.Graph.from_synth(g)
    G.set_option("drf", drf)
    G.set_option("srf", srf)
    G.set_option("warp_merge", wm)
    for k, v in opts.items():
        G.set_option(k, v)
    G.set_coords(g.init_xy)
    G.layout(T, theta=0.99, seed=seed, iter_begin=t, iter_end=t + 1)
    got = G.get_coords()
    n_units = O.n_selections(g, 10, srf)
    want, moved = O.layout_variant(g, g.init_xy, T=T, seed=seed, t_begin=t, t_end=t + 1, drf=drf, wm=wm,
                                   n_units=n_units)
    return got, want, moved


@pytest.mark.parametrize("drf,wm,opts", [
    (1, 0, {}), (1, 1, {}), (2, 0, {}), (4, 1, {}), (8, 0, {}),
    # the other compiled shapes of the plain update loop (the default is the pipelined one at 2)
    (1, 0, dict(pipeline=0, updates_per_thread=1)), (1, 0, dict(pipeline=1, updates_per_thread=1)),
    (1, 0, dict(pipeline=1, updates_per_thread=2)), (1, 0, dict(pipeline=1, updates_per_thread=2, min_blocks=3)),
    (1, 0, dict(pipeline=1, updates_per_thread=4, min_blocks=2)),
    (1, 0, dict(pipeline=0, min_blocks=6)), (1, 0, dict(pipeline=0, updates_per_thread=2, min_blocks=1)),
    (1, 0, dict(pipeline=0, updates_per_thread=2)), (1, 0, dict(pipeline=0, updates_per_thread=4)),
    (1, 0, dict(pipeline=0, min_blocks=1)), (1, 1, dict(updates_per_thread=4)),
    # the asynchronous step-record loop: one block of 256 threads, so every thread
    # runs 4 updates and cycles through its slots
    (1, 0, dict(async_depth=2, max_concurrent=256)), (1, 0, dict(async_depth=3, max_concurrent=256)),
    (1, 0, dict(async_depth=4, max_concurrent=256)), (1, 0, dict(async_depth=6, max_concurrent=256)),
    (1, 0, dict(async_depth=8, max_concurrent=256)), (1, 0, dict(async_depth=4, min_blocks=3)),
    (1, 0, dict(async_depth=4, min_blocks=5)),
])
def test_kernel_updates_match_the_oracle_on_a_sparse_iteration(pg, mid, drf, wm, opts):
    srf = -(-10 * mid.n_steps // 1024)  # about 1024 selections on 220 k nodes
    got, want, moved = _sparse_iteration(pg, mid, drf, wm, srf, **opts)
    assert moved > 0.5 * 1024 * drf
    init = mid.init_xy
    gpu_touched = np.any(got != init, axis=1)
    orc_touched = np.any(np.abs(want - init) > 1e-9, axis=1)
    # the same nodes move (a move can round to nothing in FP32 only rarely)
    assert (gpu_touched != orc_touched).sum() <= 1e-3 * orc_touched.sum() + 2
    close = np.all(np.abs(got - want) <= 1e-2 + 1e-5 * np.abs(want), axis=1)
    frac = close[orc_touched].mean()
    print("drf", drf, "wm", wm, opts, "touched", orc_touched.sum(), "close", frac)
    assert frac >= 0.99, frac


@pytest.mark.parametrize("drf,srf,wm", [(1, 1, 1), (2, 2, 0), (4, 4, 0)])
def test_layout_quality_matches_the_oracle_mirror(pg, drf, srf, wm):
    g = make_graph("tiny")
    ref, got = [], []
    for seed in range(1, 6):
        xy, _ = O.layout_variant(g, g.init_xy, T=T, seed=seed, drf=drf, srf=srf, wm=wm)
        ref.append(O.sampled_stress(g, xy, seed=7)["mean"])
        G = pg.Graph.from_synth(g)
        G.set_option("drf", drf)
        G.set_option("srf", srf)
        G.set_option("warp_merge", wm)
        G.set_coords(g.init_xy)
        G.layout(T, theta=0.99, seed=seed)
        got.append(G.stress(100, seed=7)["mean"])
    ref, got = np.array(ref), np.array(got)
    se = np.hypot(ref.std(ddof=1), got.std(ddof=1)) / np.sqrt(len(ref))
    print(drf, srf, wm, got.mean(), ref.mean(), se)
    assert abs(got.mean() - ref.mean()) <= max(0.01 * ref.mean(), 3 * se), (got, ref)


def test_variant_options_are_checked(pg):
    from paper_2409_00876_gb300 import PgsgdError
    g = make_graph("tiny")
    G = pg.Graph.from_synth(g)
    for name, bad in [("drf", 3), ("drf", 16), ("srf", 0)]:
        with pytest.raises(PgsgdError):
            G.set_option(name, bad)
    G.set_coords(g.init_xy)
    G.set_option("drf", 2)
    G.set_option("pipeline", 1)  # set by hand: an error, since data reuse runs the plain loop
    with pytest.raises(PgsgdError, match="pipeline"):
        G.layout(T)
    G.set_option("pipeline", -1)  # automatic: the plain loop under data reuse
    G.layout(T, iter_end=1)
    for name, bad in [("pipeline", 2), ("pipeline", -2), ("updates_per_thread", 3)]:
        with pytest.raises(PgsgdError):
            G.set_option(name, bad)
    G.set_option("pipeline", 0)
    G.set_option("drf", 1)
    with pytest.raises(PgsgdError, match="reuse is off"):
        G.debug_sample_reuse(0, T, 0.99, 1, 0, 10)
    with pytest.raises(PgsgdError, match="async depth"):
        G.set_option("async_depth", 5)
    G.set_option("async_depth", 4)
    G.set_option("updates_per_thread", 2)
    with pytest.raises(PgsgdError, match="one update per thread"):
        G.layout(T)
