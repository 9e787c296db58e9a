"""Pins of the oracle's warp-merging and data-reuse variants (readings of
Section V-B3 and Section VII-D): special cases that reduce to the standard
sampler, group structure, distributions, fixed points and convergence."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from synth import make_custom, make_graph, make_linear_path

T = 30
FIELDS = ["g", "i", "j", "d_ref", "path", "cooling", "e_i", "e_j", "skip"]


@pytest.fixture(scope="module")
def tiny():
    return make_graph("tiny")


def _same(a, b, fields=FIELDS):
    for f in fields:
        np.testing.assert_array_equal(a[f], b[f], err_msg=f)


def test_warp_merging_off_is_the_standard_sampler(tiny):
    _same(O.sample_wm(tiny, T, 4, 0.99, 11, 12345, 20_000, wm=0), O.sample(tiny, T, 4, 0.99, 11, 12345, 20_000))


def test_warp_merging_takes_the_coin_of_the_group_leader(tiny):
    t = 3  # before the forced-cooling half
    n = 32 * 2000
    wm = O.sample_wm(tiny, T, t, 0.99, 7, 0, n, wm=1)
    std = O.sample(tiny, T, t, 0.99, 7, 0, n)
    groups = wm["cooling"].reshape(-1, 32)
    assert np.all(groups == groups[:, :1])
    np.testing.assert_array_equal(groups[:, 0], std["cooling"].reshape(-1, 32)[:, 0])
    # where an update's own coin agrees with its group's, it is the standard update
    agree = wm["cooling"] == std["cooling"]
    assert 0.4 < agree.mean() < 0.9
    _same(wm[agree], std[agree])
    # other fields never depend on the coin
    _same(wm, std, ["g", "i", "path", "e_i", "e_j"])
    # the groups' coins are fair
    assert stats.binomtest(int(groups[:, 0].sum()), len(groups), 0.5).pvalue > 1e-3
    # in the cooling half every update takes the power law either way
    late = O.sample_wm(tiny, T, 20, 0.99, 7, 0, 3200, wm=1)
    assert np.all(late["cooling"] == 1)


def test_warp_merging_from_an_unaligned_start(tiny):
    a = O.sample_wm(tiny, T, 2, 0.99, 3, 0, 3200, wm=1)
    b = O.sample_wm(tiny, T, 2, 0.99, 3, 17, 3000, wm=1)
    _same(a[17:3017], b)


@pytest.fixture(scope="module")
def reuse(tiny):
    n_sel = O.n_selections(tiny, 10, 2)
    return n_sel, O.sample_reuse(tiny, T, 5, 0.99, 21, 4, n_sel, 0, 32 * 3000)


def test_reuse_groups_share_a_path_and_round_zero_is_the_own_pair(tiny, reuse):
    n_sel, r = reuse
    paths = r["path"].reshape(-1, 32 * 4)
    assert np.all(paths == paths[:, :1])
    # path of a group in proportion to its number of steps
    lens = np.diff(tiny.path_off.astype(np.int64))
    obs = np.bincount(paths[:, 0], minlength=tiny.n_paths)
    exp = lens / lens.sum() * len(paths)
    assert stats.chisquare(obs, exp).pvalue > 1e-4


def test_reuse_rounds_pair_each_lane_with_one_shifted_lane(tiny, reuse):
    n_sel, r = reuse
    G = r.shape[0] // 32
    offs = np.zeros((G, 3), int)
    for gi in range(G):
        blk = r[gi * 32:(gi + 1) * 32]
        own = blk[:, 0]
        for k in range(1, 4):
            found = [o for o in range(1, 32)
                     if np.array_equal(blk[:, k]["j"], np.roll(own["j"], -o))
                     and np.array_equal(blk[:, k]["e_j"], np.roll(own["e_j"], -o))
                     and np.array_equal(blk[:, k]["i"], own["i"])]
            assert found, (gi, k)
            offs[gi, k - 1] = found[0]
    # the offsets are uniform on 1..31
    obs = np.bincount(offs.ravel(), minlength=32)[1:]
    assert stats.chisquare(obs).pvalue > 1e-4


def test_reuse_step_i_is_uniform_on_the_group_path(tiny, reuse):
    n_sel, r = reuse
    own = r[:, 0]
    lens = np.diff(tiny.path_off.astype(np.int64))
    frac = own["i"] / lens[own["path"]]
    obs = np.histogram(frac, bins=20, range=(0, 1))[0]
    assert stats.chisquare(obs).pvalue > 1e-4


def test_reuse_reference_distances_follow_the_steps(tiny, reuse):
    n_sel, r = reuse
    flat = r.ravel()
    ok = flat["skip"] != 1
    off = tiny.path_off[flat["path"][ok]].astype(np.int64)

    def ep(step, e):
        node = tiny.step_node[step]
        return tiny.step_pos[step] + np.where((e ^ tiny.step_rev[step]) & 1, tiny.node_len[node], 0)

    a = ep(off + flat["i"][ok].astype(np.int64), flat["e_i"][ok])
    b = ep(off + flat["j"][ok].astype(np.int64), flat["e_j"][ok])
    np.testing.assert_array_equal(np.abs(a - b), flat["d_ref"][ok])
    np.testing.assert_array_equal(flat["skip"][ok] == 2, flat["d_ref"][ok] == 0)


def test_reuse_skips_selections_past_the_end(tiny):
    n_sel = 32 * 10 + 7
    r = O.sample_reuse(tiny, T, 5, 0.99, 21, 2, n_sel, 32 * 10, 32)
    assert np.all(r[7:, 0]["skip"] == 1)
    assert np.all(r[:7, 0]["skip"] != 1)


def test_reuse_without_reuse_factor_is_the_standard_layout(tiny):
    a, ma = O.layout_variant(tiny, tiny.init_xy, seed=3, drf=1, srf=1)
    b, mb = O.layout(tiny, tiny.init_xy, T=T, seed=3)
    np.testing.assert_array_equal(a, b)
    assert ma == mb
    # step reduction alone is the standard sampler with fewer updates
    c, mc = O.layout_variant(tiny, tiny.init_xy, seed=3, drf=1, srf=4)
    d, md = O.layout(tiny, tiny.init_xy, T=T, seed=3, n_updates=O.n_selections(tiny, 10, 4))
    np.testing.assert_array_equal(c, d)


def test_a_zero_stress_layout_is_a_fixed_point_of_every_variant():
    g = make_linear_path(500, len_mean=8, seed=2, jitter=0.0)
    for drf, srf, wm in [(2, 1, 0), (4, 2, 1), (8, 8, 0)]:
        xy, moved = O.layout_variant(g, g.init_xy, seed=5, drf=drf, srf=srf, wm=wm)
        assert moved > 0
        np.testing.assert_allclose(xy, g.init_xy, rtol=0, atol=1e-7)


@pytest.mark.parametrize("drf,srf", [(2, 2), (4, 1)])
def test_a_linear_path_converges_under_data_reuse(drf, srf):
    g = make_linear_path(3000, len_mean=8, seed=4, jitter=3.0)
    xy, _ = O.layout_variant(g, g.init_xy, seed=3, drf=drf, srf=srf)
    assert O.sampled_stress(g, xy, seed=2)["mean"] < 1e-3


def test_reuse_on_a_graph_with_short_paths():
    g = make_custom([4, 5, 6], [[(0, 0)], [(1, 0), (2, 1)], []])
    n_sel = O.n_selections(g, 10, 1)
    r = O.sample_reuse(g, T, 1, 0.99, 3, 2, n_sel, 0, n_sel)
    one_step = r["path"] == 0
    assert np.all(r["skip"][one_step] == 1)
    # own pairs on the two-step path exist (later rounds may meet lanes past n_sel)
    assert np.all(r[:, 0]["skip"][~one_step[:, 0]] != 1)
    xy, _ = O.layout_variant(g, g.init_xy, drf=2)
    assert np.all(np.isfinite(xy))
