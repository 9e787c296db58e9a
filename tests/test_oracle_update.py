"""Pins for the oracle's update rule, schedule and layout loop (Algorithm 1:
the learning rate per iteration and the pair update, with the update of Zheng
et al. that Fig. 3 illustrates)."""
import numpy as np
import pytest

import oracle as O
from synth import make_custom, make_graph, make_linear_path


def _pair_stress(vi, vj, d):
    # Algorithm 1's move
    return ((np.hypot(vi[0] - vj[0], vi[1] - vj[1]) - d) / d) ** 2


def _first_valid(g, T, t, seed, want=None):
    s = O.sample(g, T, t, 0.99, seed, 0, 2000)
    for u, r in enumerate(s):
        if r["skip"] == 0 and (want is None or want(r)):
            return u, r
    raise AssertionError("no valid update")


def _points(g, xy, r):
    off = int(g.path_off[r["path"]])
    ni = int(g.step_node[off + int(r["i"])])
    nj = int(g.step_node[off + int(r["j"])])
    vi = xy[ni, 2 * r["e_i"]: 2 * r["e_i"] + 2].copy()
    vj = xy[nj, 2 * r["e_j"]: 2 * r["e_j"] + 2].copy()
    return ni, nj, vi, vj


def test_two_node_update_at_unit_rate_lands_on_reference_distance():
    g = make_custom([5, 4], [[(0, 0), (1, 0)]],
                    init_xy=np.array([[0.3, -1.2, 6.1, 2.0], [4.0, 7.5, 13.25, -3.0]]))
    u, r = _first_valid(g, 30, 0, 21)
    eta = 1e12  # mu = min(eta / d^2, 1) = 1
    delta = O.sweep(g, g.init_xy, 30, 0, eta, 0.99, 21, u, 1)[0]
    _, _, vi, vj = _points(g, g.init_xy, r)
    vi2, vj2 = vi + delta[:2], vj + delta[2:]
    assert abs(np.hypot(*(vi2 - vj2)) - r["d_ref"]) <= 4e-16 * r["d_ref"] * 4
    # both points move by the same amount in opposite directions along vi - vj
    assert np.allclose(delta[:2], -delta[2:], rtol=0, atol=1e-15)
    cross = (vi - vj)[0] * delta[1] - (vi - vj)[1] * delta[0]
    assert abs(cross) < 1e-12 * np.linalg.norm(vi - vj) * np.linalg.norm(delta[:2]) + 1e-300


def test_update_is_quarter_rate_gradient_step_when_uncapped():
    # move of v_i = -(eta / 4) d stress_ij / d v_i while eta / d^2 < 1
    g = make_custom([40, 30], [[(0, 0), (1, 0)]],
                    init_xy=np.array([[0.0, 0.0, 47.0, 5.0], [41.0, -3.0, 66.0, 9.0]]))
    u, r = _first_valid(g, 30, 0, 5)
    d = float(r["d_ref"])
    eta = 0.3 * d * d
    delta = O.sweep(g, g.init_xy, 30, 0, eta, 0.99, 5, u, 1)[0]
    _, _, vi, vj = _points(g, g.init_xy, r)
    h = 1e-5
    grad_i = np.zeros(2)
    grad_j = np.zeros(2)
    for a in range(2):
        e = np.zeros(2)
        e[a] = h
        grad_i[a] = (_pair_stress(vi + e, vj, d) - _pair_stress(vi - e, vj, d)) / (2 * h)
        grad_j[a] = (_pair_stress(vi, vj + e, d) - _pair_stress(vi, vj - e, d)) / (2 * h)
    np.testing.assert_allclose(delta[:2], -(eta / 4) * grad_i, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(delta[2:], -(eta / 4) * grad_j, rtol=1e-6, atol=1e-9)


def test_coincident_points_do_not_move():
    g = make_custom([5, 4], [[(0, 0), (1, 0)]],
                    init_xy=np.array([[1.0, 1.0, 1.0, 1.0], [1.0, 1.0, 1.0, 1.0]]))
    d = O.sweep(g, g.init_xy, 30, 0, 1e9, 0.99, 3, 0, 500)
    assert np.all(d == 0)


def test_sweep_matches_one_sequential_update():
    g = make_graph("tiny")
    s = O.sample(g, 30, 3, 0.99, 9, 0, 50)
    u = int(np.nonzero(s["skip"] == 0)[0][0])
    eta = O.eta_schedule(30, O.default_eta_max(g))
    xy1, moved = O.layout(g, g.init_xy, T=30, eta=eta, theta=0.99, seed=9, t_begin=3, t_end=4,
                          n_updates=u + 1)
    assert moved == 1
    d = O.sweep(g, g.init_xy, 30, 3, eta[3], 0.99, 9, u, 1)[0]
    ni, nj, vi, vj = _points(g, g.init_xy, s[u])
    want = g.init_xy.copy()
    want[ni, 2 * s[u]["e_i"]: 2 * s[u]["e_i"] + 2] += d[:2]
    want[nj, 2 * s[u]["e_j"]: 2 * s[u]["e_j"] + 2] += d[2:]
    np.testing.assert_array_equal(xy1, want)


def test_eta_schedule_closed_form():
    T, emax, emin = 30, 1.7e8, 0.01
    eta = O.eta_schedule(T, emax, emin)
    assert eta[0] == emax
    assert abs(eta[-1] - emin) <= 1e-12 * emin
    ratios = eta[1:] / eta[:-1]
    np.testing.assert_allclose(ratios, (emin / emax) ** (1 / (T - 1)), rtol=1e-12)


def test_linear_path_converges_to_a_straight_line():
    # one forward path: the exact zero-stress layout exists (x = nucleotide position)
    g = make_linear_path(300, len_mean=8, seed=4, jitter=3.0)
    before = O.sampled_stress(g, g.init_xy, seed=2)["mean"]
    xy, _ = O.layout(g, g.init_xy, T=30, theta=0.99, seed=3)
    after = O.sampled_stress(g, xy, seed=2)["mean"]
    assert after < 1e-3 < before


def test_layout_lowers_stress_on_tiny_pangenome():
    g = make_graph("tiny")
    before = O.sampled_stress(g, g.init_xy, seed=2)["mean"]
    xy, moved = O.layout(g, g.init_xy, T=30, theta=0.99, seed=1)
    after = O.sampled_stress(g, xy, seed=2)["mean"]
    assert after < 0.5 * before
    assert 0 < moved <= 30 * 10 * g.n_steps


@pytest.mark.parametrize("n_threads", [2, 4])
def test_threaded_hogwild_reaches_same_quality(n_threads):
    g = make_graph("tiny")
    xy1, _ = O.layout(g, g.init_xy, seed=1)
    xyn, _ = O.layout(g, g.init_xy, seed=1, n_threads=n_threads)
    s1 = O.sampled_stress(g, xy1, seed=2)["mean"]
    sn = O.sampled_stress(g, xyn, seed=2)["mean"]
    assert abs(sn - s1) < 0.5 * s1


def test_too_little_randomness_does_not_converge():
    # Section III-C: fewer, more local updates leave the layout far worse
    g = make_graph("tiny")
    full, _ = O.layout(g, g.init_xy, seed=1)
    few, _ = O.layout(g, g.init_xy, seed=1, n_updates=g.n_steps // 10)
    assert O.sampled_stress(g, few, seed=2)["mean"] > 1.5 * O.sampled_stress(g, full, seed=2)["mean"]
