"""Pins for the oracle's differentiable sampled stress and its gradient."""
import numpy as np

import oracle as O
from synth import make_graph


def test_gradient_matches_central_differences_of_the_objective():
    g = make_graph("tiny")
    rng = np.random.default_rng(3)
    xy = g.init_xy + rng.normal(0, 2.0, g.init_xy.shape)
    n, seed = 200_000, 5
    grad = O.dstress_grad(g, xy, n, seed)
    h = 1e-3
    for flat in rng.choice(xy.size, size=60, replace=False):
        v, c = divmod(int(flat), 4)
        xp = xy.copy(); xp[v, c] += h
        xm = xy.copy(); xm[v, c] -= h
        fd = (O.dstress(g, xp, n, seed)[0] - O.dstress(g, xm, n, seed)[0]) / (2 * h)
        assert abs(fd - grad[v, c]) <= 1e-6 * max(1.0, abs(grad).max()) + 1e-4 * abs(grad[v, c]), (v, c, fd, grad[v, c])


def test_objective_estimates_the_sampled_stress_expectation():
    # paths in proportion to |p| and uniform pairs: the same expectation as
    # Eq. 2. The terms are heavy-tailed, so compare medians over sample sets.
    g = make_graph("tiny")
    xy, _ = O.layout(g, g.init_xy, seed=1)
    d = [O.dstress(g, xy, 2_000_000, s)[0] for s in range(5)]
    e = [O.sampled_stress(g, xy, per_step=100, seed=s)["mean"] for s in range(5)]
    assert abs(np.median(d) - np.median(e)) <= 0.1 * np.median(e)


def test_gradient_vanishes_at_an_exact_layout():
    # one forward path laid out at its nucleotide positions: every term is 0
    from synth import make_linear_path
    g = make_linear_path(50, seed=1, jitter=0.0)
    f, _ = O.dstress(g, g.init_xy, 10_000, 1)
    assert f < 1e-20
    assert np.abs(O.dstress_grad(g, g.init_xy, 10_000, 1)).max() < 1e-12
