"""Pins for the oracle's pair sampler (Algorithm 1: path, steps, cooling).

Distributions are checked against their closed forms with chi-square tests;
the reference distance against the hand-worked pair of Fig. 3.
"""
import json
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O
from synth import make_custom

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _chi2_ok(counts, probs, alpha=1e-4):
    counts = np.asarray(counts, dtype=np.float64)
    probs = np.asarray(probs, dtype=np.float64)
    exp = probs / probs.sum() * counts.sum()
    keep = exp > 5
    # lump the small-expectation cells together so chi-square stays valid
    c = np.append(counts[keep], counts[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] == 0:
        c, e = c[:-1], e[:-1]
    stat = ((c - e) ** 2 / e).sum()
    p = stats.chi2.sf(stat, len(c) - 1)
    return p > alpha, p


# ------------------------------------------------------------------ Zipf

@pytest.mark.parametrize("theta", [0.0, 0.5, 0.99, 1.5])
def test_zipf_matches_closed_form_small_support(theta):
    N = 200
    k = O.zipf_sample(theta, N, seed=3, count=400_000)
    assert k.min() >= 1 and k.max() <= N
    counts = np.bincount(k.astype(np.int64), minlength=N + 1)[1:]
    probs = np.arange(1, N + 1, dtype=np.float64) ** -theta
    ok, p = _chi2_ok(counts, probs)
    assert ok, p


def test_zipf_two_point_support_exact_probability():
    # N = 2: P(k = 1) = 1 / (1 + 2^-theta)
    theta = 0.99
    k = O.zipf_sample(theta, 2, seed=9, count=200_000)
    p1 = 1.0 / (1.0 + 2.0 ** -theta)
    frac = np.mean(k == 1)
    assert abs(frac - p1) < 5 * np.sqrt(p1 * (1 - p1) / len(k))


def test_zipf_one_point_support():
    assert np.all(O.zipf_sample(0.99, 1, seed=1, count=1000) == 1)


def test_zipf_log_binned_chromosome_support():
    # the longest synthetic chromosome path has ~5.2 M steps
    N = 5_000_000
    theta = 0.99
    k = O.zipf_sample(theta, N, seed=4, count=1_000_000).astype(np.int64)
    assert k.min() >= 1 and k.max() <= N
    edges = [1 << b for b in range(0, 24)] + [N + 1]
    edges = sorted(set(e for e in edges if e <= N + 1))
    counts = np.histogram(k, bins=edges)[0]
    w = np.arange(1, N + 1, dtype=np.float64) ** -theta
    cw = np.concatenate([[0.0], np.cumsum(w)])
    probs = np.array([cw[b - 1] - cw[a - 1] for a, b in zip(edges[:-1], edges[1:])])
    ok, p = _chi2_ok(counts, probs)
    assert ok, p


# ------------------------------------------------------------------ path / step / cooling

def _graph_with_paths(lengths, node_len=3):
    V = max(lengths) + 1
    paths = [[(v % V, 0) for v in range(n)] for n in lengths]
    return make_custom(np.full(V, node_len, np.uint32), paths)


def test_path_drawn_proportional_to_length_and_step_uniform():
    lengths = [1, 2, 5, 40, 300, 0, 700]
    g = _graph_with_paths(lengths)
    s = O.sample(g, 30, 0, 0.99, 5, 0, 300_000)
    counts = np.bincount(s["path"], minlength=len(lengths))
    ok, p = _chi2_ok(counts[np.array(lengths) > 0], np.array([x for x in lengths if x > 0]))
    assert ok, p
    assert counts[5] == 0  # an empty path is never drawn
    # the global step g is uniform over all steps, i = g - off[p]
    off = g.path_off.astype(np.int64)
    assert np.all(s["i"] == s["g"] - off[s["path"]])
    ok, p = _chi2_ok(np.bincount(s["g"].astype(np.int64), minlength=g.n_steps), np.ones(g.n_steps))
    assert ok, p
    # a single-step path gives no update
    assert np.all(s["skip"][s["path"] == 0] == 1)
    assert np.all(s["skip"][s["path"] != 0] != 1)


@pytest.mark.parametrize("T", [30, 31])
def test_cooling_schedule(T):
    g = _graph_with_paths([50, 80])
    first_cool = (T + 1) // 2  # iter >= N_iters / 2
    for t in range(T):
        s = O.sample(g, T, t, 0.99, 2, 0, 20_000)
        frac = s["cooling"].mean()
        if t >= first_cool:
            assert frac == 1.0
        else:
            assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(len(s))


def test_uniform_pairs_cover_all_ordered_pairs_equally():
    n = 7
    g = _graph_with_paths([n])
    s = O.sample(g, 30, 0, 0.99, 8, 0, 400_000)
    s = s[s["cooling"] == 0]
    assert np.all(s["i"] != s["j"]) and np.all(s["j"] < n)
    cells = np.bincount(s["i"].astype(np.int64) * n + s["j"].astype(np.int64), minlength=n * n)
    cells = cells.reshape(n, n)
    assert np.all(np.diag(cells) == 0)
    off = cells[~np.eye(n, dtype=bool)]
    ok, p = _chi2_ok(off, np.ones_like(off))
    assert ok, p


def test_power_law_pairs_distance_distribution():
    # interior i far from both ends: |j - i| follows Zipf(theta) on [1, n-1] exactly
    n = 4001
    g = _graph_with_paths([n])
    T = 30
    s = O.sample(g, T, 20, 0.99, 3, 0, 400_000)  # t >= T/2: all cooling
    assert np.all(s["cooling"] == 1)
    assert np.all(s["i"] != s["j"]) and np.all(s["j"] < n)
    k = np.abs(s["j"].astype(np.int64) - s["i"].astype(np.int64))
    i = s["i"].astype(np.int64)
    # rows where both directions are inside the path for every k <= 100
    inner = (i >= 100) & (i <= n - 1 - 100) & (k <= 100)
    counts = np.bincount(k[inner], minlength=101)[1:]
    probs = np.arange(1, 101, dtype=np.float64) ** -0.99
    ok, p = _chi2_ok(counts, probs)
    assert ok, p
    # direction is a fair coin where both are possible
    fwd = (s["j"].astype(np.int64) > i)[inner]
    assert abs(fwd.mean() - 0.5) < 5 * 0.5 / np.sqrt(fwd.size)


def test_two_step_path_always_pairs_the_two_steps():
    g = _graph_with_paths([2])
    for t in (0, 29):
        s = O.sample(g, 30, t, 0.99, 4, 0, 5000)
        assert np.all(s["i"] + s["j"] == 1)


def test_power_law_partner_is_proportional_to_distance_power_over_the_path():
    # P(j | i) proportional to |j - i|^-theta over the path's other steps,
    # near the ends as well: no mass piles up on the end steps
    n = 60
    g = _graph_with_paths([n])
    s = O.sample(g, 30, 20, 0.99, 8, 0, 2_000_000)
    i = s["i"].astype(np.int64)
    j = s["j"].astype(np.int64)
    assert np.all((j >= 0) & (j < n) & (j != i))
    for i0 in (0, 1, 7, 30, 58, 59):
        sel = i == i0
        counts = np.bincount(j[sel], minlength=n).astype(np.float64)
        others = np.arange(n) != i0
        probs = np.abs(np.arange(n) - i0)[others].astype(np.float64) ** -0.99
        ok, p = _chi2_ok(counts[others], probs)
        assert ok, (i0, p)


def test_power_law_partner_on_a_three_step_path():
    # from the middle step only k = 1 fits: either neighbour, equally often
    g = _graph_with_paths([3])
    s = O.sample(g, 30, 25, 0.99, 6, 0, 50_000)
    mid = s["i"] == 1
    assert np.all(np.isin(s["j"][mid], [0, 2]))
    assert abs((s["j"][mid] == 2).mean() - 0.5) < 5 * 0.5 / np.sqrt(mid.sum())
    # from an end, the partner is the middle step (k = 1) or the other end (k = 2)
    end = s["i"] == 0
    w = np.array([1.0, 2.0 ** -0.99])
    ok, p = _chi2_ok([np.sum(s["j"][end] == 1), np.sum(s["j"][end] == 2)], w)
    assert ok, p


def test_reference_distance_fig3_worked_pair():
    with open(os.path.join(GOLDEN, "fig3_pair.json")) as f:
        gold = json.load(f)
    for rev_j in (0, 1):
        g = make_custom(gold["node_len"], [[(0, 0), (1, rev_j)]])
        s = O.sample(g, 30, 0, 0.99, 12, 0, 4000)
        s = s[s["skip"] != 1]
        for case in gold["cases"]:
            if case["rev_j"] != rev_j:
                continue
            # orient the record as (step 0, step 1)
            first_is_i = s["i"] == 0
            e0 = np.where(first_is_i, s["e_i"], s["e_j"])
            e1 = np.where(first_is_i, s["e_j"], s["e_i"])
            sel = (e0 == case["e_i"]) & (e1 == case["e_j"])
            assert sel.sum() > 100
            assert np.all(s["d_ref"][sel] == case["d_ref"])
            want_skip = 2 if case["d_ref"] == 0 else 0
            assert np.all(s["skip"][sel] == want_skip)
