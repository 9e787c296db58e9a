"""Exhaustive pin of the oracle's power-law trial (the Zipf draw behind
Algorithm 1's power-law partner, Section V-B3's cooling branch).

One rejection-inversion trial (Hoermann and Derflinger, ACM TOMACS 1996)
reads only bits 8-31 of its word, so its whole behaviour is the 2^24 values
of those bits: orc_zipf_trials runs the trial on every one of them. In exact
arithmetic, with U uniform on [0, 1), u = B + U (A - B) is uniform on an
interval of length D = B - A (A = H(3/2) - h(1), B = H(N + 1/2),
H(x) = (x^(1-theta) - 1) / (1 - theta), h(k) = k^-theta), and the trial
accepts k <= 255 on a u-interval of length exactly h(k); draws with
k >= 256 are accepted without the test, on the u-interval of x in
[k - 1/2, k + 1/2), of length H(k + 1/2) - H(k - 1/2). On the grid of 2^24
words the exact count of bin k is therefore 2^24 h(k) / D to within one word
at each end of its interval. The binary32 trial is checked against those
exact counts bin by bin, and through its cumulative distribution over the
whole support, for theta in {0.5, 0.99, 1.5} and N in {10, 1000, 5e6}.
Bounds: 4 words per bin (one for the grid and up to three for the binary32
rounding of a boundary), and 3 words per rejection interval plus 4 for the
cumulative count (the k <= 255 bins each add their own boundary errors).
"""
import numpy as np
import pytest

import oracle as O

M = 1 << 24
CASES = [(th, N) for th in (0.5, 0.99, 1.5) for N in (10, 1000, 5_000_000)]


def _H(x, theta):
    x = np.asarray(x, dtype=np.float64)
    return np.log(x) if theta == 1.0 else np.expm1((1.0 - theta) * np.log(x)) / (1.0 - theta)


def _exact_mass(theta, N):
    """u-length of the accepted region of every bin k = 1..N, and D."""
    A = float(_H(1.5, theta)) - 1.0
    B = float(_H(N + 0.5, theta))
    k = np.arange(1, N + 1, dtype=np.float64)
    mass = k ** -theta
    if N > 255:
        edges = np.concatenate([[255.5], k[255:] + 0.5])
        mass[255:] = np.diff(_H(edges, theta))
    return mass, B - A


@pytest.fixture(scope="module", params=CASES, ids=[f"theta{t}-N{n}" for t, n in CASES])
def enumerated(request):
    theta, N = request.param
    k = O.zipf_trials(theta, N)
    assert k.shape == (M,) and int(k.max()) <= N
    counts = np.bincount(k.astype(np.int64), minlength=N + 1)
    mass, D = _exact_mass(theta, N)
    return theta, N, counts, mass, D


def test_every_bin_below_256_holds_its_exact_share_of_the_words(enumerated):
    theta, N, counts, mass, D = enumerated
    K0 = min(N, 255)
    exact = M * mass[:K0] / D
    dev = np.abs(counts[1:K0 + 1] - exact)
    assert dev.max() <= 4.0, (int(np.argmax(dev)) + 1, dev.max())


def test_cumulative_distribution_over_the_whole_support(enumerated):
    theta, N, counts, mass, D = enumerated
    F = np.cumsum(counts[1:]).astype(np.float64)
    Fx = M * np.cumsum(mass) / D
    bound = 3.0 * np.minimum(np.arange(1, N + 1), 255) + 4.0
    assert np.all(np.abs(F - Fx) <= bound), float(np.max(np.abs(F - Fx) - bound))


def test_accepted_draws_follow_k_to_the_minus_theta(enumerated):
    """The accepted k against the target law k^-theta / H_N: bins below 256
    within their count bound, and the tail k >= 256 in total. Accepting the
    tail without the test replaces sum h(k) by the integral of h over
    [255.5, N + 0.5], a relative change below theta / (24 * 255.5^(theta+1))
    of the tail's mass (midpoint rule), taken into the bound."""
    theta, N, counts, mass, D = enumerated
    k = np.arange(1, N + 1, dtype=np.float64)
    target = k ** -theta
    target /= target.sum()
    acc = counts[1:].sum()
    K0 = min(N, 255)
    emp = counts[1:K0 + 1] / acc
    bound = (4.0 + 3.0 * 255 + 4.0) / (M * mass[:K0] / D) + 1e-6
    assert np.all(np.abs(emp / target[:K0] - 1.0) <= bound)
    if N > 255:
        tail_emp = counts[256:].sum() / acc
        tail_target = target[255:].sum()
        slack = (3.0 * 255 + 4.0) / acc + theta / (24 * 255.5 ** (theta + 1)) * tail_target
        assert abs(tail_emp - tail_target) <= 2 * slack + 1e-7, (tail_emp, tail_target)


def test_acceptance_rate_and_the_64_trial_fallback(enumerated):
    """The exact acceptance rate of one trial, and the probability that a
    power-law partner draw runs out of its 64 trials (then j = i +- 1). A
    trial from step i of a path of n = N + 1 steps is accepted when the Zipf
    test accepts and i +- k lies on the path; its direction bit (bit 4) is
    independent of bits 8-31, so at a path end, the worst case, the chance is
    half the acceptance rate."""
    theta, N, counts, mass, D = enumerated
    rate = counts[1:].sum() / M
    exact = mass.sum() / D
    assert abs(rate - exact) <= (3.0 * 255 + 4.0) / M
    worst = 0.5 * rate
    p_fallback = (1.0 - worst) ** 64
    assert rate > 0.98 and p_fallback < 1e-18, (rate, p_fallback)
