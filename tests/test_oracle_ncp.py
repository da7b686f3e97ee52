"""Pins of the oracle's normalized cumulative periodogram (NCP) and of the NCP stopping rule
(Sec. 3.2).

The NCP of a residual row is fixed by closed forms: a pure sinusoid at frequency f puts all
its power in one bin, so its NCP is the step 0 (i < f), 1 (i >= f); adding a constant, scaling
or circularly shifting a row leaves the NCP unchanged (the zero frequency is left out and the
periodogram is shift-invariant); Parseval ties the periodogram's sum to the row's energy.
White Gaussian noise passes the Kolmogorov-Smirnov band at about the nominal rate, smooth and
random-walk residuals fail it.  The stopping rule returns the iterate of the last checked
step before the NCP distance first grows.
"""
import math

import numpy as np
import pytest

import synth
from oracle import proj as P
from oracle import solver as S


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("n", [16, 17, 95, 768])
def test_ncp_of_a_sinusoid_is_a_step(n):
    q = n // 2
    t = np.arange(n)
    for f in sorted({1, 2, q // 2 + 1, q}):
        for phase in (0.0, 0.7):
            row = 3.0 * np.cos(2 * np.pi * f * t / n + phase)
            if 2 * f == n:                     # at the Nyquist frequency only cos survives
                row = 3.0 * np.cos(np.pi * t)
            c = S.ncp(row.reshape(1, -1))
            step = (np.arange(1, q + 1) >= f).astype(float)
            np.testing.assert_allclose(c, step, atol=1e-12)
            d = S.ncp_distance(row.reshape(1, -1))
            np.testing.assert_allclose(d, np.linalg.norm(step - np.arange(1, q + 1) / q),
                                       rtol=1e-12)


def test_ncp_ignores_mean_scale_and_circular_shift():
    rng = _rng(3)
    rows = rng.standard_normal((5, 64)).cumsum(axis=1)
    c = S.ncp(rows)
    np.testing.assert_allclose(S.ncp(rows + 7.5), c, atol=1e-12)
    np.testing.assert_allclose(S.ncp(-4.0 * rows), c, atol=1e-12)
    np.testing.assert_allclose(S.ncp(np.roll(rows, 11, axis=1)), c, atol=1e-12)


@pytest.mark.parametrize("n", [10, 33, 768])
def test_periodogram_obeys_parseval(n):
    """For a real row: sum_{j=1}^{n-1} |r^_j|^2 = n sum r_t^2 - (sum r_t)^2, and the bins above
    q mirror those below, so 2 sum_{j<=q} p_j - [n even] p_{n/2} equals it."""
    rng = _rng(n)
    r = rng.standard_normal((3, n)) + 0.3
    p = S.periodogram(r)
    lhs = 2 * p.sum(axis=1) - (p[:, -1] if n % 2 == 0 else 0.0)
    rhs = n * (r * r).sum(axis=1) - r.sum(axis=1) ** 2
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


def test_ncp_averages_rows_and_skips_rows_without_power():
    n, q = 40, 20
    t = np.arange(n)
    rows = np.stack([np.cos(2 * np.pi * 3 * t / n), np.sin(2 * np.pi * 12 * t / n),
                     np.full(n, 2.0), np.zeros(n)])
    i = np.arange(1, q + 1)
    expect = 0.5 * ((i >= 3).astype(float) + (i >= 12).astype(float))
    np.testing.assert_allclose(S.ncp(rows), expect, atol=1e-12)
    assert S.ncp(np.zeros((2, n))) is None and S.ncp_distance(np.zeros((2, n))) == 0.0


def test_white_noise_passes_and_correlated_residuals_fail_the_ks_band():
    n = 512
    white = [S.ncp_is_white(_rng(s).standard_normal(n)) for s in range(60)]
    assert sum(white) >= 51                    # nominal 95 %: 57 of 60
    kern = np.ones(9) / 9.0
    for s in range(20):
        g = _rng(1000 + s).standard_normal(n + 8)
        smooth = np.convolve(g, kern, mode="valid")
        assert not S.ncp_is_white(smooth)          # low-pass: power piles up at low frequency
        assert not S.ncp_is_white(g.cumsum()[:n])  # random walk
    # averaged over many white rows the distance shrinks like 1/sqrt(rows)
    d1 = S.ncp_distance(_rng(5).standard_normal((1, n)))
    d64 = S.ncp_distance(_rng(5).standard_normal((64, n)))
    assert d64 < 0.4 * d1


def _problem(seed=1, eta=0.03):
    g = synth.fanflat2d(16, 24, 24, 64.0, 96.0)
    x = synth.ellipse_phantom(16, seed=seed)
    b, e = synth.add_noise(P.forward(g, x).reshape(-1), eta, seed + 50)
    return g, x.reshape(-1), b


@pytest.mark.parametrize("method", ["ab", "ba"])
@pytest.mark.parametrize("every", [1, 3])
def test_ncp_stop_returns_the_last_checked_iterate_before_the_distance_grows(method, every):
    g, x, b = _problem()
    A, B = P.operators(g)
    K = 30
    full = S.hybrid_gmres(method, A, B, b, K, rule="none", keep_iterates=tuple(range(1, K + 1)))
    checks = [k for k in range(1, K + 1) if k % every == 0 or k == K]
    dist = {k: S.ncp_distance((b - A(full["iterates"][k])).reshape(-1, g.n_det_u))
            for k in checks}
    stop = next((checks[i - 1] for i in range(1, len(checks))
                 if dist[checks[i]] > dist[checks[i - 1]]), None)
    assert stop is not None and stop < K, "the test problem must stop early"
    res = S.hybrid_gmres(method, A, B, b, K, rule="none", stop_rule="ncp", ncp_row=g.n_det_u,
                         stop_every=every)
    assert res["status"] == "stopped" and res["k"] == stop
    np.testing.assert_allclose(res["x"], full["iterates"][stop], rtol=1e-10, atol=1e-12)
    assert len(res["lambdas"]) == stop and len(res["resid"]) == stop
    got = dict(res["ncp"])
    for k, d in got.items():
        np.testing.assert_allclose(d, dist[k], rtol=1e-9)
