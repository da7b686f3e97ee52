"""Pins of the FP64 oracle solver (Algorithms 1/2, Eq. (hybrid_proj), GCV, DP).

The oracle is tied to: the Arnoldi relation and orthonormality (Eq. (Hessenberg)); the
identity between the projected residual and the true residual (Sec. 2.1); the matched-case
equivalences with LSQR and LSMR written from the Golub-Kahan process (Sec. 3, 'Relation to
existing methods'); brute-force minimisation over an explicit Krylov basis; the
full-dimension closed forms (Sec. 3, 'Optimality conditions', read with lambda^2); a dense
evaluation of the GCV definition (Sec. 3.1) and of the Tikhonov least-squares problem.
"""
import math

import numpy as np
import pytest

import synth
from oracle import proj as P
from oracle import solver as S


def _problem(kind="parallel", N=16, views=20, seed=0, eta=0.01):
    if kind == "parallel":
        g = synth.parallel2d(N, views)
    else:
        g = synth.fanflat2d(N, views, int(1.5 * N), 4.0 * N, 6.0 * N)
    x = synth.ellipse_phantom(N, seed=seed)
    bt = P.forward(g, x).reshape(-1)
    b, e = synth.add_noise(bt, eta, seed + 100)
    return g, x.reshape(-1), b, e


@pytest.mark.parametrize("method", ["ab", "ba"])
def test_arnoldi_relation_and_orthogonality(method):
    g, x, b, e = _problem("fan", N=16, views=24)
    A, B = P.operators(g)
    res = S.hybrid_gmres(method, A, B, b, 15, rule="gcv")
    W, H, k = res["W"], res["H"], res["k"]
    M = (lambda w: A(B(w))) if method == "ab" else (lambda w: B(A(w)))
    MW = np.stack([M(W[i]) for i in range(k)], axis=1)
    rel = np.linalg.norm(MW - W[: k + 1].T @ H) / np.linalg.norm(MW)
    assert rel <= 1e-10
    assert np.abs(W[: k + 1] @ W[: k + 1].T - np.eye(k + 1)).max() <= 1e-10


@pytest.mark.parametrize("method", ["ab", "ba"])
@pytest.mark.parametrize("rule", ["gcv", "fixed", "none"])
def test_projected_residual_is_true_residual(method, rule):
    """AB: ||b - A x_k|| equals ||H y - beta e1||; BA: ||B(b - A x_k)|| does."""
    g, x, b, e = _problem("parallel", N=16, views=20)
    A, B = P.operators(g)
    res = S.hybrid_gmres(method, A, B, b, 12, rule=rule, lam_fixed=0.3, true_residual=True)
    np.testing.assert_allclose(res["resid"], res["true_resid"], rtol=1e-9)


def _krylov_basis(M, r0, k):
    K = [r0]
    for _ in range(k - 1):
        K.append(M(K[-1]))
    Q, _ = np.linalg.qr(np.stack(K, axis=1))
    return Q


@pytest.mark.parametrize("method", ["ab", "ba"])
def test_hybrid_iterate_matches_bruteforce_krylov_minimiser(method):
    """Hybrid AB: u_k = argmin_{u in K_k(AB, b)} ||ABu - b||^2 + lam^2 ||u||^2, x_k = B u_k;
    hybrid BA: x_k = argmin_{x in K_k(BA, Bb)} ||BAx - Bb||^2 + lam^2 ||x||^2."""
    g, x, b, e = _problem("fan", N=12, views=16)
    A, B = P.operators(g)
    k, lam = 5, 0.7
    res = S.hybrid_gmres(method, A, B, b, k, rule="fixed", lam_fixed=lam)
    if method == "ab":
        M, rhs = (lambda w: A(B(w))), b
    else:
        M, rhs = (lambda w: B(A(w))), B(b)
    Q = _krylov_basis(M, rhs, k)
    MQ = np.stack([M(Q[:, i]) for i in range(k)], axis=1)
    stacked = np.vstack([MQ, lam * np.eye(k)])
    yb = np.linalg.lstsq(stacked, np.concatenate([rhs, np.zeros(k)]), rcond=None)[0]
    xb = B(Q @ yb) if method == "ab" else Q @ yb
    np.testing.assert_allclose(res["x"], xb, rtol=1e-7, atol=1e-9 * np.abs(xb).max())


def test_matched_ab_is_lsqr_and_ba_is_lsmr():
    """B = A^T: AB-GMRES iterates equal LSQR's, BA-GMRES iterates equal LSMR's (lambda = 0);
    hybrid BA-GMRES equals hybrid LSMR at fixed lambda; hybrid AB-GMRES does not equal hybrid
    LSQR."""
    g, x, b, e = _problem("parallel", N=12, views=16)
    A, At = P.operators(g, matched=True)
    for k in (3, 8, 12):
        ab = S.hybrid_gmres("ab", A, At, b, k, rule="none")["x"]
        ba = S.hybrid_gmres("ba", A, At, b, k, rule="none")["x"]
        lq = S.lsqr_iterate(A, At, b, k)
        lm = S.lsmr_iterate(A, At, b, k)
        assert np.linalg.norm(ab - lq) <= 1e-8 * np.linalg.norm(lq)
        assert np.linalg.norm(ba - lm) <= 1e-8 * np.linalg.norm(lm)
    lam, k = 2.0, 8
    hba = S.hybrid_gmres("ba", A, At, b, k, rule="fixed", lam_fixed=lam)["x"]
    assert np.linalg.norm(hba - S.lsmr_iterate(A, At, b, k, lam)) <= 1e-8 * np.linalg.norm(hba)
    hab = S.hybrid_gmres("ab", A, At, b, k, rule="fixed", lam_fixed=lam)["x"]
    hlq = S.lsqr_iterate(A, At, b, k, lam)
    assert np.linalg.norm(hab - hlq) > 1e-3 * np.linalg.norm(hlq)


def test_full_dimension_limits():
    """BA at k = n gives ((BA)^T BA + lam^2 I)^{-1} (BA)^T B b; AB at k = m gives
    B ((AB)^T AB + lam^2 I)^{-1} (AB)^T b (generic dense operators, no breakdown)."""
    rng = np.random.Generator(np.random.PCG64(3))
    lam = 0.4
    m, n = 14, 9                                   # m >= n for BA
    A = rng.standard_normal((m, n))
    B = A.T + 0.3 * rng.standard_normal((n, m))
    b = rng.standard_normal(m)
    res = S.hybrid_gmres("ba", lambda v: A @ v, lambda v: B @ v, b, n, rule="fixed",
                         lam_fixed=lam)
    BA = B @ A
    xf = np.linalg.solve(BA.T @ BA + lam ** 2 * np.eye(n), BA.T @ (B @ b))
    np.testing.assert_allclose(res["x"], xf, rtol=1e-9, atol=1e-11)
    m, n = 8, 13                                   # n >= m for AB
    A = rng.standard_normal((m, n))
    B = A.T + 0.3 * rng.standard_normal((n, m))
    b = rng.standard_normal(m)
    res = S.hybrid_gmres("ab", lambda v: A @ v, lambda v: B @ v, b, m, rule="fixed",
                         lam_fixed=lam)
    AB = A @ B
    xf = B @ np.linalg.solve(AB.T @ AB + lam ** 2 * np.eye(m), AB.T @ b)
    np.testing.assert_allclose(res["x"], xf, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("k", [1, 4, 17, 30])
def test_tikhonov_and_gcv_against_dense_definitions(k):
    rng = np.random.Generator(np.random.PCG64(k))
    H = np.triu(rng.standard_normal((k + 1, k)), -1) * np.logspace(0, -5, k)[None, :]
    beta = 2.5
    s, c, Vt = S.projected_svd(H, beta)
    e1 = np.zeros(k + 1)
    e1[0] = beta
    for lam in (1e-6, 1e-3, 0.05, 0.8, 3.0):
        y = S.tikhonov_y(lam, s, c, Vt)
        yd = np.linalg.lstsq(np.vstack([H, lam * np.eye(k)]),
                             np.concatenate([e1, np.zeros(k)]), rcond=None)[0]
        np.testing.assert_allclose(y, yd, rtol=1e-8, atol=1e-10 * np.abs(yd).max())
        num = np.linalg.norm(H @ yd - e1) ** 2
        Hl = np.linalg.solve(H.T @ H + lam ** 2 * np.eye(k), H.T)
        tr = np.trace(np.eye(k + 1) - H @ Hl)
        np.testing.assert_allclose(S.gcv_value(lam, s, c), num / tr ** 2, rtol=1e-8)
        np.testing.assert_allclose(S.residual_sq(lam, s, c), num, rtol=1e-8)


@pytest.mark.parametrize("k", [3, 12, 40])
def test_gcv_minimiser_is_global_minimum_on_dense_grid(k):
    rng = np.random.Generator(np.random.PCG64(100 + k))
    H = np.triu(rng.standard_normal((k + 1, k)), -1) * np.logspace(0, -4, k)[None, :]
    s, c, Vt = S.projected_svd(H, 1.0)
    lam = S.gcv_lambda(s, c)
    assert s[0] * 1e-8 * (1 - 1e-12) <= lam <= s[0] * (1 + 1e-12)
    dense = s[0] * np.logspace(-8, 0, 20001)
    gmin = min(S.gcv_value(l, s, c) for l in dense)
    assert S.gcv_value(lam, s, c) <= gmin * (1 + 1e-7)


@pytest.mark.parametrize("k", [5, 25])
def test_dp_lambda_hits_target(k):
    rng = np.random.Generator(np.random.PCG64(200 + k))
    H = np.triu(rng.standard_normal((k + 1, k)), -1) * np.logspace(0, -4, k)[None, :]
    beta = 3.0
    s, c, Vt = S.projected_svd(H, beta)
    lo = math.sqrt(S.residual_sq(s[0] * 1e-8, s, c))
    hi = math.sqrt(S.residual_sq(s[0], s, c))
    target = 0.5 * (lo + hi)
    lam = S.dp_lambda(s, c, target)
    y = S.tikhonov_y(lam, s, c, Vt)
    e1 = np.zeros(k + 1)
    e1[0] = beta
    np.testing.assert_allclose(np.linalg.norm(H @ y - e1), target, rtol=1e-10)


def test_lambda_zero_svd_path_equals_givens_path():
    rng = np.random.Generator(np.random.PCG64(9))
    for k in (1, 5, 20):
        H = np.triu(rng.standard_normal((k + 1, k)), -1)
        s, c, Vt = S.projected_svd(H, 1.7)
        y_svd = S.tikhonov_y(0.0, s, c, Vt)
        y_giv, res = S.givens_gmres_y(H, 1.7)
        e1 = np.zeros(k + 1)
        e1[0] = 1.7
        y_ls = np.linalg.lstsq(H, e1, rcond=None)[0]
        np.testing.assert_allclose(y_svd, y_ls, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(y_giv, y_ls, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(res, np.linalg.norm(H @ y_ls - e1), rtol=1e-9, atol=1e-14)


def test_zero_rhs_breaks_down_at_start():
    g, x, b, e = _problem("parallel", N=8, views=6)
    A, B = P.operators(g)
    res = S.hybrid_gmres("ab", A, B, np.zeros_like(b), 5)
    assert res["status"] == "breakdown" and res["k"] == 0
    assert np.all(res["x"] == 0)


def test_hybrid_stabilises_semi_convergence():
    """Sec. 4: plain AB-GMRES semi-converges, the hybrid (GCV) variant keeps the error low."""
    g, x, b, e = _problem("parallel", N=32, views=30, eta=0.05)
    A, B = P.operators(g)
    ks = (5, 10, 20, 40)
    plain = S.hybrid_gmres("ab", A, B, b, 40, rule="none", keep_iterates=ks)
    hyb = S.hybrid_gmres("ab", A, B, b, 40, rule="gcv", keep_iterates=ks)
    e_plain = [S.rre(plain["iterates"][k], x) for k in ks]
    e_hyb = [S.rre(hyb["iterates"][k], x) for k in ks]
    assert e_plain[-1] > min(e_plain) * 1.05          # semi-convergence
    assert e_hyb[-1] < e_plain[-1]


@pytest.mark.parametrize("k", [4, 17])
def test_lcurve_curvature_matches_finite_differences(k):
    """The closed-form curvature against central differences of the parametric curve
    (log ||H y - beta e1||, log ||y||) in t = ln lambda, with y from the stacked least-squares
    problem (no SVD); curvature does not depend on the parametrisation."""
    rng = np.random.Generator(np.random.PCG64(300 + k))
    H = np.triu(rng.standard_normal((k + 1, k)), -1) * np.logspace(0, -4, k)[None, :]
    beta = 1.3
    s, c, Vt = S.projected_svd(H, beta)
    e1 = np.zeros(k + 1)
    e1[0] = beta

    def point(t):
        lam = math.exp(t)
        y = np.linalg.lstsq(np.vstack([H, lam * np.eye(k)]), np.concatenate([e1, np.zeros(k)]),
                            rcond=None)[0]
        return math.log(np.linalg.norm(H @ y - e1)), math.log(np.linalg.norm(y))

    for lam in s[0] * np.array([1e-4, 1e-3, 1e-2, 0.1, 0.5]):
        t, h = math.log(lam), 1e-3
        (xm2, ym2), (xm, ym), (x0, y0), (xp, yp), (xp2, yp2) = [point(t + j * h) for j in (-2, -1, 0, 1, 2)]
        x1 = (-xp2 + 8 * xp - 8 * xm + xm2) / (12 * h)
        y1 = (-yp2 + 8 * yp - 8 * ym + ym2) / (12 * h)
        x2 = (-xp2 + 16 * xp - 30 * x0 + 16 * xm - xm2) / (12 * h * h)
        y2 = (-yp2 + 16 * yp - 30 * y0 + 16 * ym - ym2) / (12 * h * h)
        kfd = (x1 * y2 - x2 * y1) / (x1 * x1 + y1 * y1) ** 1.5
        kcf = S.lcurve_curvature(lam, s, c)
        assert abs(kcf - kfd) <= 1e-4 * max(1.0, abs(kfd)), (lam, kcf, kfd)


@pytest.mark.parametrize("k", [6, 20])
def test_lcurve_corner_is_the_curvature_maximum(k):
    rng = np.random.Generator(np.random.PCG64(400 + k))
    H = np.triu(rng.standard_normal((k + 1, k)), -1) * np.logspace(0, -4, k)[None, :]
    s, c, Vt = S.projected_svd(H, 2.0)
    lam = S.lcurve_lambda(s, c)
    assert s[0] * 1e-8 * (1 - 1e-12) <= lam <= s[0] * (1 + 1e-12)
    dense = s[0] * np.logspace(-8, 0, 20001)
    kmax = max(S.lcurve_curvature(l, s, c) for l in dense)
    assert S.lcurve_curvature(lam, s, c) >= kmax * (1 - 1e-6)


@pytest.mark.parametrize("method", ["ab", "ba"])
def test_dp_stopping_rule_stops_at_first_consistent_residual(method):
    """Sec. 3.2: the DP stop returns the first iterate whose residual, computed from the
    iterate with the operators (not from the projected problem), is within tau ||e||."""
    g, x_true, b, e = _problem("fan", N=16, views=24, seed=3, eta=0.02)
    A, B = P.operators(g)
    noise = np.linalg.norm(e) if method == "ab" else np.linalg.norm(B(e))
    # lambda = 0: the residual falls through the noise level within the 25 steps
    full = S.hybrid_gmres(method, A, B, b, 25, rule="none", keep_iterates=tuple(range(1, 26)))
    res = S.hybrid_gmres(method, A, B, b, 25, rule="none", stop_rule="dp", stop_target=1.01 * noise)
    k = res["k"]
    assert res["status"] == "stopped" and 1 <= k < 25

    def true_res(x):
        r = b - A(x)
        return np.linalg.norm(r if method == "ab" else B(r))
    assert true_res(res["x"]) <= 1.01 * noise * (1 + 1e-9)
    if k > 1:
        assert true_res(full["iterates"][k - 1]) > 1.01 * noise
    np.testing.assert_allclose(res["x"], full["iterates"][k], rtol=1e-10, atol=1e-12)


def test_rns_stopping_rule():
    g, x_true, b, e = _problem("parallel", N=16, views=20, seed=4, eta=0.01)
    A, B = P.operators(g)
    full = S.hybrid_gmres("ab", A, B, b, 30, rule="gcv", true_residual=True)
    res = S.hybrid_gmres("ab", A, B, b, 30, rule="gcv", stop_rule="rns", stop_tol=1e-3)
    k = res["k"]
    tr = full["true_resid"]            # ||b - A x_k|| from the iterates themselves
    rel_change = [abs(tr[j - 1] - tr[j]) / tr[j - 1] for j in range(1, len(tr))]
    first = next(j + 2 for j, v in enumerate(rel_change) if v < 1e-3 * (1 + 1e-6))
    assert k == first


# ----------------------------------------------------------------------------- initial guess
def _shifted_krylov_minimiser(method, A, B, b, x0, k, lam):
    """x0 + (B) Q z with Q an orthonormal basis of the Krylov space of Sec. 2.1 started at the
    shifted residual (AB: K_k(AB, b - A x0); BA: K_k(BA, B(b - A x0))) and z the minimiser of
    ||M Q z - r0||^2 + lam^2 ||z||^2 by dense least squares."""
    if method == "ab":
        M, r0 = (lambda w: A(B(w))), b - A(x0)
    else:
        M, r0 = (lambda w: B(A(w))), B(b - A(x0))
    Q = _krylov_basis(M, r0, k)
    MQ = np.stack([M(Q[:, i]) for i in range(k)], axis=1)
    z = np.linalg.lstsq(np.vstack([MQ, lam * np.eye(k)]), np.concatenate([r0, np.zeros(k)]),
                        rcond=None)[0]
    return x0 + (B(Q @ z) if method == "ab" else Q @ z), float(np.linalg.norm(MQ @ z - r0))


@pytest.mark.parametrize("method", ["ab", "ba"])
def test_initial_guess_iterate_matches_shifted_krylov_minimiser(method):
    """Algorithms 1/2 from x0 != 0 (AB: x0 = B u0): the iterate is x0 plus the hybrid
    minimiser over the Krylov space of the initial residual, and the projected residual is
    that minimiser's residual."""
    g, x, b, e = _problem("fan", N=12, views=16, seed=2)
    A, B = P.operators(g)
    rng = np.random.Generator(np.random.PCG64(17))
    x0 = B(rng.standard_normal(g.m)) if method == "ab" else 0.5 * x + rng.random(g.n)
    k, lam = 5, 0.7
    res = S.hybrid_gmres(method, A, B, b, k, rule="fixed", lam_fixed=lam, x0=x0)
    xb, rb = _shifted_krylov_minimiser(method, A, B, b, x0, k, lam)
    np.testing.assert_allclose(res["x"], xb, rtol=1e-7, atol=1e-9 * np.abs(xb).max())
    np.testing.assert_allclose(res["resid"][-1], rb, rtol=1e-8)
    # the initial guess really moved the answer (the pin is not the x0 = 0 case again)
    x_zero = S.hybrid_gmres(method, A, B, b, k, rule="fixed", lam_fixed=lam)["x"]
    assert np.linalg.norm(res["x"] - x_zero) > 1e-3 * np.linalg.norm(x_zero)


def test_matched_ab_from_initial_guess_is_lsqr_of_shifted_data():
    """B = A^T, lambda = 0: AB-GMRES from x0 = A^T u0 equals x0 + LSQR(b - A x0) (Sec. 3,
    relation to existing methods, applied to the shifted system A d = b - A x0)."""
    g, x, b, e = _problem("parallel", N=12, views=16, seed=5)
    A, At = P.operators(g, matched=True)
    rng = np.random.Generator(np.random.PCG64(23))
    x0 = At(rng.standard_normal(g.m))
    for k in (3, 7):
        ab = S.hybrid_gmres("ab", A, At, b, k, rule="none", x0=x0)["x"]
        lq = x0 + S.lsqr_iterate(A, At, b - A(x0), k)
        assert np.linalg.norm(ab - lq) <= 1e-8 * np.linalg.norm(lq)


# ----------------------------------------------------------------------------- restarting
def _dense_pair(m, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.standard_normal((m, n))
    B = A.T + 0.3 * rng.standard_normal((n, m))
    return A, B, rng.standard_normal(m), rng.standard_normal(n)


def test_restart_at_full_dimension_follows_the_closed_form():
    """Sec. 3.3 with p = n (BA) or p = m (AB): each cycle from x_{c-1} lands on the closed form
    of Sec. 3 (optimality conditions, lambda^2 reading) for the shifted system, so
    x_c = x_{c-1} + (M^T M + lam^2 I)^{-1} M^T r(x_{c-1}) (BA: M = BA, r = B(b - A x);
    AB: x_c = x_{c-1} + B (N^T N + lam^2 I)^{-1} N^T (b - A x_{c-1}), N = AB).
    The regularisation acts on the update, not on the iterate, so the cycles keep moving."""
    lam = 0.4
    A, B, b, x0 = _dense_pair(14, 9, 3)
    Af, Bf = (lambda v: A @ v), (lambda v: B @ v)
    M = B @ A
    x, hist = S.restarted_hybrid_gmres("ba", Af, Bf, b, 9, 3, x0=x0, rule="fixed", lam_fixed=lam)
    xc = x0.copy()
    for c in range(3):
        xc = xc + np.linalg.solve(M.T @ M + lam ** 2 * np.eye(9), M.T @ (B @ (b - A @ xc)))
        np.testing.assert_allclose(hist[c]["x"], xc, rtol=1e-9, atol=1e-11)
    A, B, b, _ = _dense_pair(8, 13, 4)
    Af, Bf = (lambda v: A @ v), (lambda v: B @ v)
    N = A @ B
    x, hist = S.restarted_hybrid_gmres("ab", Af, Bf, b, 8, 2, rule="fixed", lam_fixed=lam)
    xc = np.zeros(13)
    for c in range(2):
        xc = xc + B @ np.linalg.solve(N.T @ N + lam ** 2 * np.eye(8), N.T @ (b - A @ xc))
        np.testing.assert_allclose(hist[c]["x"], xc, rtol=1e-9, atol=1e-11)
    assert np.linalg.norm(hist[1]["x"] - hist[0]["x"]) > 1e-3 * np.linalg.norm(hist[0]["x"])


@pytest.mark.parametrize("method", ["ab", "ba"])
def test_restarted_cycles_are_shifted_krylov_minimisers(method):
    """Sec. 3.3 on a CT problem: cycle 1 is the minimiser over K_p from x = 0, cycle 2 the
    minimiser over K_p of the residual of cycle 1's iterate, added to it; one cycle of the
    restarted solve is the plain solve."""
    g, x, b, e = _problem("fan", N=12, views=16, seed=6)
    A, B = P.operators(g)
    p, lam = 4, 0.5
    xr, hist = S.restarted_hybrid_gmres(method, A, B, b, p, 2, rule="fixed", lam_fixed=lam)
    x1, _ = _shifted_krylov_minimiser(method, A, B, b, np.zeros(g.n), p, lam)
    x2, _ = _shifted_krylov_minimiser(method, A, B, b, x1, p, lam)
    np.testing.assert_allclose(hist[0]["x"], x1, rtol=1e-7, atol=1e-9 * np.abs(x1).max())
    np.testing.assert_allclose(xr, x2, rtol=1e-7, atol=1e-9 * np.abs(x2).max())
    plain = S.hybrid_gmres(method, A, B, b, p, rule="fixed", lam_fixed=lam)["x"]
    np.testing.assert_allclose(hist[0]["x"], plain, rtol=1e-12, atol=1e-14)
