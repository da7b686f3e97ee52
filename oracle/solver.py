"""FP64 oracle of hybrid AB-/BA-GMRES (arXiv 2602.17892, Sec. 3, Algorithms 1 and 2).

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously-correct reference the GPU library is
checked against.  It shares no code with the CUDA path.  Operators are plain callables on
flat FP64 vectors, so the same routines run with the C oracle projectors, with explicit
matrices, or with the matched pair B = A^T.

Step by step it follows the paper:

* Sec. 2.1, Eq. (AB_optimality)/(BA_optimality): the Krylov spaces of AB and BA, started from
  r0 = b - A x0 (AB, x0 = B u0) or r0 = B (b - A x0) (BA);
* Eq. (Hessenberg): the Arnoldi relation M W_k = W_{k+1} H_k, built with modified
  Gram-Schmidt and one full second MGS pass whose coefficients are added to H
  (reorthogonalisation);
* Eq. (hybrid_proj): Tikhonov on the projected problem, solved through the SVD of the
  (k+1) x k Hessenberg matrix H_k = U diag(sigma) V^T, c = ||r0|| U^T e1,
  y = sum_i v_i sigma_i c_i / (sigma_i^2 + lambda^2);
* Sec. 3.1: GCV(lambda) = ||H y - beta e1||^2 / trace(I - H H_lambda)^2 with
  H_lambda = (H^T H + lambda^2 I)^{-1} H^T (lambda^2 throughout, as in Eq. (tikhonov));
* Sec. 3.2: the discrepancy principle, used here to pick lambda: ||H y - beta e1|| = tau eta;
  the stopping criteria DP, NCP and RNS;
* Sec. 3 (the hybrid iterate): x_k = x0 + B W_k y_k (AB) or x0 + W_k y_k (BA);
* Sec. 3.3: restarting from the previous cycle's iterate.

Readings where the paper is silent (the GPU library implements the same readings):
* GCV minimiser: 256 log-spaced lambda in [sigma_1 1e-8, sigma_1], first grid minimum, then
  40 golden-section steps in log lambda on the neighbouring bracket (ties to the left); the
  refined value is kept only if it is not worse than the grid point.
* DP as a lambda rule: solve rho(lambda) = tau * noise_norm by 60 bisection steps in log
  lambda over the same range; clamp to the range ends when there is no root.
* x0 = 0 (u0 = 0) unless given; breakdown when h_{k+1,k} <= 1e-14 ||M w_k||.
* NCP (Sec. 3.2, after Hansen's normalized cumulative periodogram): the data-space residual
  b - A x_k, split into detector rows, each row's periodogram without the zero frequency,
  normalised and accumulated; the rows' NCPs are averaged and compared with the white-noise
  line i/q.  The iteration stops at the first checked step whose distance from that line is
  larger than at the previous checked step, and returns the previous checked step's iterate.
"""
from __future__ import annotations

import math

import numpy as np

GCV_GRID = 256
GCV_GOLDEN_STEPS = 40
DP_BISECT_STEPS = 60
LAMBDA_RANGE = 1e-8
BREAKDOWN_TOL = 1e-14


# ----------------------------------------------------------------------------- small problem

def projected_svd(Hk: np.ndarray, beta: float):
    """SVD of the (k+1) x k Hessenberg matrix and c = beta U^T e1 (length k+1)."""
    U, s, Vt = np.linalg.svd(Hk, full_matrices=True)
    c = beta * U[0, :]
    return s, c, Vt


def residual_sq(lam: float, s: np.ndarray, c: np.ndarray) -> float:
    """||H y_lambda - beta e1||^2 = sum_i (lam^2 c_i / (s_i^2 + lam^2))^2 + c_{k+1}^2."""
    k = len(s)
    f = lam * lam / (s * s + lam * lam)
    return float(np.sum((f * c[:k]) ** 2) + np.sum(c[k:] ** 2))


def gcv_value(lam: float, s: np.ndarray, c: np.ndarray) -> float:
    """GCV(lambda); trace(I_{k+1} - H H_lambda) = (k+1) - sum_i s_i^2/(s_i^2+lam^2)."""
    k = len(s)
    tr = (k + 1) - float(np.sum(s * s / (s * s + lam * lam)))
    return residual_sq(lam, s, c) / (tr * tr)


def gcv_lambda(s: np.ndarray, c: np.ndarray) -> float:
    s1 = float(s[0])
    grid = s1 * np.power(10.0, np.linspace(math.log10(LAMBDA_RANGE), 0.0, GCV_GRID))
    G = np.array([gcv_value(l, s, c) for l in grid])
    i = int(np.argmin(G))                     # first minimum: ties go to the smaller lambda
    a = math.log(grid[max(i - 1, 0)])
    b = math.log(grid[min(i + 1, GCV_GRID - 1)])
    invphi = (math.sqrt(5.0) - 1.0) / 2.0
    for _ in range(GCV_GOLDEN_STEPS):
        x1 = b - invphi * (b - a)
        x2 = a + invphi * (b - a)
        if gcv_value(math.exp(x1), s, c) <= gcv_value(math.exp(x2), s, c):
            b = x2
        else:
            a = x1
    lam = math.exp(0.5 * (a + b))
    if gcv_value(lam, s, c) > G[i]:
        lam = float(grid[i])
    return lam


def dp_lambda(s: np.ndarray, c: np.ndarray, target: float) -> float:
    """lambda with rho(lambda) = target; rho is increasing in lambda."""
    s1 = float(s[0])
    lo, hi = math.log(s1 * LAMBDA_RANGE), math.log(s1)
    rho = lambda L: math.sqrt(residual_sq(math.exp(L), s, c))
    if rho(lo) >= target:
        return math.exp(lo)
    if rho(hi) <= target:
        return math.exp(hi)
    for _ in range(DP_BISECT_STEPS):
        mid = 0.5 * (lo + hi)
        if rho(mid) < target:
            lo = mid
        else:
            hi = mid
    return math.exp(0.5 * (lo + hi))


def tikhonov_y(lam: float, s: np.ndarray, c: np.ndarray, Vt: np.ndarray) -> np.ndarray:
    """Solution of Eq. (hybrid_proj) from the SVD; lam = 0 gives the pseudo-inverse (GMRES)."""
    k = len(s)
    with np.errstate(divide="ignore", invalid="ignore"):
        coef = np.where(s > 0, s * c[:k] / (s * s + lam * lam), 0.0)
    return Vt.T @ coef


def lcurve_curvature(lam: float, s: np.ndarray, c: np.ndarray) -> float:
    """Curvature of the projected L-curve (log ||H y_lam - beta e1||, log ||y_lam||) at lam
    (Sec. 3.1, L-curve criterion), in closed form from eta = ||y||^2, rho = ||H y - beta e1||^2
    and eta' = d eta / d lam (filter factors f_i = s_i^2 / (s_i^2 + lam^2)).  With
    X = log sqrt(rho), Y = log sqrt(eta) and rho' = -lam^2 eta', the curvature
    (X' Y'' - X'' Y') / (X'^2 + Y'^2)^(3/2) reduces to
        kappa = 2 eta rho (lam^2 eta' rho + 2 lam eta rho + lam^4 eta eta')
                / (|eta'| (lam^4 eta^2 + rho^2)^(3/2))."""
    k = len(s)
    pos = s > 0
    d = s * s + lam * lam
    f = s * s / d
    g = lam * lam / d                      # 1 - f without cancellation at small lambda
    ci = c[:k]
    eta = float(np.sum((f[pos] * ci[pos] / s[pos]) ** 2))
    rho = float(np.sum((g * ci) ** 2) + np.sum(c[k:] ** 2))
    deta = float(-4.0 / lam * np.sum(g[pos] * f[pos] ** 2 * (ci[pos] / s[pos]) ** 2))
    if eta == 0.0 or rho == 0.0 or deta == 0.0:
        return 0.0
    num = lam * lam * deta * rho + 2.0 * lam * eta * rho + lam ** 4 * eta * deta
    return 2.0 * eta * rho * num / (abs(deta) * (lam ** 4 * eta * eta + rho * rho) ** 1.5)


def lcurve_lambda(s: np.ndarray, c: np.ndarray) -> float:
    """The L-curve corner: the first maximum of the curvature on the 256-point grid of GCV,
    refined by 40 golden-section steps in log lambda on the neighbouring bracket (kept only if
    not worse)."""
    s1 = float(s[0])
    grid = s1 * np.power(10.0, np.linspace(math.log10(LAMBDA_RANGE), 0.0, GCV_GRID))
    K = np.array([lcurve_curvature(l, s, c) for l in grid])
    i = int(np.argmax(K))
    a = math.log(grid[max(i - 1, 0)])
    b = math.log(grid[min(i + 1, GCV_GRID - 1)])
    invphi = (math.sqrt(5.0) - 1.0) / 2.0
    for _ in range(GCV_GOLDEN_STEPS):
        x1 = b - invphi * (b - a)
        x2 = a + invphi * (b - a)
        if lcurve_curvature(math.exp(x1), s, c) >= lcurve_curvature(math.exp(x2), s, c):
            b = x2
        else:
            a = x1
    lam = math.exp(0.5 * (a + b))
    if lcurve_curvature(lam, s, c) < K[i]:
        lam = float(grid[i])
    return lam


def choose_lambda(rule: str, s, c, lam_fixed=None, dp_target=None) -> float:
    if rule == "none":
        return 0.0
    if rule == "fixed":
        return float(lam_fixed)
    if rule == "gcv":
        return gcv_lambda(s, c)
    if rule == "dp":
        return dp_lambda(s, c, dp_target)
    if rule == "lcurve":
        return lcurve_lambda(s, c)
    raise ValueError(rule)


def givens_gmres_y(Hk: np.ndarray, beta: float):
    """lambda = 0 path of Eq. (proj_pbm) by Givens rotations (Sec. 2.1: 'Givens rotations or
    a QR factorisation of H_k').  Returns (y, |residual|)."""
    k1, k = Hk.shape
    R = Hk.astype(np.float64).copy()
    g = np.zeros(k1)
    g[0] = beta
    for j in range(k):
        a, b = R[j, j], R[j + 1, j]
        r = math.hypot(a, b)
        cs, sn = (1.0, 0.0) if r == 0 else (a / r, b / r)
        rows = R[[j, j + 1], j:].copy()
        R[j, j:] = cs * rows[0] + sn * rows[1]
        R[j + 1, j:] = -sn * rows[0] + cs * rows[1]
        gj, gj1 = g[j], g[j + 1]
        g[j], g[j + 1] = cs * gj + sn * gj1, -sn * gj + cs * gj1
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - R[i, i + 1:k] @ y[i + 1:]) / R[i, i]
    return y, abs(g[k])


# ----------------------------------------------------------------------------- stopping rules

NCP_KS_95 = 1.358      # asymptotic Kolmogorov-Smirnov critical value at 5 % significance


def periodogram(rows: np.ndarray) -> np.ndarray:
    """|DFT|^2 of every row of a (R, n) array at the frequencies 1..q, q = floor(n/2) (the
    zero frequency is left out: it carries the row's mean, not its whiteness)."""
    rows = np.asarray(rows, np.float64)
    q = rows.shape[1] // 2
    return np.abs(np.fft.fft(rows, axis=1)[:, 1:q + 1]) ** 2


def ncp(rows: np.ndarray) -> np.ndarray:
    """Normalized cumulative periodogram (Sec. 3.2; Hansen's NCP) of a residual split into
    rows of one detector row each: per row c_i = (p_1 + ... + p_i) / (p_1 + ... + p_q), then the
    mean over the rows whose periodogram is not zero.  For white noise c_i is close to i/q.
    Returns None when no row has any power (an exactly fitted residual)."""
    p = periodogram(rows)
    tot = p.sum(axis=1)
    keep = tot > 0
    if not keep.any():
        return None
    c = np.cumsum(p[keep], axis=1) / tot[keep, None]
    return c.mean(axis=0)


def ncp_distance(rows: np.ndarray) -> float:
    """||c - c_white||_2 with c_white,i = i/q (0 for a residual without power)."""
    c = ncp(rows)
    if c is None:
        return 0.0
    q = c.size
    return float(np.linalg.norm(c - np.arange(1, q + 1) / q))


def ncp_is_white(row: np.ndarray) -> bool:
    """Kolmogorov-Smirnov test of one row's NCP against the white-noise line at 5 %."""
    c = ncp(np.asarray(row, np.float64).reshape(1, -1))
    q = c.size
    return bool(np.max(np.abs(c - np.arange(1, q + 1) / q)) < NCP_KS_95 / math.sqrt(q))


def stop_reached(stop_rule, resid, k: int, stop_target=None, stop_tol=None) -> bool:
    """Norm-based stopping criteria of Sec. 3.2 on the residual norms rho_1..rho_k (resid,
    0-based): 'dp'  stops at the first k with rho_k <= tau ||e|| (stop_target; the paper prints
    the inequality reversed), 'rns' at the first k >= 2 with
    |rho_{k-1} - rho_k| / rho_{k-1} < stop_tol."""
    if stop_rule is None or stop_rule == "none":
        return False
    if stop_rule == "dp":
        return resid[k - 1] <= stop_target
    if stop_rule == "rns":
        return k >= 2 and abs(resid[k - 2] - resid[k - 1]) < stop_tol * resid[k - 2]
    raise ValueError(stop_rule)


# ----------------------------------------------------------------------------- Algorithms 1 / 2

def hybrid_gmres(method: str, A, B, b, iters: int, rule: str = "gcv", lam_fixed=None,
                 dp_target=None, reorth: bool = True, keep_iterates=(), x0=None,
                 true_residual: bool = False, stop_rule=None, stop_tol=None, stop_target=None,
                 ncp_row=None, stop_every: int = 1):
    """Hybrid AB-GMRES (method='ab', Algorithm 1) or hybrid BA-GMRES ('ba', Algorithm 2).

    A, B: callables on flat FP64 vectors.  rule in {'none', 'fixed', 'gcv', 'dp', 'lcurve'};
    dp_target is tau * ||e|| for AB and tau * ||B e|| for BA (the noise in the space where
    Alg. 2 measures its residual).  x0: initial image (AB: x0 = B u0 for some u0).
    stop_rule in {None, 'dp', 'rns', 'ncp'} ends the iteration early (Sec. 3.2; stop_target,
    stop_tol; 'ncp' needs ncp_row, the detector row length that the data residual is split by,
    and is checked at the steps stop_every, 2 stop_every, ... and the last).  Returns a dict
    with the final iterate, the per-iteration lambda and projected residual, H, W, y, the NCP
    distances of the checked steps and the iterates at the steps in keep_iterates.
    """
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    x0v = np.zeros_like(B(b)) if x0 is None else np.asarray(x0, np.float64).reshape(-1)
    # Krylov spaces of Sec. 2.1, shifted by the initial guess: AB-GMRES solves A B u = r0 with
    # r0 = b - A x0 in the data space; BA-GMRES solves B A x = r0 with r0 = B (b - A x0)
    if method == "ab":
        r0 = b - A(x0v)
        M = lambda w: A(B(w))
    elif method == "ba":
        r0 = B(b - A(x0v))
        M = lambda w: B(A(w))
    else:
        raise ValueError(method)

    L = r0.size
    beta = float(np.linalg.norm(r0))
    out = dict(lambdas=[], resid=[], status="ok", iterates={}, beta=beta, true_resid=[],
               ncp=[])
    if beta == 0.0:
        out.update(x=x0v.copy(), H=np.zeros((1, 0)), W=np.zeros((0, L)), y=np.zeros(0), k=0,
                   status="breakdown")
        return out
    W = np.zeros((iters + 1, L))
    H = np.zeros((iters + 1, iters))
    W[0] = r0 / beta
    y = np.zeros(0)
    k_done = 0
    ncp_prev = None                                      # (k, distance, y) of the last check
    for k in range(1, iters + 1):
        # Arnoldi relation M W_k = W_{k+1} H_k (Eq. (Hessenberg)): column k of H from
        # q = M w_k by modified Gram-Schmidt, then one more full pass (reorthogonalisation)
        q = M(W[k - 1])
        qnorm0 = float(np.linalg.norm(q))
        for _pass in range(2 if reorth else 1):
            for i in range(k):
                d = float(q @ W[i])
                H[i, k - 1] += d
                q = q - d * W[i]
        hk = float(np.linalg.norm(q))
        H[k, k - 1] = hk
        broke = hk <= BREAKDOWN_TOL * qnorm0
        if not broke:
            W[k] = q / hk
        # projected Tikhonov problem (Eq. (hybrid_proj)) with lambda_k from the rule
        Hk = H[: k + 1, :k]
        s, c, Vt = projected_svd(Hk, beta)
        lam = choose_lambda(rule, s, c, lam_fixed, dp_target)
        y = tikhonov_y(lam, s, c, Vt)
        out["lambdas"].append(lam)
        out["resid"].append(math.sqrt(residual_sq(lam, s, c)))
        k_done = k
        ncp_check = stop_rule == "ncp" and (k % stop_every == 0 or k == iters)
        if k in keep_iterates or true_residual or ncp_check:
            xk = _form_x(method, B, x0v, W[:k], y)       # the hybrid iterate of Sec. 3
            if k in keep_iterates:
                out["iterates"][k] = xk
            if true_residual or ncp_check:
                r = b - A(xk)
            if true_residual:
                out["true_resid"].append(float(np.linalg.norm(r if method == "ab" else B(r))))
            if ncp_check:
                dist = ncp_distance(r.reshape(-1, ncp_row))
                out["ncp"].append((k, dist))
                if ncp_prev is not None and dist > ncp_prev[1]:
                    k_done, y = ncp_prev[0], ncp_prev[2]
                    out["lambdas"] = out["lambdas"][:k_done]
                    out["resid"] = out["resid"][:k_done]
                    out["status"] = "stopped"
                    break
                ncp_prev = (k, dist, y)
        if broke:
            out["status"] = "breakdown"
            break
        if stop_rule != "ncp" and stop_reached(stop_rule, out["resid"], k, stop_target,
                                               stop_tol):
            out["status"] = "stopped"
            break
    out.update(x=_form_x(method, B, x0v, W[:k_done], y), H=H[: k_done + 1, :k_done],
               W=W[: k_done + 1], y=y, k=k_done)
    return out


def _form_x(method, B, x0v, Wk, y):
    """x_k = x0 + B W_k y (hybrid AB-GMRES) or x0 + W_k y (hybrid BA-GMRES), Sec. 3."""
    z = Wk.T @ y
    return x0v + (B(z) if method == "ab" else z)


def restarted_hybrid_gmres(method, A, B, b, cycle: int, n_cycles: int, x0=None, **kw):
    """Sec. 3.3: after p = cycle iterations the method starts again from the current iterate
    (the first cycle from x0, zero when not given)."""
    x = x0
    hist = []
    for _ in range(n_cycles):
        res = hybrid_gmres(method, A, B, b, cycle, x0=x, **kw)
        x = res["x"]
        hist.append(res)
    return x, hist


# ----------------------------------------------------------------------------- comparators

def golub_kahan(A, At, b, k: int):
    """Golub-Kahan bidiagonalisation with full reorthogonalisation:
    A V_k = U_{k+1} Bk,  A^T U_{k+1} = V_k Bk^T + alpha_{k+1} v_{k+1} e_{k+1}^T."""
    b = np.asarray(b, np.float64).reshape(-1)
    beta1 = np.linalg.norm(b)
    U = [b / beta1]
    v = At(U[0])
    alpha = np.linalg.norm(v)
    V = [v / alpha]
    alphas, betas = [alpha], []
    for j in range(k):
        u = A(V[j]) - alphas[j] * U[j]
        for _ in range(2):
            for ui in U:
                u = u - (u @ ui) * ui
        bet = np.linalg.norm(u)
        U.append(u / bet)
        betas.append(bet)
        v = At(U[j + 1]) - bet * V[j]
        for _ in range(2):
            for vi in V:
                v = v - (v @ vi) * vi
        al = np.linalg.norm(v)
        V.append(v / al)
        alphas.append(al)
    Bk = np.zeros((k + 1, k))
    for j in range(k):
        Bk[j, j] = alphas[j]
        Bk[j + 1, j] = betas[j]
    return beta1, np.array(U), np.array(V), Bk, np.array(alphas), np.array(betas)


def lsqr_iterate(A, At, b, k: int, lam: float = 0.0):
    """(Hybrid) LSQR iterate: x = V_k argmin ||Bk y - beta1 e1||^2 + lam^2 ||y||^2."""
    beta1, U, V, Bk, al, be = golub_kahan(A, At, b, k)
    rhs = np.zeros(k + 1)
    rhs[0] = beta1
    M = np.vstack([Bk, lam * np.eye(k)])
    y = np.linalg.lstsq(M, np.concatenate([rhs, np.zeros(k)]), rcond=None)[0]
    return V[:k].T @ y


def lsmr_iterate(A, At, b, k: int, lam: float = 0.0):
    """(Hybrid) LSMR iterate: x = V_k y minimising ||A^T(b - A V_k y)||^2 + lam^2 ||y||^2.
    With the Golub-Kahan relations ||A^T r||^2 = ||alpha1 beta1 e1 - Bk^T Bk y||^2
    + (alpha_{k+1} beta_{k+1} y_k)^2."""
    beta1, U, V, Bk, al, be = golub_kahan(A, At, b, k)
    T = Bk.T @ Bk
    last = np.zeros((1, k))
    last[0, k - 1] = al[k] * be[k - 1]
    M = np.vstack([T, last, lam * np.eye(k)])
    rhs = np.zeros(2 * k + 1)
    rhs[0] = al[0] * beta1
    y = np.linalg.lstsq(M, rhs, rcond=None)[0]
    return V[:k].T @ y


def rre(x, x_true) -> float:
    """Relative reconstruction error ||x - x_true|| / ||x_true|| (Sec. 4)."""
    x = np.asarray(x, np.float64).reshape(-1)
    x_true = np.asarray(x_true, np.float64).reshape(-1)
    return float(np.linalg.norm(x - x_true) / np.linalg.norm(x_true))
