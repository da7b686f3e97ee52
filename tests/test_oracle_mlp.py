"""Pins of the learned-lambda network oracle: analytic gradients against central
differences, the GELU derivative against its finite difference, a closed-form single-step
Adam update, and BF16 rounding against the format's definition."""
import math

import numpy as np

from oracle import mlp as M


def test_gelu_derivative_matches_finite_difference():
    z = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)
    # special values: GELU(0) = 0, GELU'(0) = 1/2, GELU(z) -> z for large z
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert abs(M.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    assert abs(M.gelu(np.array([8.0]))[0] - 8.0) < 1e-12


def test_backward_matches_central_differences():
    rng = np.random.Generator(np.random.PCG64(4))
    p = M.init_params(1)
    X = rng.standard_normal((7, M.N_IN))
    y = rng.standard_normal(7)
    p["mu"] = rng.standard_normal(M.N_IN) * 0.3          # a non-trivial standardisation
    p["isd"] = 0.5 + rng.random(M.N_IN)
    g = M.backward(p, X, y)
    assert not g["mu"].any() and not g["isd"].any()      # fixed, not trained
    h = 1e-6
    for key in ("W1", "b1", "W2", "b2", "w3", "b3"):
        flat = p[key].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss(p, X, y)
            flat[idx] = old - h
            lm = M.loss(p, X, y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[key].reshape(-1)[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (key, idx)


def test_first_adam_step_is_signed_learning_rate():
    """With m0 = v0 = 0 the bias-corrected first step is -lr * g / (|g| + eps)."""
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 0.0])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    M.adam_step(p, g, m, v, 1, lr=0.01)
    np.testing.assert_allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01, 3.0], rtol=0, atol=1e-9)


def test_bf16_rounding_definition():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.1415926, 1e-3])
    r = M.bf16_round(vals)
    assert r[0] == 1.0 and r[1] == 1.0          # 1 + 2^-8 is a tie: rounds to the even 1.0
    assert r[2] == 1.0 + 2 ** -7
    for v, rv in zip(vals, r):
        assert abs(rv - v) <= 2 ** -8 * abs(v)


def test_features_layout():
    s = np.array([4.0, 2.0, 1.0])
    c = np.array([1.0, -0.5, 0.25, -0.125])
    f = M.features(3, 30, s, c, 2.0)
    assert f.shape == (80,) and f[0] == 0.1
    np.testing.assert_allclose(f[1:4], [0.0, math.log10(0.5), math.log10(0.25)])
    assert np.all(f[4:33] == -16.0)
    np.testing.assert_allclose(f[33:36], [0.5, 0.25, 0.125])
    assert np.all(f[36:65] == 0.0)
    assert f[65] == 0.0625
    assert abs(f[66] - math.log10(4.0)) < 1e-15 and abs(f[67] - math.log10(2.0)) < 1e-15
    assert np.all(f[68:] == 0.0)


def test_features_of_a_known_svd():
    """H = [diag(d); 0] rotated on the left by an orthogonal Q: singular values d, and
    c = beta Q^T e1 up to the signs of the singular vectors."""
    rng = np.random.Generator(np.random.PCG64(9))
    d = np.array([3.0, 1.5, 0.2, 1e-20])
    Q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    H = Q @ np.vstack([np.diag(d), np.zeros((1, 4))])
    U, s, Vt = np.linalg.svd(H, full_matrices=True)
    f = M.features(4, 8, s, 2.0 * U[0, :], 2.0)
    np.testing.assert_allclose(f[1:4], np.log10(d[:3] / 3.0), rtol=1e-12)
    assert f[4] == -16.0                       # log10(1e-20 / 3) clamps to -16
    np.testing.assert_allclose(f[33:37], np.abs(Q[0, :4]), rtol=1e-10)
    np.testing.assert_allclose(f[65], abs(Q[0, 4]), rtol=1e-10)


def _tiny_label_case(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    k, n = 6, 40
    H = np.triu(rng.standard_normal((k + 1, k)), -1)
    H[np.arange(1, k + 1), np.arange(k)] = np.abs(H[np.arange(1, k + 1), np.arange(k)]) + 0.1
    H = H @ np.diag(np.logspace(0, -4, k))           # graded columns: a wide singular spectrum
    Z = rng.standard_normal((n, k))
    beta = 1.7
    y_true = np.linalg.lstsq(H, beta * np.eye(k + 1)[:, 0], rcond=None)[0]
    x_true = Z @ y_true + 0.05 * rng.standard_normal(n)
    return H, beta, Z, x_true


def test_optimal_lambda_against_brute_force():
    """lambda* against a direct search: y from the regularised normal equations (no SVD),
    the error from the explicit Z, on 4001 log-spaced lambda."""
    for seed in (1, 2, 3):
        H, beta, Z, x_true = _tiny_label_case(seed)
        k = H.shape[1]
        G, g = Z.T @ Z, Z.T @ x_true
        lam = M.optimal_lambda(H, beta, G, g)
        s1 = np.linalg.norm(H, 2)
        rhs = beta * H[0, :]

        def err(l):
            y = np.linalg.solve(H.T @ H + l * l * np.eye(k), rhs)
            return float(np.sum((Z @ y - x_true) ** 2))

        grid = s1 * np.logspace(-8, 0, 4001)
        E = np.array([err(l) for l in grid])
        assert err(lam) <= E.min() * (1 + 1e-6) + 1e-12, seed
        assert 1e-8 * s1 * (1 - 1e-12) <= lam <= s1 * (1 + 1e-12)
        assert abs(math.log10(lam) - math.log10(grid[np.argmin(E)])) < 0.05, seed


def test_label_special_cases():
    """x_true = 0: the error ||Z y||^2 is smallest for the largest lambda on the search range.
    x_true = the unregularised solution's image, exactly: lambda* at the bottom of the range."""
    H, beta, Z, _ = _tiny_label_case(4)
    k = H.shape[1]
    G = Z.T @ Z
    s1 = np.linalg.norm(H, 2)
    assert abs(M.label(H, beta, G, np.zeros(k))) < 1e-9          # lambda* = s_1
    y0 = np.linalg.lstsq(H, beta * np.eye(k + 1)[:, 0], rcond=None)[0]
    lam = M.optimal_lambda(H, beta, G, G @ y0)
    assert lam <= 1e-7 * s1
