"""FP64 oracle of the learned lambda rule's network (not in the paper).

TEST INFRASTRUCTURE ONLY.  A 3-layer perceptron, 80 (padded) inputs -> 64 -> 64 -> 1 with GELU
(tanh form) after the two hidden layers, trained by mean-squared error and Adam.  The inputs are
first standardised, x' = (x - mu) * isd, with mu and isd fixed before training (zero
gradient).  The GPU
training kernels are checked against forward(), backward() and adam_step() here on the same
BF16-rounded weights and inputs.

Features of one projected problem (step k of a solve of K steps), H_k = U diag(s) V^T,
c = beta U^T e1 (k+1 entries, the last one the component outside range(H_k)), 80 entries:
  [0]        k / K
  [1..32]    log10(s_i / s_1) for the 32 largest s_i (padded with -16)
  [33..64]   |c_i| / beta for the same i (padded with 0); singular vectors have no fixed sign
  [65]       |c_{k+1}| / beta
  [66]       log10(s_1)
  [67]       log10(beta)
  [68..79]   0
Target (label): log10(lambda* / s_1), lambda* the lambda that minimises the reconstruction
error ||x_k(lambda) - x_true|| of hybrid AB-GMRES, searched like GCV (256 log-spaced points on
[1e-8 s_1, s_1], the best refined by 40 golden-section steps in log lambda).  With
x_k(lambda) = Z_k y_k(lambda), Z = B W (u0 = 0), the error is y^T G y - 2 g^T y + ||x_true||^2,
G = Z_k^T Z_k and g = Z_k^T x_true.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID = 80, 64
GELU_C = math.sqrt(2.0 / math.pi)


def features(k: int, K: int, s: np.ndarray, c: np.ndarray, beta: float) -> np.ndarray:
    """s: the k singular values of H_k in decreasing order; c: beta U^T e1 (k+1 entries)."""
    f = np.zeros(N_IN)
    f[0] = k / K
    s1 = float(s[0])
    m = min(32, k)
    with np.errstate(divide="ignore"):
        f[1:33] = -16.0
        f[1:1 + m] = np.maximum(np.log10(np.maximum(s[:m], 0.0) / s1), -16.0)
    f[33:33 + m] = np.abs(c[:m]) / beta
    f[65] = abs(c[k]) / beta
    f[66] = math.log10(s1)
    f[67] = math.log10(beta)
    return f


def tikhonov_error(lam: float, s, c, Vt, G, g) -> float:
    """y^T G y - 2 g^T y for the Tikhonov solution y = V diag(s / (s^2 + lam^2)) c[:k]."""
    k = len(s)
    y = Vt.T @ (s * c[:k] / (s * s + lam * lam))
    return float(y @ G @ y - 2.0 * g @ y)


def optimal_lambda(Hk: np.ndarray, beta: float, G: np.ndarray, g: np.ndarray) -> float:
    """The label's lambda*: grid of 256 log-spaced values on [1e-8 s_1, s_1], the first
    minimum refined by 40 golden-section steps in log lambda (kept only if not worse)."""
    U, s, Vt = np.linalg.svd(Hk, full_matrices=True)
    c = beta * U[0, :]
    s1 = float(s[0])
    grid = s1 * np.power(10.0, np.linspace(-8.0, 0.0, 256))
    E = np.array([tikhonov_error(l, s, c, Vt, G, g) for l in grid])
    i = int(np.argmin(E))
    a = math.log(grid[max(i - 1, 0)])
    b = math.log(grid[min(i + 1, 255)])
    invphi = (math.sqrt(5.0) - 1.0) / 2.0
    for _ in range(40):
        x1 = b - invphi * (b - a)
        x2 = a + invphi * (b - a)
        if tikhonov_error(math.exp(x1), s, c, Vt, G, g) <= tikhonov_error(math.exp(x2), s, c, Vt, G, g):
            b = x2
        else:
            a = x1
    lam = math.exp(0.5 * (a + b))
    if tikhonov_error(lam, s, c, Vt, G, g) > E[i]:
        lam = float(grid[i])
    return lam


def label(Hk: np.ndarray, beta: float, G: np.ndarray, g: np.ndarray) -> float:
    s1 = float(np.linalg.svd(Hk, compute_uv=False)[0])
    return math.log10(optimal_lambda(Hk, beta, G, g) / s1)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    u = GELU_C * (z + 0.044715 * z ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3 * 0.044715 * z * z)


def init_params(seed: int = 0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return {
        "W1": rng.standard_normal((N_HID, N_IN)) * math.sqrt(2.0 / N_IN),
        "b1": np.zeros(N_HID),
        "W2": rng.standard_normal((N_HID, N_HID)) * math.sqrt(2.0 / N_HID),
        "b2": np.zeros(N_HID),
        "w3": rng.standard_normal(N_HID) * math.sqrt(1.0 / N_HID),
        "b3": np.zeros(1),
        "mu": np.zeros(N_IN),
        "isd": np.ones(N_IN),
    }


def forward(p, X):
    """X: (B, 80).  Returns prediction (B,) and the cache for backward."""
    X = (X - p["mu"]) * p["isd"]
    z1 = X @ p["W1"].T + p["b1"]
    a1 = gelu(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = gelu(z2)
    out = a2 @ p["w3"] + p["b3"][0]
    return out, (X, z1, a1, z2, a2)


def loss(p, X, y):
    out, _ = forward(p, X)
    return float(np.mean((out - y) ** 2))


def backward(p, X, y):
    """Gradients of the mean-squared error w.r.t. every parameter."""
    out, (X, z1, a1, z2, a2) = forward(p, X)
    B = X.shape[0]
    d_out = 2.0 * (out - y) / B
    g = {"w3": a2.T @ d_out, "b3": np.array([d_out.sum()])}
    d_a2 = np.outer(d_out, p["w3"])
    d_z2 = d_a2 * gelu_grad(z2)
    g["W2"] = d_z2.T @ a1
    g["b2"] = d_z2.sum(0)
    d_a1 = d_z2 @ p["W2"]
    d_z1 = d_a1 * gelu_grad(z1)
    g["W1"] = d_z1.T @ X
    g["b1"] = d_z1.sum(0)
    g["mu"] = np.zeros_like(p["mu"])       # the standardisation is not trained
    g["isd"] = np.zeros_like(p["isd"])
    return g


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba), bias-corrected, in place; t counts from 1."""
    for key in p:
        m[key] = b1 * m[key] + (1 - b1) * g[key]
        v[key] = b2 * v[key] + (1 - b2) * g[key] ** 2
        mh = m[key] / (1 - b1 ** t)
        vh = v[key] / (1 - b2 ** t)
        p[key] = p[key] - lr * mh / (np.sqrt(vh) + eps)
    return p


def bf16_round(a):
    """Round an FP64 array to the nearest BF16 value (round to nearest even)."""
    x = np.asarray(a, dtype=np.float32)
    bits = x.view(np.uint32).astype(np.uint64)
    rounding = ((bits >> 16) & 1) + 0x7FFF
    out = ((bits + rounding) >> 16) << 16
    return out.astype(np.uint32).view(np.float32).astype(np.float64)
