"""Helpers shared by the GPU parity tests: seeded problems (oracle FP64 data) and thin calls
through the C ABI."""
import numpy as np

import synth
from oracle import proj as OP


def cuda():
    import torch
    return torch


def to_dev(a):
    torch = cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(-1)).cuda()


def gpu_geom(geom):
    from paper_2602_17892_gb300 import Geom, build
    build.build()
    return Geom.from_geometry(geom)


def gpu_A(G, x):
    torch = cuda()
    from paper_2602_17892_gb300 import ct_forward_A
    y = torch.empty(G.m, device="cuda", dtype=torch.float32)
    ct_forward_A(G, to_dev(x), y)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def gpu_B(G, y):
    torch = cuda()
    from paper_2602_17892_gb300 import ct_back_B
    x = torch.empty(G.n, device="cuda", dtype=torch.float32)
    ct_back_B(G, to_dev(y), x)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64)


def f32(a):
    """FP64 copy of the FP32-rounded array: the input both sides see."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def problem(geom, phantom_seed, eta, noise_seed):
    """x_true, b (FP32-rounded, as FP64), e, from the oracle's FP64 projector."""
    x = synth.ellipse_phantom(geom.nx, seed=phantom_seed, ny=geom.ny, h=geom.h)
    bt = OP.forward(geom, x).reshape(-1)
    b, e = synth.add_noise(bt, eta, noise_seed)
    return x.reshape(-1), f32(b), e


EPS32 = 2.0 ** -24


def max_filter(a, shape, axes):
    """Largest |a| over each entry and its +-1 neighbours along `axes` (zero outside)."""
    m = np.abs(np.asarray(a, np.float64).reshape(shape))
    out = m.copy()
    for ax in axes:
        for sh in (-1, 1):
            r = np.roll(m, sh, axis=ax)
            idx = [slice(None)] * m.ndim
            idx[ax] = 0 if sh == 1 else -1
            r[tuple(idx)] = 0.0
            out = np.maximum(out, r)
    return out


def assert_elementwise(got, ref, scale, units, what=""):
    """max_i |got_i - ref_i| <= 8 units eps32 scale_i (+ 1 % of the largest such bound): the
    FP32 rounding of a projector entry grows with the number of interpolation positions it
    walks (units) times the magnitudes it interpolates (scale, the operator applied to the
    local maximum of |input|).  Catches a wrong row, bin or pixel that relative L2 hides."""
    got = np.asarray(got, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    scale = np.asarray(scale, np.float64).reshape(-1)
    lim = 8.0 * units * EPS32 * scale
    lim = lim + 1e-2 * lim.max() + 1e-30
    err = np.abs(got - ref)
    i = int(np.argmax(err / lim))
    assert err[i] <= lim[i], (what, i, err[i], lim[i], got[i], ref[i])
