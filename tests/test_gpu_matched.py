"""The matched pair on the GPU: the Joseph adjoint A^T (2D and cone) against the oracle's exact
transpose, the adjoint identity, and the solvers with B = A^T against the oracle's LSQR and
LSMR (Sec. 2: with a matched pair AB-GMRES is LSQR and BA-GMRES is LSMR; hybrid BA-GMRES at a
fixed lambda is hybrid LSMR)."""
import math

import numpy as np
import pytest

import synth
from oracle import proj as OP
from oracle import solver as OS
from tests._common import f32, gpu_A, gpu_geom, problem, rel, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-5
ITER_TOL = 1e-4

GEOMS = {
    "parallel_64_90x95": synth.parallel2d(64, 90, 95),
    "parallel_ragged_37x45": synth.parallel2d(37, 33, 61, pitch=0.83, ny=45, h=1.1),
    "fan_64": synth.fanflat2d(64, 72, 96, 200.0, 320.0),
    "fan_45deg_ties": synth.fanflat2d(40, 8, 64, 120.0, 200.0, angles=np.arange(8) * math.pi / 4),
    "detector_wider_than_image": synth.parallel2d(8, 5, 300, pitch=0.5),
}


def _gpu_AT(G, y):
    import torch
    from paper_2602_17892_gb300 import ct_back_AT
    yd = to_dev(y)
    xd = torch.empty(G.n, dtype=torch.float32, device="cuda")
    ct_back_AT(G, yd, xd)
    torch.cuda.synchronize()
    return xd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_adjoint_matches_oracle_transpose(name):
    g = GEOMS[name]
    y = f32(synth.standard_normal(g.m, 31))
    G = gpu_geom(g)
    assert rel(_gpu_AT(G, y), OP.back_adjoint(g, y).reshape(-1)) <= TOL


def test_adjoint_identity_on_the_gpu():
    """<A x, y> = <x, A^T y> with both operators on the GPU (FP32 arithmetic)."""
    g = GEOMS["fan_64"]
    G = gpu_geom(g)
    x = f32(synth.standard_normal(g.n, 32))
    y = f32(synth.standard_normal(g.m, 33))
    lhs = float(np.dot(gpu_A(G, x).astype(np.float64), y.astype(np.float64)))
    rhs = float(np.dot(x.astype(np.float64), _gpu_AT(G, y)))
    assert abs(lhs - rhs) <= 1e-5 * math.sqrt(abs(lhs) * abs(rhs)) + 1e-9


def _solve(method, G, b, iters, rule, **kw):
    import torch
    from paper_2602_17892_gb300 import ab_gmres_hybrid, ba_gmres_hybrid
    x = torch.zeros(G.n, dtype=torch.float32, device="cuda")
    fn = ab_gmres_hybrid if method == "ab" else ba_gmres_hybrid
    info = fn(G, to_dev(b), x, max_iters=iters, rule=rule, **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64), info


@pytest.mark.parametrize("k", [4, 8])
def test_matched_solvers_are_lsqr_and_lsmr(k):
    """lambda = 0 at small k (without regularisation FP32 noise grows quickly with k, most for
    BA, whose operator is A^T A); hybrid BA at lambda = 50 over 15 steps."""
    from paper_2602_17892_gb300 import ct_geom_set_backprojector
    case = synth.small_parallel_case()
    g = case["geom"]
    _, b, _ = problem(g, case["phantom_seed"], case["eta"], case["noise_seed"])
    G = gpu_geom(g)
    ct_geom_set_backprojector(G, "adjoint")
    A, At = OP.operators(g, matched=True)
    xab, iab = _solve("ab", G, b, k, "none")
    xba, iba = _solve("ba", G, b, k, "none")
    assert iab["iters_done"] == k and iba["iters_done"] == k
    assert rel(xab, OS.lsqr_iterate(A, At, b, k)) <= ITER_TOL
    assert rel(xba, OS.lsmr_iterate(A, At, b, k)) <= ITER_TOL
    lam = 50.0      # about 1 % of the largest singular value of the projected A^T A
    xh, _ = _solve("ba", G, b, 15, "fixed", lambda_fixed=lam)
    assert rel(xh, OS.lsmr_iterate(A, At, b, 15, lam)) <= ITER_TOL
    # the geometry's B switches back: the unmatched solve differs from the matched one
    ct_geom_set_backprojector(G, "pixel")
    xu, _ = _solve("ab", G, b, k, "none")
    assert rel(xu, xab) > 1e-3


def _cone(nx, ny, nz, n_views, ndu, ndv, pu, pv, sid, sdd, h=1.0, angles=None):
    ang = synth.uniform_angles(n_views, 2 * math.pi) if angles is None else np.asarray(angles, float)
    return synth.Geometry(synth.CONE3D, nx, ny, nz, h, ang, ndu, ndv, pu, pv, float(sid), float(sdd))


CONES = {
    "cone_32": synth.cone3d(32, 30, 48, 40, 100.0, 160.0),
    "cone_ragged_40x36x20": _cone(40, 36, 20, 37, 56, 29, 1.3, 1.2, 90.0, 150.0, h=1.1),
    "cone_45deg_ties": _cone(24, 24, 16, 8, 40, 24, 1.5, 1.5, 60.0, 100.0,
                             angles=np.arange(8) * math.pi / 4),
    "cone_z_driven_rows": _cone(24, 20, 40, 12, 40, 64, 1.5, 4.0, 40.0, 80.0),
}


@pytest.mark.parametrize("name", sorted(CONES))
def test_cone_adjoint_matches_oracle_transpose(name):
    g = CONES[name]
    y = f32(synth.standard_normal(g.m, 41))
    G = gpu_geom(g)
    assert rel(_gpu_AT(G, y), OP.back_adjoint(g, y).reshape(-1)) <= TOL


def test_matched_cone_ab_is_lsqr():
    """B = A^T on a small cone problem: AB-GMRES (lambda = 0) is LSQR."""
    from paper_2602_17892_gb300 import ct_geom_set_backprojector
    g = _cone(24, 24, 16, 20, 36, 20, 1.5, 1.5, 60.0, 100.0)
    x_true = synth.ellipsoid_phantom(24, seed=2)[:16]
    b, _ = synth.add_noise(OP.forward(g, x_true).reshape(-1), 0.01, 77)
    b = f32(b)
    G = gpu_geom(g)
    ct_geom_set_backprojector(G, "adjoint")
    A, At = OP.operators(g, matched=True)
    x, info = _solve("ab", G, b, 6, "none")
    assert info["iters_done"] == 6
    assert rel(x, OS.lsqr_iterate(A, At, b, 6)) <= ITER_TOL
