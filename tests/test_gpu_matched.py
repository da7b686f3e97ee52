"""The matched pair on the GPU: the Joseph adjoint A^T against the oracle's
exact transpose, the adjoint identity, and the solvers with B = A^T against the oracle's LSQR and
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


def test_adjoint_refuses_cone_geometries():
    from paper_2602_17892_gb300 import CtError, ct_geom_set_backprojector
    g = synth.cone3d(16, 8, 24, 16, 100.0, 160.0)
    G = gpu_geom(g)
    with pytest.raises(CtError):
        ct_geom_set_backprojector(G, "adjoint")
