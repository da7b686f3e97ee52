"""Failure detection on the GPU, in the forms that leave the GPU healthy.

* Non-finite data: a NaN planted in b on the host makes the first normalisation record
  CT_ENONFINITE; the solver returns that status, the output holds the initial guess (zero), and
  the next solve on the same geometry is correct.
* A bounded wait that runs out: the test hook leaves the asynchronous copies of one tile of a
  Gram-Schmidt pass unissued (nothing is in flight for them), so that block's mbarrier waits give
  up after a short limit; the pass records CT_ETIMEOUT, the rest of the solve is skipped, and
  the next solve on the same geometry is correct.  No fault, trap or unbounded wait is used.
"""
import numpy as np
import pytest

import synth
from oracle import proj as OP
from oracle import solver as OS
from tests._common import gpu_geom, problem, rel, to_dev

pytestmark = pytest.mark.gpu


def _setup():
    g = synth.fanflat2d(45, 60, 70, 150.0, 240.0, ny=38)
    x_true, b, e = problem(g, 5, 0.02, 77)
    return g, b


def _solve(method, G, b, **kw):
    import torch
    from paper_2602_17892_gb300 import ab_gmres_hybrid, ba_gmres_hybrid
    x = torch.full((G.n,), 3.0, dtype=torch.float32, device="cuda")
    fn = ab_gmres_hybrid if method == "ab" else ba_gmres_hybrid
    info = fn(G, to_dev(b), x, max_iters=10, rule="gcv", **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64), info


def _check_recovers(method, g, G, b):
    xg, info = _solve(method, G, b)
    assert info["status"] == "CT_OK" and info["iters_done"] == 10
    A, B = OP.operators(g)
    ref = OS.hybrid_gmres(method, A, B, b, 10, rule="fixed", lam_fixed=info["lambdas"][-1])
    assert rel(xg, ref["x"]) <= 1e-4


@pytest.mark.parametrize("method", ["ab", "ba"])
def test_nan_in_the_data_returns_enonfinite(method):
    from paper_2602_17892_gb300 import _binding as Bn
    g, b = _setup()
    G = gpu_geom(g)
    bad = b.copy()
    bad[123] = np.nan
    with pytest.raises(Bn.CtError) as ei:
        _solve(method, G, bad)
    assert ei.value.status == Bn.CT_ENONFINITE
    assert b"non-finite" in Bn.load().ct_last_error()
    _check_recovers(method, g, G, b)


@pytest.mark.parametrize("method", ["ab", "ba"])
def test_expired_bounded_wait_returns_etimeout(method):
    import torch
    from paper_2602_17892_gb300 import _binding as Bn
    g, b = _setup()
    G = gpu_geom(g)
    _check_recovers(method, g, G, b)          # the tile path runs on this geometry
    Bn.ct_test_drop_tile_copy(True, 1 << 20)
    try:
        with pytest.raises(Bn.CtError) as ei:
            _solve(method, G, b)
        assert ei.value.status == Bn.CT_ETIMEOUT
        assert b"bounded device wait" in Bn.load().ct_last_error()
    finally:
        Bn.ct_test_drop_tile_copy(False)
    torch.cuda.synchronize()                  # the context is still usable
    _check_recovers(method, g, G, b)
