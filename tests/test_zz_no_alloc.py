"""The allocation-free Arnoldi step (ct_arnoldi_step_noalloc) against the allocating entry
point (ct_arnoldi_step), through the C ABI, on two calls in a row.

The allocation-free variant is for callers that must not allocate device memory while they
run: cudaFree synchronises the whole device (it would stall acquisition or other work running
on other streams), and an application that reserves the GPU's memory through its own pool
cannot let a library take more.  Its scratch is a static device array shared by every call.
This file is collected last so that a run stopping at the first failure has run all others.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL_H = 1e-5       # the Arnoldi-step tolerance used by the other GPU tests
TOL_W = 1e-4


def _inputs(L, k, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    Q, _ = np.linalg.qr(rng.standard_normal((L, k + 1)))
    W = np.zeros((k + 2, L), np.float32)
    W[: k + 1] = Q.T
    q = (rng.standard_normal(L) + 2.0 * Q[:, -1]).astype(np.float32)
    return W, q


def _run(fn, W, q, L, k):
    import torch
    Wd = torch.from_numpy(W.copy()).cuda()
    qd = torch.from_numpy(q.copy()).cuda()
    hd = torch.full((k + 2,), float("nan"), dtype=torch.float64, device="cuda")
    fn(Wd, L, L, k, qd, hd)
    torch.cuda.synchronize()
    return hd.cpu().numpy(), Wd[k + 1].cpu().numpy().astype(np.float64)


def test_noalloc_step_matches_allocating_step_twice():
    import torch
    from paper_2602_17892_gb300 import build
    build.build()
    from paper_2602_17892_gb300 import _binding as Bn
    for call, (L, k, seed) in enumerate([(262_144, 9, 1), (100_000, 3, 2)]):
        W, q = _inputs(L, k, seed)
        h_ref, w_ref = _run(Bn.ct_arnoldi_step, W, q, L, k)
        h_new, w_new = _run(Bn.ct_arnoldi_step_noalloc, W, q, L, k)
        assert np.all(np.isfinite(h_new)), f"call {call}"
        assert np.linalg.norm(h_new - h_ref) <= TOL_H * np.linalg.norm(h_ref), f"call {call}"
        assert np.linalg.norm(w_new - w_ref) <= TOL_W * np.linalg.norm(w_ref), f"call {call}"
        assert abs(np.linalg.norm(w_new) - 1.0) <= TOL_H


def _fp64_mgs_twice(W, q, k):
    """FP64 modified Gram-Schmidt, two passes, on the same FP32 inputs (Eq. (Hessenberg))."""
    W64 = W[: k + 1].astype(np.float64)
    qq = q.astype(np.float64)
    h = np.zeros(k + 2)
    for _ in range(2):
        for i in range(k + 1):
            d = qq @ W64[i]
            h[i] += d
            qq -= d * W64[i]
    h[k + 1] = np.linalg.norm(qq)
    return h, qq / h[k + 1]


def test_noalloc_step_at_its_limit_then_smaller_matches_fp64_gram_schmidt():
    """k = 126 fills the static scratch (128 partial-sum columns of each block, the last h
    slot); a smaller step afterwards must not see the previous call's contents."""
    from paper_2602_17892_gb300 import _binding as Bn
    for call, (L, k, seed) in enumerate([(4096, 126, 5), (8192, 17, 6), (4096, 126, 7),
                                         (1024, 0, 8)]):
        W, q = _inputs(L, k, seed)
        h_ref, w_ref = _run(Bn.ct_arnoldi_step, W, q, L, k)
        h_new, w_new = _run(Bn.ct_arnoldi_step_noalloc, W, q, L, k)
        h64, w64 = _fp64_mgs_twice(W, q, k)
        assert np.all(np.isfinite(h_new)), f"call {call}"
        assert np.linalg.norm(h_new - h64) <= TOL_H * np.linalg.norm(h64), f"call {call}"
        assert np.linalg.norm(w_new - w64) <= TOL_W * np.linalg.norm(w64), f"call {call}"
        assert np.linalg.norm(h_new - h_ref) <= TOL_H * np.linalg.norm(h_ref), f"call {call}"
        assert np.linalg.norm(w_new - w_ref) <= TOL_W * np.linalg.norm(w_ref), f"call {call}"


def test_noalloc_step_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2602_17892_gb300 import _binding as Bn
    W, q = _inputs(1024, 0, 3)
    Wd = torch.zeros((129, 1024), dtype=torch.float32, device="cuda")
    qd = torch.from_numpy(q).cuda()
    hd = torch.zeros(130, dtype=torch.float64, device="cuda")
    with pytest.raises(Bn.CtError) as ei:
        Bn.ct_arnoldi_step_noalloc(Wd, 1024, 1024, 127, qd, hd)
    assert ei.value.status == Bn.CT_EINVAL
