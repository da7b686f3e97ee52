"""Batched solves (ct_batch / abba_solve): many uneven problems in one captured CUDA graph.

Each problem in a batch runs the same kernels on the same data as its single-problem solve, so
at the same launch shapes the iterates must agree with ab_gmres_hybrid / ba_gmres_hybrid (to
rounding: the batch caps the Gram-Schmidt passes at one block per SM, which only reorders their
FP32 block sums on large problems) and, through them, with the FP64 oracle.  Launch shapes
leave a ray's and a pixel's arithmetic unchanged except for the four-fold backprojector, whose
view parts reorder each pixel's sum.
"""
import numpy as np
import pytest

import synth
from oracle import proj as OP
from oracle import solver as OS
from tests._common import gpu_geom, problem, rel, to_dev

pytestmark = pytest.mark.gpu


def _cases():
    return [
        (synth.parallel2d(40, 30, 61), "ab"),
        (synth.fanflat2d(56, 44, 90, 160.0, 260.0, ny=48), "ba"),
        (synth.parallel2d(64, 24, 95), "auto"),
        (synth.fanflat2d(33, 60, 50, 120.0, 200.0), "ab"),
        (synth.parallel2d(48, 90, 72, ny=36), "ba"),
        (synth.fanflat2d(72, 16, 110, 220.0, 330.0), "auto"),
    ]


def _single(G, method, b, K, rule, **kw):
    import torch
    from paper_2602_17892_gb300 import ab_gmres_hybrid, ba_gmres_hybrid
    x = torch.zeros(G.n, dtype=torch.float32, device="cuda")
    fn = ab_gmres_hybrid if method == "ab" else ba_gmres_hybrid
    fn(G, to_dev(b), x, max_iters=K, rule=rule, history=False, **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("rule", ["gcv", "dp"])
def test_batch_matches_single_solves_and_oracle(rule):
    import torch
    from paper_2602_17892_gb300 import Batch, ct_geom_get_launch_shapes, ct_geom_set_launch_shapes
    cases = _cases()
    data, geoms, methods, noises = [], [], [], []
    for i, (g, m) in enumerate(cases):
        x_true, b, e = problem(g, 100 + i, 0.01, 200 + i)
        mm = m if m != "auto" else ("ab" if g.m < g.n else "ba")
        noise = np.linalg.norm(e) if mm == "ab" else np.linalg.norm(OP.back_pixel(g, e))
        data.append((g, mm, b, noise))
        geoms.append(gpu_geom(g))
        methods.append(m)
        noises.append(noise)
    K = 12
    bt = Batch(geoms, methods, max_iters=K, rule=rule, tau=1.01)
    bs = [to_dev(d[2]) for d in data]
    xs = [torch.zeros(G.n, dtype=torch.float32, device="cuda") for G in geoms]
    infos = bt.solve(bs, xs, noise_norms=noises)
    assert bt.launches() > 0
    for i, (g, mm, b, noise) in enumerate(data):
        assert infos[i]["iters_done"] == K, infos[i]
        xb = xs[i].cpu().numpy().astype(np.float64)
        # the single solve with the launch shapes the batch's autotuner chose for this problem:
        # shapes only reorder FP32 sums, and a GCV minimiser moves with such rounding by up to
        # ~sqrt(eps), so the comparison is made at equal shapes
        G1 = gpu_geom(g)
        ct_geom_set_launch_shapes(G1, ct_geom_get_launch_shapes(geoms[i]))
        xs1 = _single(G1, mm, b, K, rule, noise_norm=noise, tau=1.01)
        assert rel(xb, xs1) <= 1e-6, i
        if i in (0, 1):
            A, B = OP.operators(g)
            ref = OS.hybrid_gmres(mm, A, B, b, K, rule=rule, dp_target=1.01 * noise)
            assert rel(xb, ref["x"]) <= 1e-4, i
    # replay with new data in the same buffers: the graph reads the buffers' contents
    x_first = [x.clone() for x in xs]
    for i, (g, mm, b, noise) in enumerate(data):
        bs[i].copy_(to_dev(2.0 * b))
    infos2 = bt.solve(bs, xs, noise_norms=[2.0 * nz for nz in noises])
    for i in range(len(data)):
        assert rel(xs[i].cpu().numpy(), 2.0 * x_first[i].cpu().numpy()) <= 1e-4, i
    bt.close()


def test_abba_solve_one_shot_and_breakdown_inside_batch():
    import torch
    from paper_2602_17892_gb300 import abba_solve, ct_geom_autotune
    g1 = synth.parallel2d(32, 20, 49)
    g2 = synth.fanflat2d(40, 30, 64, 150.0, 240.0)
    x1, b1, e1 = problem(g1, 7, 0.01, 8)
    G1, G2 = gpu_geom(g1), gpu_geom(g2)
    sh = ct_geom_autotune(G2)
    # the autotuner's candidates (threads, views per block, views per warp) for the Joseph A and
    # (pixel rows per block, views per iteration, pixel rows per warp) for B; this scan has no
    # four-fold symmetry (30 views), so B's four-fold shapes are not among them
    assert (sh["a_threads"], sh["a_views"], sh["a_warp_views"]) in (
        (128, 1, 1), (128, 2, 1), (128, 4, 1), (256, 1, 1), (256, 2, 1), (256, 4, 1), (512, 4, 1),
        (512, 8, 1), (128, 2, 2), (128, 4, 2), (128, 4, 4), (256, 4, 4), (256, 8, 4), (256, 8, 8),
        (512, 8, 4))
    assert (sh["b_rows"], sh["b_views"], sh["b_warp_rows"]) in tuple(
        (rows, views, wr) for wr in (1, 2, 4) for rows, views in ((4, 1), (8, 1), (16, 1), (4, 2),
                                                                  (8, 2)))
    bs = [to_dev(b1), torch.zeros(G2.m, dtype=torch.float32, device="cuda")]
    xs = [torch.zeros(G.n, dtype=torch.float32, device="cuda") for G in (G1, G2)]
    infos = abba_solve([G1, G2], bs, xs, methods=["ab", "ab"], max_iters=8, rule="gcv")
    assert infos[0]["status"] == "CT_OK" and infos[0]["iters_done"] == 8
    assert infos[1]["status"] == "CT_BREAKDOWN" and infos[1]["iters_done"] == 0
    assert torch.all(xs[1] == 0)
    A, B = OP.operators(g1)
    ref = OS.hybrid_gmres("ab", A, B, b1, 8, rule="gcv")
    assert rel(xs[0].cpu().numpy(), ref["x"]) <= 1e-4
