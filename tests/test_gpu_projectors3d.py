"""3D cone-beam projectors on the GPU vs the FP64 oracle (relative L2 <= 1e-5 on the same
FP32-rounded input), at sizes the oracle finishes in seconds, with ragged volumes, view
angles that tie the driving axes, and detector rows steep enough to drive along z; at the
512^3 / 400-view / 768 x 768 cone workload, sampled rays and voxels against the oracle's
single-ray and single-voxel functions; and hybrid AB-GMRES on a small cone problem against the
oracle iterate."""
import math

import numpy as np
import pytest

import synth
from oracle import proj as OP
from oracle import solver as OS
from tests._common import (assert_elementwise, f32, gpu_A, gpu_B, gpu_geom, max_filter, rel,
                           to_dev)

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _cone(nx, ny, nz, n_views, ndu, ndv, pu, pv, sid, sdd, h=1.0, angles=None):
    ang = synth.uniform_angles(n_views, 2 * math.pi) if angles is None else np.asarray(angles, float)
    return synth.Geometry(synth.CONE3D, nx, ny, nz, h, ang, ndu, ndv, pu, pv, float(sid), float(sdd))


GEOMS = {
    "cone_32": synth.cone3d(32, 30, 48, 40, 100.0, 160.0),
    "cone_ragged_40x36x20": _cone(40, 36, 20, 37, 56, 29, 1.3, 1.2, 90.0, 150.0, h=1.1),
    "cone_45deg_ties": _cone(24, 24, 16, 8, 40, 24, 1.5, 1.5, 60.0, 100.0,
                             angles=np.arange(8) * math.pi / 4),
    "cone_z_driven_rows": _cone(24, 20, 40, 12, 40, 64, 1.5, 4.0, 40.0, 80.0),
    "cone_1x1x1": _cone(1, 1, 1, 3, 3, 3, 1.0, 1.0, 10.0, 20.0),
}


def _volume(g, seed):
    base = synth.ellipsoid_phantom(max(g.nx, g.ny, g.nz), seed=seed, h=g.h)
    vol = base[:g.nz, :g.ny, :g.nx]
    return f32(vol + 0.1 * synth.standard_normal(vol.shape, seed + 1))


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_forward_matches_oracle_3d(name):
    g = GEOMS[name]
    x = _volume(g, 3)
    G = gpu_geom(g)
    assert (G.n, G.m) == (g.n, g.m)
    yg = gpu_A(G, x)
    yo = OP.forward(g, x).reshape(-1)
    assert rel(yg, yo) <= TOL
    scale = OP.forward(g, max_filter(x, g.image_shape, (0, 1, 2)))
    assert_elementwise(yg, yo, scale, max(g.nx, g.ny, g.nz), "A")


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_backprojector_matches_oracle_3d(name):
    g = GEOMS[name]
    y = f32(np.abs(synth.standard_normal(g.m, 11)) + 1.0)
    G = gpu_geom(g)
    xg = gpu_B(G, y)
    xo = OP.back_pixel(g, y).reshape(-1)
    assert rel(xg, xo) <= TOL
    scale = OP.back_pixel(g, max_filter(y, g.sino_shape, (1, 2)))
    assert_elementwise(xg, xo, scale, max(g.n_det_u, g.n_det_v, g.n_views), "B")


def test_z_driven_rows_exist_in_that_geometry():
    """The steep geometry really has rays whose largest direction component is z."""
    g = GEOMS["cone_z_driven_rows"]
    v_max = (g.n_det_v - 1) / 2 * g.pitch_v
    assert v_max > g.sdd        # |D_z| = |v| exceeds the in-plane component (about SDD)


def test_cone512_workload_sampled_against_oracle():
    """The 512^3 volume, 400 views, 768 x 768 detector: the full A and B on the GPU, 256
    random rays and 256 random voxels recomputed one by one by the oracle."""
    import torch
    from paper_2602_17892_gb300 import ct_back_B, ct_forward_A
    case = synth.cone512_case()
    g = case["geom"]
    x64 = synth.ellipsoid_phantom(512, seed=case["phantom_seed"])
    x32 = x64.astype(np.float32)
    x64 = x32.astype(np.float64)
    G = gpu_geom(g)
    xd = torch.from_numpy(x32.reshape(-1)).cuda()
    yd = torch.empty(G.m, dtype=torch.float32, device="cuda")
    ct_forward_A(G, xd, yd)
    rng = np.random.Generator(np.random.PCG64(5))
    idx = rng.integers(0, g.m, 256)
    yg = yd[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    nu, nv = g.n_det_u, g.n_det_v
    yo = np.array([OP.forward_ray(g, x64, int(i // (nu * nv)), int(i % nu), int((i // nu) % nv))
                   for i in idx])
    assert rel(yg, yo) <= TOL
    # B of the GPU sinogram, sampled voxels against the oracle on the same FP32 sinogram
    xb = torch.empty(G.n, dtype=torch.float32, device="cuda")
    ct_back_B(G, yd, xb)
    y64 = yd.cpu().numpy().astype(np.float64)
    vidx = rng.integers(0, g.n, 256)
    xg = xb[torch.from_numpy(vidx).cuda()].cpu().numpy().astype(np.float64)
    xo = np.array([OP.back_pixel_one(g, y64, int(i // (512 * 512)), int((i // 512) % 512), int(i % 512))
                   for i in vidx])
    assert rel(xg, xo) <= TOL


@pytest.mark.parametrize("basis,tol", [("f32", 1e-4), ("bf16", 2e-2)])
def test_hybrid_ab_on_a_cone_problem(basis, tol):
    import torch
    from paper_2602_17892_gb300 import ab_gmres_hybrid
    g = _cone(24, 24, 16, 20, 36, 20, 1.5, 1.5, 60.0, 100.0)
    x_true = synth.ellipsoid_phantom(24, seed=2)[:16]
    bt = OP.forward(g, x_true).reshape(-1)
    b, _ = synth.add_noise(bt, 0.01, 77)
    b = f32(b)
    G = gpu_geom(g)
    x = torch.zeros(G.n, dtype=torch.float32, device="cuda")
    out = ab_gmres_hybrid(G, to_dev(b), x, max_iters=10, rule="gcv", basis=basis)
    A, B = OP.operators(g)
    ref = OS.hybrid_gmres("ab", A, B, b, 10, rule="gcv")
    assert out["iters_done"] == 10
    assert rel(x.cpu().numpy(), ref["x"]) <= tol


def test_autotuned_slab_thickness_keeps_the_result():
    """The 3D autotuner picks a z-slab thickness; A is the same up to summation order."""
    from paper_2602_17892_gb300 import ct_geom_autotune
    g = GEOMS["cone_32"]
    x = _volume(g, 4)
    G = gpu_geom(g)
    y_default = gpu_A(G, x)
    sh = ct_geom_autotune(G)
    assert (sh["a_slab"], sh["a_views"], sh["a_rays"]) in (
        (16, 1, 1), (16, 4, 1), (16, 8, 1), (64, 4, 1), (64, 8, 1), (1 << 20, 1, 1),
        (1 << 20, 4, 1), (1 << 20, 8, 1), (16, 4, 2), (64, 4, 2), (1 << 20, 2, 2), (1 << 20, 4, 2))
    y_tuned = gpu_A(G, x)
    assert rel(y_tuned, y_default) <= 1e-6
    assert rel(y_tuned, OP.forward(g, x).reshape(-1)) <= TOL


def test_cone64_k100_iterates_match_oracle():
    """The cone workload on a reduced copy the oracle solves in about a minute: 64^3 ellipsoids,
    100 views over 360 deg, 96 x 96 detector (SID, SDD scaled by 64/512), 1 % noise, hybrid
    AB-GMRES with K = 100 and GCV.  The FP32-basis iterate is compared with the oracle's
    iterate at the lambda the GPU's GCV chose (GCV is flat near its minimum); the BF16-basis
    solve at that same lambda is compared with the same oracle iterate: its error is stated
    and bounded by the 16-bit storage (2^-8 relative per entry, 2e-2 as for the fan problem)."""
    import torch
    from paper_2602_17892_gb300 import ab_gmres_hybrid
    case = synth.cone512_case(64)
    g = synth.cone3d(64, 100, 96, 96, 1000.0 * 64 / 512, 1500.0 * 64 / 512)
    x_true = synth.ellipsoid_phantom(64, seed=case["phantom_seed"])
    b, _ = synth.add_noise(OP.forward(g, x_true).reshape(-1), 0.01, case["noise_seed"])
    b = f32(b)
    G = gpu_geom(g)
    x = torch.zeros(G.n, dtype=torch.float32, device="cuda")
    out = ab_gmres_hybrid(G, to_dev(b), x, max_iters=100, rule="gcv")
    torch.cuda.synchronize()
    assert out["iters_done"] == 100
    lam = float(out["lambdas"][-1])
    xf32 = x.cpu().numpy().astype(np.float64)
    x.zero_()
    ab_gmres_hybrid(G, to_dev(b), x, max_iters=100, rule="fixed", lambda_fixed=lam, basis="bf16")
    torch.cuda.synchronize()
    xbf16 = x.cpu().numpy().astype(np.float64)
    A, B = OP.operators(g)
    ref = OS.hybrid_gmres("ab", A, B, b, 100, rule="fixed", lam_fixed=lam)["x"]
    err32, err16 = rel(xf32, ref), rel(xbf16, ref)
    print(f"cone 64^3 K=100: FP32 basis {err32:.2e}, BF16 basis {err16:.2e} vs FP64")
    assert err32 <= 1e-4, err32
    assert err16 <= 2e-2, err16


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_two_rays_per_thread_is_bitwise_the_single_ray_kernel(name):
    """The cone Joseph kernel with two detector rows per thread (shared in-plane coordinate)
    performs each ray's operations in the same order as the one-ray kernel: A agrees bit for
    bit across rays per thread, warp rows per block and z-slab thickness, including rays
    driven along z, ragged volumes and odd detector row counts."""
    from paper_2602_17892_gb300 import ct_geom_get_launch_shapes, ct_geom_set_launch_shapes
    g = GEOMS[name]
    x = _volume(g, 6)
    G = gpu_geom(g)
    base = ct_geom_get_launch_shapes(G)
    yo = OP.forward(g, x).reshape(-1)
    one_pass = None
    for slab in (1 << 20, 16, 3):
        ref = None                        # slabs add per-slab partial sums: one order per slab
        for views, rays in ((1, 1), (4, 1), (8, 1), (1, 2), (2, 2), (4, 2), (8, 2)):
            ct_geom_set_launch_shapes(G, dict(base, a_slab=slab, a_views=views, a_rays=rays))
            y = gpu_A(G, x)
            if ref is None:
                ref = y
                assert rel(y, yo) <= TOL
                one_pass = y if one_pass is None else one_pass
                assert rel(y, one_pass) <= 1e-6
            assert np.array_equal(y, ref), (slab, views, rays)
