"""GPU projectors vs the FP64 oracle (relative L2 <= 1e-5 on the same FP32-rounded input)."""
import math

import numpy as np
import pytest

import synth
from oracle import proj as OP
from tests._common import assert_elementwise, f32, gpu_A, gpu_B, gpu_geom, max_filter, rel

pytestmark = pytest.mark.gpu
TOL = 1e-5

GEOMS = {
    "parallel_64_90x95": synth.parallel2d(64, 90, 95),
    "parallel_ragged_37x45": synth.parallel2d(37, 33, 61, pitch=0.83, ny=45, h=1.1),
    "parallel_45deg_ties": synth.parallel2d(40, 8, 60, angles=np.arange(8) * math.pi / 4),
    "fan_64": synth.fanflat2d(64, 72, 96, 200.0, 320.0),
    "fan_ragged_50x33": synth.fanflat2d(50, 37, 77, 150.0, 260.0, ny=33, h=0.9),
    "fan_45deg_ties": synth.fanflat2d(40, 8, 64, 120.0, 200.0, angles=np.arange(8) * math.pi / 4),
    "tiny_1x1_1view_1bin": synth.parallel2d(1, 1, 1),
    "detector_wider_than_image": synth.parallel2d(8, 5, 300, pitch=0.5),
}


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_forward_matches_oracle(name):
    g = GEOMS[name]
    x = f32(synth.ellipse_phantom(g.nx, seed=3, ny=g.ny, h=g.h) + 0.1 * synth.standard_normal(g.image_shape, 9))
    G = gpu_geom(g)
    yg = gpu_A(G, x)
    yo = OP.forward(g, x).reshape(-1)
    assert rel(yg, yo) <= TOL
    _check_A_entries(g, x, yg, yo)


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_backprojector_matches_oracle(name):
    g = GEOMS[name]
    y = f32(np.abs(synth.standard_normal(g.m, 11)) + 1.0)
    G = gpu_geom(g)
    xg = gpu_B(G, y)
    xo = OP.back_pixel(g, y).reshape(-1)
    assert rel(xg, xo) <= TOL
    _check_B_entries(g, y, xg, xo)


def _check_A_entries(g, x, yg, yo):
    """Every ray, not just the norm: |A_gpu x - A x| within the FP32 bound of that ray."""
    scale = OP.forward(g, max_filter(x, g.image_shape, range(len(g.image_shape))))
    assert_elementwise(yg, yo, scale, max(g.nx, g.ny, g.nz), "A")


def _check_B_entries(g, y, xg, xo):
    """Every pixel: |B_gpu y - B y| within the FP32 bound of that pixel."""
    axes = (1, 2) if g.kind == synth.CONE3D else (1,)
    scale = OP.back_pixel(g, max_filter(y, g.sino_shape, axes))
    assert_elementwise(xg, xo, scale, max(g.n_det_u, g.n_det_v, g.n_views), "B")


def test_fan512_full_size_projectors():
    """The 512^2 fan-beam workload (720 views x 768 bins): full A and B against the oracle."""
    g = synth.fan512_case()["geom"]
    x = f32(synth.ellipse_phantom(512, seed=0))
    G = gpu_geom(g)
    yg, yo = gpu_A(G, x), OP.forward(g, x).reshape(-1)
    assert rel(yg, yo) <= TOL
    _check_A_entries(g, x, yg, yo)
    y = f32(yo)
    xg, xo = gpu_B(G, y), OP.back_pixel(g, y).reshape(-1)
    assert rel(xg, xo) <= TOL
    _check_B_entries(g, y, xg, xo)


def test_projectors_are_linear_and_unmatched():
    g = GEOMS["fan_64"]
    G = gpu_geom(g)
    x1 = f32(synth.standard_normal(g.n, 1))
    y1 = f32(synth.standard_normal(g.m, 2))
    lhs = float(gpu_A(G, x1) @ y1)
    rhs_bt = float(x1 @ gpu_B(G, y1))
    rhs_at = float(x1 @ OP.back_adjoint(g, y1).reshape(-1))
    assert abs(lhs - rhs_at) <= 1e-5 * abs(lhs) + 1e-3
    assert abs(lhs - rhs_bt) > 1e-4 * abs(lhs)      # B is not A^T


@pytest.mark.parametrize("name", ["fan_64", "fan_ragged_50x33", "parallel_ragged_37x45"])
def test_launch_shapes_leave_results_bitwise_unchanged(name):
    """Every 2D launch shape (threads, views per Joseph block and views per Joseph warp; pixel
    rows per B block, one or two views per B iteration and pixel rows per B warp) computes each
    ray and pixel with the same operations in the same order: A and B agree bit for bit across
    shapes, on images and detectors that fill neither the blocks nor the warps' tiles."""
    from paper_2602_17892_gb300 import ct_geom_get_launch_shapes, ct_geom_set_launch_shapes
    g = GEOMS[name]
    G = gpu_geom(g)
    x = f32(synth.standard_normal(g.n, 21))
    y = f32(synth.standard_normal(g.m, 22))
    base = ct_geom_get_launch_shapes(G)
    ya, xb = gpu_A(G, x), gpu_B(G, y)
    for a_threads, a_views, a_wv in ((128, 1, 1), (256, 2, 1), (512, 8, 1), (128, 4, 1),
                                     (128, 2, 2), (128, 4, 4), (256, 8, 8), (512, 8, 4),
                                     (128, 8, 8)):
        sh = dict(base, a_threads=a_threads, a_views=a_views, a_warp_views=a_wv)
        ct_geom_set_launch_shapes(G, sh)
        assert ct_geom_get_launch_shapes(G) == sh
        assert np.array_equal(gpu_A(G, x), ya)
    for b_rows, b_views, b_wr in ((4, 1, 1), (8, 2, 1), (16, 1, 1), (4, 2, 1), (4, 1, 4),
                                  (8, 1, 2), (16, 1, 4), (4, 2, 2), (8, 2, 4)):
        sh = dict(base, b_rows=b_rows, b_views=b_views, b_warp_rows=b_wr)
        ct_geom_set_launch_shapes(G, sh)
        assert ct_geom_get_launch_shapes(G) == sh
        assert np.array_equal(gpu_B(G, y), xb)


def test_warp_shapes_out_of_range_are_rejected():
    """Views per Joseph warp must divide the views per block and leave a warp no more bins than
    the block has; pixel rows per B warp must fit the block's (orbit) rows.  A refused shape
    leaves the geometry's shapes unchanged."""
    from paper_2602_17892_gb300 import _binding as Bn
    from paper_2602_17892_gb300 import ct_geom_get_launch_shapes, ct_geom_set_launch_shapes
    G = gpu_geom(GEOMS["fan_64"])
    base = ct_geom_get_launch_shapes(G)
    for bad in (dict(a_threads=128, a_views=2, a_warp_views=4),
                dict(a_threads=128, a_views=8, a_warp_views=1),
                dict(a_threads=128, a_views=4, a_warp_views=3),
                dict(b_rows=4, b_views=1, b_warp_rows=8),
                dict(b_rows=4, b_views=4, b_warp_rows=4),      # four-fold: 2 orbit rows
                dict(b_rows=16, b_views=4, b_warp_rows=4)):
        with pytest.raises(Bn.CtError):
            ct_geom_set_launch_shapes(G, dict(base, **bad))
        assert ct_geom_get_launch_shapes(G) == base


@pytest.mark.parametrize("kind", ["parallel", "fan"])
def test_backprojector_view_chunks(kind):
    """More views than one chunk of the round-down floor's offset range (2^22 floats of padded
    sinogram): 501 views of 19001 bins make chunks of 220 views, so the paired loop meets full
    chunks of 13 gather batches and 6 single pairs, a last chunk of 3 batches and 6 pairs, and
    an odd last view; every B launch shape agrees with the oracle and bit for bit with the
    others."""
    from paper_2602_17892_gb300 import ct_geom_get_launch_shapes, ct_geom_set_launch_shapes
    if kind == "parallel":
        g = synth.parallel2d(16, 501, 19001, pitch=0.002)
    else:
        g = synth.fanflat2d(16, 501, 19001, 60.0, 100.0)
    y = f32(np.abs(synth.standard_normal(g.m, 31)) + 1.0)
    G = gpu_geom(g)
    xo = OP.back_pixel(g, y).reshape(-1)
    base = ct_geom_get_launch_shapes(G)
    ref = None
    for b_rows, b_views in ((8, 1), (8, 2), (4, 2), (16, 1)):
        ct_geom_set_launch_shapes(G, dict(base, b_rows=b_rows, b_views=b_views))
        xg = gpu_B(G, y)
        assert rel(xg, xo) <= TOL
        if ref is None:
            ref = xg
        assert np.array_equal(xg, ref)


def test_paired_backprojector_rejects_tall_blocks():
    """The paired-view B kernel is built for blocks of at most 8 pixel rows (256 threads)."""
    from paper_2602_17892_gb300 import _binding as Bn
    from paper_2602_17892_gb300 import ct_geom_get_launch_shapes, ct_geom_set_launch_shapes
    G = gpu_geom(GEOMS["fan_64"])
    base = ct_geom_get_launch_shapes(G)
    with pytest.raises(Bn.CtError):
        ct_geom_set_launch_shapes(G, dict(base, b_rows=16, b_views=2))
    assert ct_geom_get_launch_shapes(G) == base


@pytest.mark.parametrize("name", ["fan_64", "fan512"])
def test_four_fold_backprojector(name):
    """The four-fold B (b_views 4) on fan scans whose views come in quadruples a quarter turn
    apart: each pixel within its element-wise FP32 bound of the oracle, within FP32 rounding of
    the general kernel, and bitwise the same for both block heights with two view parts."""
    from paper_2602_17892_gb300 import ct_geom_get_launch_shapes, ct_geom_set_launch_shapes
    g = GEOMS["fan_64"] if name == "fan_64" else synth.fan512_case()["geom"]
    y = f32(np.abs(synth.standard_normal(g.m, 41)) + 1.0)
    G = gpu_geom(g)
    base = dict(ct_geom_get_launch_shapes(G), b_rows=8, b_views=1)
    ct_geom_set_launch_shapes(G, base)
    x_general = gpu_B(G, y)
    xo = OP.back_pixel(g, y).reshape(-1)
    outs = []
    for rows in (4, 8, 16):
        ct_geom_set_launch_shapes(G, dict(base, b_rows=rows, b_views=4))
        xg = gpu_B(G, y)
        assert rel(xg, xo) <= TOL
        _check_B_entries(g, y, xg, xo)
        assert rel(xg, x_general) <= 1e-6
        outs.append(xg)
        # warps of 16 x 2 (and 8 x 4) orbit positions: the same sums in the same order
        for wr in ((2, 4) if rows == 8 else (2,)):
            ct_geom_set_launch_shapes(G, dict(base, b_rows=rows, b_views=4, b_warp_rows=wr))
            assert np.array_equal(gpu_B(G, y), xg)
    assert np.array_equal(outs[0], outs[1])          # the same two view parts
    assert rel(outs[2], outs[0]) <= 1e-6             # four parts: another order of the sums


NOT_FOUR_FOLD = {
    "ragged_image": GEOMS["fan_ragged_50x33"],
    "half_turn_scan": synth.fanflat2d(64, 72, 96, 200.0, 320.0, angle_range=math.pi),
    "odd_side": synth.fanflat2d(63, 72, 96, 200.0, 320.0),
    "parallel_beam": GEOMS["parallel_64_90x95"],
}


@pytest.mark.parametrize("name", sorted(NOT_FOUR_FOLD))
def test_four_fold_backprojector_needs_the_symmetry(name):
    """Geometries without the quarter-turn symmetry (a ragged image, views over half a turn, an
    odd image side, parallel beam) refuse the four-fold shape and keep their shapes."""
    from paper_2602_17892_gb300 import _binding as Bn
    from paper_2602_17892_gb300 import ct_geom_get_launch_shapes, ct_geom_set_launch_shapes
    G = gpu_geom(NOT_FOUR_FOLD[name])
    base = ct_geom_get_launch_shapes(G)
    with pytest.raises(Bn.CtError):
        ct_geom_set_launch_shapes(G, dict(base, b_rows=8, b_views=4))
    assert ct_geom_get_launch_shapes(G) == base
