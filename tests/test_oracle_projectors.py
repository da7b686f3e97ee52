"""Pins of the FP64 oracle projectors against closed forms and special cases.

Each test ties the oracle to something other than its own formula: exact line integrals of
affine images, the chord length 2 sqrt(R^2 - d^2) of a uniform disc (ball), exact sums at
special angles, the adjoint identity of the matched transpose, the constant response of the
parallel backprojector and the agreement of the backprojector's detector coordinate with the
forward projector's ray geometry.
"""
import math

import numpy as np
import pytest

import synth
from oracle import proj as P


def test_parallel_theta0_is_column_sums():
    h = 0.7
    g = synth.parallel2d(12, 1, n_det=12, pitch=h, ny=9, h=h, angles=[0.0])
    x = synth.standard_normal((9, 12), 1)
    y = P.forward(g, x)
    np.testing.assert_allclose(y[0], h * x.sum(axis=0), rtol=1e-13, atol=1e-13)


def test_parallel_theta90_is_row_sums():
    h = 1.3
    g = synth.parallel2d(10, 1, n_det=7, pitch=h, ny=7, h=h, angles=[math.pi / 2])
    x = synth.standard_normal((7, 10), 2)
    y = P.forward(g, x)
    # theta = 90 deg: the ray of bin j is the horizontal line Y = s_j through row j
    np.testing.assert_allclose(y[0], h * x.sum(axis=1), rtol=1e-13, atol=1e-13)


def _affine_image(g, a0, ax, ay):
    XX, YY = synth.pixel_centres(g.nx, g.ny, g.h)
    return a0 + ax * XX + ay * YY


@pytest.mark.parametrize("theta", [1.2, 1.9, 0.3, 2.9])
def test_parallel_affine_image_exact(theta):
    """Joseph integrates an affine image exactly along rays that stay inside it: the sum of
    equally spaced samples times h/|d_drive| is the segment length times the midpoint value."""
    N, h = 40, 0.5
    g = synth.parallel2d(N, 1, n_det=9, pitch=0.4, h=h, angles=[theta])
    a0, ax, ay = 0.3, 0.11, -0.07
    x = _affine_image(g, a0, ax, ay)
    y = P.forward(g, x)[0]
    ct, st = math.cos(theta), math.sin(theta)
    half = N * h / 2
    for j in range(9):
        s = (j - 4) * 0.4
        p0 = np.array([s * ct, s * st])
        d = np.array([-st, ct])
        if abs(d[0]) >= abs(d[1]):
            t = (0.0 - p0[0]) / d[0]
            length = 2 * half / abs(d[0])
        else:
            t = (0.0 - p0[1]) / d[1]
            length = 2 * half / abs(d[1])
        mid = p0 + t * d
        # every sample must lie inside the pixel-centre grid for the identity to hold
        exact = length * (a0 + ax * mid[0] + ay * mid[1])
        assert abs(y[j] - exact) <= 1e-11 * max(1.0, abs(exact))


def _chord(R, dist):
    return 2.0 * np.sqrt(np.maximum(R * R - dist * dist, 0.0))


@pytest.mark.parametrize("kind", ["parallel", "fan"])
def test_disc_chords_converge(kind):
    """Line integrals of a uniform disc approach 2 sqrt(R^2 - d^2) at rate O(h)."""
    R, centre = 20.0, (6.0, -4.0)
    errs = []
    for N, h in [(64, 1.0), (128, 0.5)]:
        if kind == "parallel":
            g = synth.parallel2d(N, 12, n_det=61, pitch=1.0, h=h)
        else:
            g = synth.fanflat2d(N, 12, 61, 200.0, 300.0, pitch=1.1, h=h)
        x = synth.disc_phantom(N, N, R, centre, h)
        y = P.forward(g, x)
        exact = np.zeros_like(y)
        for v, th in enumerate(g.angles):
            ct, st = math.cos(th), math.sin(th)
            u = (np.arange(g.n_det_u) - (g.n_det_u - 1) / 2) * g.pitch_u
            if kind == "parallel":
                dist = np.abs(u - (centre[0] * ct + centre[1] * st))
            else:
                S = np.array([g.sid * ct, g.sid * st])
                off = g.sdd - g.sid
                Px = -off * ct - u * st
                Py = -off * st + u * ct
                D = np.stack([Px - S[0], Py - S[1]], 1)
                D /= np.linalg.norm(D, axis=1, keepdims=True)
                rel = np.array(centre) - S
                dist = np.abs(rel[0] * D[:, 1] - rel[1] * D[:, 0])
            exact[v] = _chord(R, dist)
        errs.append(np.linalg.norm(y - exact) / np.linalg.norm(exact))
    assert errs[0] < 0.02
    assert errs[1] < 0.7 * errs[0]


def test_ball_chords_converge_cone():
    R, centre = 7.0, np.array([2.0, -1.0, 1.5])
    errs = []
    for N, h in [(24, 1.0), (48, 0.5)]:
        g = synth.cone3d(N, 6, 21, 17, 60.0, 90.0, pitch_u=1.2, pitch_v=1.2, h=h)
        c = (np.arange(N) - (N - 1) / 2) * h
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        x = (((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2) <= R * R) * 1.0
        y = P.forward(g, x)
        exact = np.zeros_like(y)
        for v, th in enumerate(g.angles):
            ct, st = math.cos(th), math.sin(th)
            S = np.array([g.sid * ct, g.sid * st, 0.0])
            off = g.sdd - g.sid
            u = (np.arange(g.n_det_u) - (g.n_det_u - 1) / 2) * g.pitch_u
            w = (np.arange(g.n_det_v) - (g.n_det_v - 1) / 2) * g.pitch_v
            W, U = np.meshgrid(w, u, indexing="ij")
            Pt = np.stack([-off * ct - U * st, -off * st + U * ct, W], -1)
            D = Pt - S
            D /= np.linalg.norm(D, axis=-1, keepdims=True)
            rel = centre - S
            proj = (D * rel).sum(-1)
            dist = np.sqrt(np.maximum((rel * rel).sum() - proj ** 2, 0.0))
            exact[v] = _chord(R, dist)
        errs.append(np.linalg.norm(y - exact) / np.linalg.norm(exact))
    assert errs[0] < 0.08      # R = 7 voxels: boundary voxels dominate at h = 1
    assert errs[1] < 0.7 * errs[0]


@pytest.mark.parametrize("geom", [
    synth.parallel2d(11, 7, n_det=15, ny=9),
    synth.fanflat2d(10, 9, 13, 40.0, 70.0),
    synth.cone3d(6, 5, 9, 7, 30.0, 50.0),
])
def test_matched_adjoint_identity(geom):
    x = synth.standard_normal(geom.n, 3)
    y = synth.standard_normal(geom.m, 4)
    lhs = float(P.forward(geom, x).reshape(-1) @ y)
    rhs = float(x @ P.back_adjoint(geom, y).reshape(-1))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_parallel_backprojector_of_ones():
    """B 1 = n_views h^2 / pitch at pixels whose projection stays inside the detector."""
    h, pitch = 0.8, 0.6
    g = synth.parallel2d(16, 13, n_det=64, pitch=pitch, h=h)
    xb = P.back_pixel(g, np.ones(g.m))
    np.testing.assert_allclose(xb, 13 * h * h / pitch * np.ones_like(xb), rtol=1e-13)


def test_parallel_backprojector_theta0():
    h = 0.9
    g = synth.parallel2d(8, 1, n_det=8, pitch=h, ny=5, h=h, angles=[0.0])
    y = synth.standard_normal((1, 8), 5)
    xb = P.back_pixel(g, y)
    np.testing.assert_allclose(xb, np.tile(h * h / h * y[0], (5, 1)), rtol=1e-13)


def _geoms_for_scale(kind, nd):
    if kind == "parallel":
        return synth.parallel2d(32, 90, nd, pitch=64 / nd * 0.95)
    if kind == "fan":
        return synth.fanflat2d(32, 90, nd, 80.0, 130.0)
    return synth.cone3d(12, 40, nd, int(nd * 0.8), 40.0, 60.0)


@pytest.mark.parametrize("kind", ["parallel", "fan", "cone"])
def test_backprojector_has_scale_of_transpose(kind):
    """B 1 agrees with A^T 1 (the exact transpose) at interior pixels: the backprojector
    weights h^2/(ray spacing) reproduce A's column sums; the spread shrinks with the pitch."""
    spreads = []
    for nd in ((50, 200) if kind != "cone" else (48, 64)):
        g = _geoms_for_scale(kind, nd)
        y = np.ones(g.m)
        xb, xa = P.back_pixel(g, y), P.back_adjoint(g, y)
        sl = tuple(slice(s // 4, 3 * s // 4) for s in g.image_shape)
        ratio = xb[sl] / xa[sl]
        assert abs(ratio.mean() - 1.0) < 2e-3
        spreads.append(ratio.std())
    if kind != "cone":
        assert spreads[1] < spreads[0]


@pytest.mark.parametrize("kind", ["parallel", "fan", "cone"])
def test_backprojector_geometry_agrees_with_forward_rays(kind):
    """For a smooth off-centre blob's sinogram, B y and A^T y agree to a few per cent: B's
    detector coordinate (the magnification formula) lands where A's rays (built from source
    and bin positions) pass.  A mirrored or shifted coordinate would differ at O(1)."""
    g = _geoms_for_scale(kind, 200 if kind != "cone" else 48)
    cs = [np.arange(s) - (s - 1) / 2 for s in g.image_shape]
    grids = np.meshgrid(*cs, indexing="ij")
    off = [3.0, -5.0, 2.0][: len(grids)]
    r2 = sum((G - o) ** 2 for G, o in zip(grids, off))
    x = np.exp(-r2 / (2 * 3.0 ** 2))
    y = P.forward(g, x)
    xb, xa = P.back_pixel(g, y), P.back_adjoint(g, y)
    sl = tuple(slice(s // 4, 3 * s // 4) for s in g.image_shape)
    rel = np.linalg.norm(xb[sl] - xa[sl]) / np.linalg.norm(xa[sl])
    assert rel < 0.02
    assert np.linalg.norm(xb - xa) > 0      # unmatched: B is not A^T
