"""Brute-force pins of the oracle's 2D projectors: the explicit matrices A (Joseph) and B
(pixel-driven), built entry by entry in NumPy from their definitions, against the oracle
applied to every unit vector.

The builders here are written independently of the oracle's loops: a ray is the implicit line
through its two defining points (not a point and a parametric unit direction), linear
interpolation is the tent function tri(t) = max(0, 1 - |t|) on the whole pixel column (not a
floor and two taps with bounds tests), and the backprojector weight is the closed form of the
definition, h^2 (SDD^2 + u^2) / (L pitch SDD), with L = |p - S| and u the detector coordinate
of the ray through the pixel centre (Sec. 2: B is the pixel-driven interpolation, an unmatched
partner of A).  Angles avoid exact 45-degree ties, where the driving-axis choice depends on the
last bit of sin and cos.
"""
import math

import numpy as np
import pytest

import synth
from oracle import proj as OP


def tri(t):
    return np.maximum(0.0, 1.0 - np.abs(t))


def centres(n, h):
    return (np.arange(n) - (n - 1) / 2.0) * h


def explicit_A(g):
    """Joseph: every driving line sampled, weight h / |cos(angle to the driving axis)|."""
    X, Y = centres(g.nx, g.h), centres(g.ny, g.h)
    rows = np.arange(g.ny)[:, None]
    cols = np.arange(g.nx)[None, :]
    A = np.zeros((g.m, g.n))
    nd = g.n_det_u
    for v, th in enumerate(g.angles):
        c, s = math.cos(th), math.sin(th)
        for j in range(nd):
            u = (j - (nd - 1) / 2.0) * g.pitch_u
            if g.kind == synth.PARALLEL2D:
                # the line X c + Y s = u through the point u (c, s), direction (-s, c)
                P0 = np.array([u * c, u * s])
                P1 = P0 + np.array([-s, c])
            else:
                P0 = g.sid * np.array([c, s])                          # source
                P1 = -(g.sdd - g.sid) * np.array([c, s]) + u * np.array([-s, c])   # bin centre
            D = P1 - P0
            nrm = math.hypot(D[0], D[1])
            W = np.zeros((g.ny, g.nx))
            if abs(D[0]) >= abs(D[1]):
                # driving along x: at column centre X_c the line has height Y(X_c)
                Yc = P0[1] + (X - P0[0]) * (D[1] / D[0])
                rstar = Yc / g.h + (g.ny - 1) / 2.0
                W += tri(rows - rstar[None, :]) * (g.h * nrm / abs(D[0]))
            else:
                Xr = P0[0] + (Y - P0[1]) * (D[0] / D[1])
                cstar = Xr / g.h + (g.nx - 1) / 2.0
                W += tri(cols - cstar[:, None]) * (g.h * nrm / abs(D[1]))
            A[v * nd + j] = W.reshape(-1)
    return A


def explicit_B(g):
    """Pixel-driven: each pixel centre projected onto the detector, tent weights on the bins."""
    Xg, Yg = np.meshgrid(centres(g.nx, g.h), centres(g.ny, g.h))
    Xg, Yg = Xg.reshape(-1), Yg.reshape(-1)
    nd = g.n_det_u
    uj = (np.arange(nd) - (nd - 1) / 2.0) * g.pitch_u
    B = np.zeros((g.n, g.m))
    for v, th in enumerate(g.angles):
        c, s = math.cos(th), math.sin(th)
        along = Xg * c + Yg * s                     # p . (cos, sin)
        across = -Xg * s + Yg * c                   # p . e_u
        if g.kind == synth.PARALLEL2D:
            up = along
            w = np.full(g.n, g.h * g.h / g.pitch_u)
        else:
            depth = g.sid - along                   # distance from the source along the axis
            up = g.sdd * across / depth
            L = np.hypot(Xg - g.sid * c, Yg - g.sid * s)
            w = g.h * g.h * (g.sdd ** 2 + up ** 2) / (L * g.pitch_u * g.sdd)
        B[:, v * nd:(v + 1) * nd] = w[:, None] * tri((up[:, None] - uj[None, :]) / g.pitch_u)
    return B


def oracle_matrix(apply, n_in):
    cols = []
    for i in range(n_in):
        e = np.zeros(n_in)
        e[i] = 1.0
        cols.append(np.asarray(apply(e)).reshape(-1))
    return np.stack(cols, axis=1)


ANGLES = np.array([0.0, 0.3, 1.1, 1.9, 2.6, 3.4, 4.4, 5.5])

GEOMS = {
    "parallel_9x7": synth.parallel2d(9, 6, 15, pitch=0.9, ny=7, h=1.0, angles=ANGLES[:6]),
    "parallel_h_0.7": synth.parallel2d(6, 5, 11, pitch=0.55, ny=8, h=0.7, angles=ANGLES[1:6]),
    "fan_8x10": synth.fanflat2d(8, 8, 13, 30.0, 48.0, ny=10, h=1.0, angles=ANGLES),
    "fan_h_1.3": synth.fanflat2d(7, 5, 12, 25.0, 40.0, pitch=1.7, ny=6, h=1.3, angles=ANGLES[2:7]),
}


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_oracle_forward_equals_explicit_joseph_matrix(name):
    g = GEOMS[name]
    A = explicit_A(g)
    Ao = oracle_matrix(lambda e: OP.forward(g, e.reshape(g.image_shape)), g.n)
    assert np.max(np.abs(A)) > 0
    assert np.max(np.abs(Ao - A)) <= 1e-13 * np.max(np.abs(A))


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_oracle_backprojector_equals_explicit_pixel_matrix(name):
    g = GEOMS[name]
    B = explicit_B(g)
    Bo = oracle_matrix(lambda e: OP.back_pixel(g, e), g.m)
    assert np.max(np.abs(B)) > 0
    assert np.max(np.abs(Bo - B)) <= 1e-13 * np.max(np.abs(B))


@pytest.mark.parametrize("name", ["parallel_9x7", "fan_8x10"])
def test_explicit_matrices_are_unmatched_but_of_one_scale(name):
    """B is not A^T, but it has A^T's scale (the reading of the backprojector weights)."""
    g = GEOMS[name]
    A, B = explicit_A(g), explicit_B(g)
    diff = np.linalg.norm(B - A.T) / np.linalg.norm(A)
    assert 1e-3 < diff < 0.5
    assert 0.7 < np.linalg.norm(B) / np.linalg.norm(A) < 1.3


# ----------------------------------------------------------------------------- cone beam
def explicit_A3(g):
    """Cone Joseph: every plane across the driving axis (the largest |D| component, ties to x
    then y) sampled, bilinear tent weights in the plane, weight h |D| / |D_drive|."""
    n = (g.nx, g.ny, g.nz)
    A = np.zeros((g.m, g.n))
    nu, nv = g.n_det_u, g.n_det_v
    for view, th in enumerate(g.angles):
        c, s = math.cos(th), math.sin(th)
        S = np.array([g.sid * c, g.sid * s, 0.0])
        for iv in range(nv):
            vv = (iv - (nv - 1) / 2.0) * g.pitch_v
            for iu in range(nu):
                u = (iu - (nu - 1) / 2.0) * g.pitch_u
                P = np.array([-(g.sdd - g.sid) * c - u * s, -(g.sdd - g.sid) * s + u * c, vv])
                D = P - S
                a = 0
                if abs(D[1]) > abs(D[a]):
                    a = 1
                if abs(D[2]) > abs(D[a]):
                    a = 2
                rest = [ax for ax in range(3) if ax != a]
                V = np.zeros(n)                          # [x][y][z]
                for i in range(n[a]):
                    Ai = (i - (n[a] - 1) / 2.0) * g.h
                    pt = S + (Ai - S[a]) / D[a] * D
                    w = {ax: tri(np.arange(n[ax]) - (pt[ax] / g.h + (n[ax] - 1) / 2.0))
                         for ax in rest}
                    sl = [slice(None)] * 3
                    sl[a] = i
                    V[tuple(sl)] += np.outer(w[rest[0]], w[rest[1]])
                V *= g.h * np.linalg.norm(D) / abs(D[a])
                A[(view * nv + iv) * nu + iu] = np.transpose(V, (2, 1, 0)).reshape(-1)
    return A


def explicit_B3(g):
    """Voxel-driven: each voxel centre projected onto the flat detector, bilinear tent weights,
    weight h^3 (SDD^2 + u^2 + v^2)^{3/2} / (L^2 pitch_u pitch_v SDD)."""
    Z, Y, X = np.meshgrid(centres(g.nz, g.h), centres(g.ny, g.h), centres(g.nx, g.h),
                          indexing="ij")
    X, Y, Z = X.reshape(-1), Y.reshape(-1), Z.reshape(-1)
    nu, nv = g.n_det_u, g.n_det_v
    uj = (np.arange(nu) - (nu - 1) / 2.0) * g.pitch_u
    vi = (np.arange(nv) - (nv - 1) / 2.0) * g.pitch_v
    B = np.zeros((g.n, g.m))
    for view, th in enumerate(g.angles):
        c, s = math.cos(th), math.sin(th)
        depth = g.sid - (X * c + Y * s)
        up = g.sdd * (-X * s + Y * c) / depth
        vp = g.sdd * Z / depth
        L2 = (X - g.sid * c) ** 2 + (Y - g.sid * s) ** 2 + Z ** 2
        w = g.h ** 3 * (g.sdd ** 2 + up ** 2 + vp ** 2) ** 1.5 / (L2 * g.pitch_u * g.pitch_v * g.sdd)
        tu = tri((up[:, None] - uj[None, :]) / g.pitch_u)            # n x nu
        tv = tri((vp[:, None] - vi[None, :]) / g.pitch_v)            # n x nv
        blk = w[:, None, None] * tv[:, :, None] * tu[:, None, :]      # n x nv x nu
        B[:, view * nv * nu:(view + 1) * nv * nu] = blk.reshape(g.n, nv * nu)
    return B


GEOMS3 = {
    "cone_4": synth.cone3d(4, 3, 5, 4, 9.0, 15.0, angles=np.array([0.2, 1.3, 3.9])),
    # steep detector rows: |v| above the in-plane distance, so some rays drive along z
    "cone_4_steep": synth.cone3d(4, 3, 5, 4, 6.0, 10.0, pitch_v=8.0,
                                 angles=np.array([0.4, 2.2, 5.1])),
}


@pytest.mark.parametrize("name", sorted(GEOMS3))
def test_oracle_cone_forward_equals_explicit_matrix(name):
    g = GEOMS3[name]
    A = explicit_A3(g)
    Ao = oracle_matrix(lambda e: OP.forward(g, e.reshape(g.image_shape)), g.n)
    assert np.max(np.abs(A)) > 0
    assert np.max(np.abs(Ao - A)) <= 1e-13 * np.max(np.abs(A))


def test_steep_case_drives_along_z():
    """The steep geometry has rays of each kind: driven along z and in the plane."""
    g = GEOMS3["cone_4_steep"]
    kinds = set()
    for th in g.angles:
        c, s = math.cos(th), math.sin(th)
        for iv in range(g.n_det_v):
            for iu in range(g.n_det_u):
                u = (iu - (g.n_det_u - 1) / 2.0) * g.pitch_u
                v = (iv - (g.n_det_v - 1) / 2.0) * g.pitch_v
                D = np.array([-g.sdd * c - u * s, -g.sdd * s + u * c, v])
                kinds.add(abs(D[2]) > max(abs(D[0]), abs(D[1])))
    assert kinds == {True, False}


@pytest.mark.parametrize("name", sorted(GEOMS3))
def test_oracle_voxel_backprojector_equals_explicit_matrix(name):
    g = GEOMS3[name]
    B = explicit_B3(g)
    Bo = oracle_matrix(lambda e: OP.back_pixel(g, e), g.m)
    assert np.max(np.abs(B)) > 0
    assert np.max(np.abs(Bo - B)) <= 1e-13 * np.max(np.abs(B))


@pytest.mark.parametrize("name", ["parallel_9x7", "fan_h_1.3", "cone_4_steep"])
def test_oracle_matched_adjoint_equals_explicit_transpose(name):
    """The matched backprojector A^T (Sec. 2, LSQR / LSMR comparators) is the transpose of
    the explicit Joseph matrix."""
    g = GEOMS.get(name) or GEOMS3[name]
    A = explicit_A3(g) if g.kind == synth.CONE3D else explicit_A(g)
    ATo = oracle_matrix(lambda e: OP.back_adjoint(g, e), g.m)
    assert np.max(np.abs(ATo - A.T)) <= 1e-13 * np.max(np.abs(A))
