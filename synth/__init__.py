"""Seeded synthetic inputs for the CT reconstruction problems.

This module is shared by the FP64 oracle tests, the GPU tests and the benchmark.  It holds
no arithmetic of the reconstruction method itself: it only draws phantoms (ellipses and
ellipsoids on the pixel grid), describes the scan geometry (angles, detector size and
pitch, source distances) and draws Gaussian vectors from a seeded PCG64 stream.

Conventions (the paper leaves them open, Sec. 4 only says the data come from a GPU
projector toolbox):

* pixel size h; pixel (r, c) of an ny x nx image has its centre at
  X = (c - (nx-1)/2) h,  Y = (r - (ny-1)/2) h  (row-major storage, index r*nx + c);
* parallel beam: view angles theta_i = i * range / n_views, range = pi, endpoint excluded;
* fan-flat / cone: theta_i = i * 2 pi / n_views, source at SID (cos, sin);
* detector bin j has its centre at (j - (n_det-1)/2) * pitch.

Detector sizes that a workload leaves open follow one recipe: parallel pitch = h and
n_det = ceil(N sqrt 2) + 4 (95 bins at N = 64); fan pitch makes the fan cover the
circle of radius N h sqrt(2)/2 around the isocentre.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

PARALLEL2D = "parallel2d"
FANFLAT2D = "fanflat2d"
CONE3D = "cone3d"


@dataclass(frozen=True)
class Geometry:
    """Scan geometry; every length is in the same unit as the pixel size ``h``."""

    kind: str
    nx: int
    ny: int
    nz: int = 1
    h: float = 1.0
    angles: np.ndarray = field(default_factory=lambda: np.zeros(0))
    n_det_u: int = 1
    n_det_v: int = 1
    pitch_u: float = 1.0
    pitch_v: float = 1.0
    sid: float = 0.0
    sdd: float = 0.0

    @property
    def n_views(self) -> int:
        return int(len(self.angles))

    @property
    def n(self) -> int:
        """Number of unknowns (pixels or voxels)."""
        return self.nx * self.ny * self.nz

    @property
    def m(self) -> int:
        """Number of measurements (rays)."""
        return self.n_views * self.n_det_u * self.n_det_v

    @property
    def image_shape(self):
        return (self.ny, self.nx) if self.kind != CONE3D else (self.nz, self.ny, self.nx)

    @property
    def sino_shape(self):
        if self.kind == CONE3D:
            return (self.n_views, self.n_det_v, self.n_det_u)
        return (self.n_views, self.n_det_u)

    def with_angles(self, angles) -> "Geometry":
        return replace(self, angles=np.asarray(angles, dtype=np.float64))


def uniform_angles(n_views: int, angle_range: float) -> np.ndarray:
    """theta_i = i * range / n_views, endpoint excluded."""
    return np.arange(n_views, dtype=np.float64) * (angle_range / n_views)


def parallel_n_det(N: int) -> int:
    return int(math.ceil(N * math.sqrt(2.0))) + 4


def parallel2d(N: int, n_views: int, n_det: int | None = None, pitch: float = 1.0,
               angle_range: float = math.pi, ny: int | None = None, h: float = 1.0,
               angles=None) -> Geometry:
    nx = N
    ny = N if ny is None else ny
    n_det = parallel_n_det(max(nx, ny)) if n_det is None else n_det
    ang = uniform_angles(n_views, angle_range) if angles is None else np.asarray(angles, np.float64)
    return Geometry(PARALLEL2D, nx, ny, 1, h, ang, n_det, 1, pitch, 1.0, 0.0, 0.0)


def fan_pitch(N: int, n_det: int, sid: float, sdd: float, h: float = 1.0) -> float:
    """Pitch so that n_det bins cover the fan through the circle of radius N h sqrt(2)/2."""
    R = N * h * math.sqrt(2.0) / 2.0
    return 2.0 * sdd * math.tan(math.asin(R / sid)) / n_det


def fanflat2d(N: int, n_views: int, n_det: int, sid: float, sdd: float,
              pitch: float | None = None, angle_range: float = 2.0 * math.pi,
              ny: int | None = None, h: float = 1.0, angles=None) -> Geometry:
    nx = N
    ny = N if ny is None else ny
    pitch = fan_pitch(max(nx, ny), n_det, sid, sdd, h) if pitch is None else pitch
    ang = uniform_angles(n_views, angle_range) if angles is None else np.asarray(angles, np.float64)
    return Geometry(FANFLAT2D, nx, ny, 1, h, ang, n_det, 1, pitch, 1.0, float(sid), float(sdd))


def cone3d(N: int, n_views: int, n_det_u: int, n_det_v: int, sid: float, sdd: float,
           pitch_u: float | None = None, pitch_v: float | None = None, h: float = 1.0,
           angle_range: float = 2.0 * math.pi, angles=None) -> Geometry:
    """Circular cone-beam scan of an N^3 volume with a flat detector.

    pitch_u covers the fan through the circumscribed circle of a slice; pitch_v covers the
    volume's half height N h / 2 at the largest magnification SDD / (SID - R)."""
    R = N * h * math.sqrt(2.0) / 2.0
    pu = fan_pitch(N, n_det_u, sid, sdd, h) if pitch_u is None else pitch_u
    pv = (2.0 * (N * h / 2.0) * sdd / (sid - R) / n_det_v) if pitch_v is None else pitch_v
    ang = uniform_angles(n_views, angle_range) if angles is None else np.asarray(angles, np.float64)
    return Geometry(CONE3D, N, N, N, h, ang, n_det_u, n_det_v, pu, pv, float(sid), float(sdd))


# ----------------------------------------------------------------------------- phantoms

def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def ellipse_params(N: int, n_ellipses: int, seed: int) -> np.ndarray:
    """Rows (cx, cy, a, b, phi, value): centres uniform in the disc of radius 0.7 N/2,
    semi-axes U[0.05, 0.35] N/2, orientation U[0, pi), value U[0, 1]."""
    g = _rng(seed)
    half = N / 2.0
    rad = 0.7 * half * np.sqrt(g.random(n_ellipses))
    ang = 2.0 * np.pi * g.random(n_ellipses)
    a = half * (0.05 + 0.30 * g.random(n_ellipses))
    b = half * (0.05 + 0.30 * g.random(n_ellipses))
    phi = np.pi * g.random(n_ellipses)
    val = g.random(n_ellipses)
    return np.stack([rad * np.cos(ang), rad * np.sin(ang), a, b, phi, val], axis=1)


def pixel_centres(nx: int, ny: int, h: float = 1.0):
    X = (np.arange(nx, dtype=np.float64) - (nx - 1) / 2.0) * h
    Y = (np.arange(ny, dtype=np.float64) - (ny - 1) / 2.0) * h
    return np.meshgrid(X, Y, indexing="xy")


def ellipse_phantom(N: int, n_ellipses: int = 10, seed: int = 0, ny: int | None = None,
                    h: float = 1.0) -> np.ndarray:
    """FP64 (ny, nx) image: sum of ellipse indicators sampled at pixel centres."""
    nx = N
    ny = N if ny is None else ny
    XX, YY = pixel_centres(nx, ny, h)
    img = np.zeros((ny, nx), dtype=np.float64)
    scale = min(nx, ny) * h
    for cx, cy, a, b, phi, v in ellipse_params(1, n_ellipses, seed):
        cx, cy, a, b = cx * scale, cy * scale, a * scale, b * scale
        dx, dy = XX - cx, YY - cy
        cp, sp = math.cos(phi), math.sin(phi)
        u = dx * cp + dy * sp
        w = -dx * sp + dy * cp
        img[(u / a) ** 2 + (w / b) ** 2 <= 1.0] += v
    return img


def ellipsoid_phantom(N: int, n_ellipsoids: int = 10, seed: int = 0, h: float = 1.0) -> np.ndarray:
    """FP64 (N, N, N) volume [z][y][x]: sum of ellipsoid indicators at voxel centres; centres
    uniform in the ball of radius 0.7 N/2, semi-axes U[0.05, 0.35] N/2, Euler angles U[0, pi).

    Each ellipsoid is evaluated only on the voxels of its bounding box, with the same
    elementwise arithmetic for every voxel (the result does not depend on the box)."""
    g = _rng(seed)
    half = N * h / 2.0
    c = (np.arange(N, dtype=np.float64) - (N - 1) / 2.0) * h
    vol = np.zeros((N, N, N), dtype=np.float64)
    for _ in range(n_ellipsoids):
        d = g.standard_normal(3)
        d /= np.linalg.norm(d)
        centre = d * 0.7 * half * g.random() ** (1.0 / 3.0)
        axes = half * (0.05 + 0.30 * g.random(3))
        al, be, ga = np.pi * g.random(3)
        val = g.random()
        ca, sa, cb, sb, cg, sg = (math.cos(al), math.sin(al), math.cos(be), math.sin(be),
                                  math.cos(ga), math.sin(ga))
        Rz1 = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1.0]])
        Rx = np.array([[1.0, 0, 0], [0, cb, -sb], [0, sb, cb]])
        Rz2 = np.array([[cg, -sg, 0], [sg, cg, 0], [0, 0, 1.0]])
        R = Rz1 @ Rx @ Rz2
        # half-extent of the ellipsoid along each axis: |R_i| . axes (row norms of R diag(axes))
        ext = np.sqrt(((R * axes[None, :]) ** 2).sum(axis=1)) + 2.0 * h
        lo = np.clip(np.floor((centre - ext) / h + (N - 1) / 2.0).astype(int), 0, N)
        hi = np.clip(np.ceil((centre + ext) / h + (N - 1) / 2.0).astype(int) + 1, 0, N)
        if np.any(hi <= lo):
            continue
        X = (c[lo[0]:hi[0]] - centre[0])[None, None, :]
        Y = (c[lo[1]:hi[1]] - centre[1])[None, :, None]
        Z = (c[lo[2]:hi[2]] - centre[2])[:, None, None]
        q = np.zeros((hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0]))
        for k in range(3):          # coordinates in the ellipsoid frame: (P R)_k / axes_k
            Lk = X * R[0, k] + Y * R[1, k] + Z * R[2, k]
            q += (Lk / axes[k]) ** 2
        vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]][q <= 1.0] += val
    return vol


def disc_phantom(nx: int, ny: int, radius: float, centre=(0.0, 0.0), h: float = 1.0) -> np.ndarray:
    """Indicator of a disc sampled at pixel centres (value 1 inside)."""
    XX, YY = pixel_centres(nx, ny, h)
    return (((XX - centre[0]) ** 2 + (YY - centre[1]) ** 2) <= radius ** 2).astype(np.float64)


# ----------------------------------------------------------------------------- noise

def standard_normal(shape, seed: int) -> np.ndarray:
    return _rng(seed).standard_normal(shape)


def add_noise(b_true: np.ndarray, eta: float, seed: int):
    """Noise level eta (a fraction, 0.01 = 1 %): e = eta ||b_true|| g / ||g||, g ~ N(0, I).

    Returns (b, e) with b = b_true + e."""
    g = standard_normal(b_true.shape, seed)
    e = eta * np.linalg.norm(b_true) * g / np.linalg.norm(g)
    return b_true + e, e


# ----------------------------------------------------------------------------- workloads

def small_parallel_case():
    """64 x 64 image of 10 ellipses, 90 parallel views over [0, 180 deg), 95 bins, 1 % noise;
    hybrid AB-GMRES, 30 iterations, GCV."""
    geom = parallel2d(64, 90, 95)
    return dict(geom=geom, phantom_seed=0, eta=0.01, noise_seed=1000, method="ab",
                iters=30, rule="gcv")


def fan512_case():
    """512 x 512 ellipse phantom, fan-flat, 720 views over 360 deg, 768 bins, SID 1000,
    SDD 1500, 2 % noise; hybrid AB- and BA-GMRES 100 iterations each, discrepancy principle."""
    geom = fanflat2d(512, 720, 768, 1000.0, 1500.0)
    return dict(geom=geom, phantom_seed=0, eta=0.02, noise_seed=2000, iters=100, rule="dp",
                tau=1.01)


def batched_slices(n_slices: int = 256, seed: int = 7):
    """Uneven batch: N ~ U{256, 512, 768, 1024}, parallel or fan with probability 1/2,
    views ~ U{180..1440}; fan SID/SDD = (1000, 1500) * N / 512 and 1.5 N bins."""
    g = _rng(seed)
    out = []
    for s in range(n_slices):
        N = int(256 * g.integers(1, 5))
        views = int(g.integers(180, 1441))
        if g.random() < 0.5:
            geom = parallel2d(N, views)
        else:
            geom = fanflat2d(N, views, int(1.5 * N), 1000.0 * N / 512, 1500.0 * N / 512)
        out.append(dict(geom=geom, phantom_seed=10_000 + s, noise_seed=20_000 + s, eta=0.01))
    return out


def cone512_case(N: int = 512):
    """N^3 ellipsoid phantom, cone beam, 400 views over 360 deg, 768 x 768 detector (scaled
    with N / 512 for reduced copies), SID 1000, SDD 1500, 1 % noise; hybrid AB-GMRES 100
    iterations, GCV."""
    nd = max(8, int(round(768 * N / 512)))
    geom = cone3d(N, 400 if N >= 512 else max(16, int(400 * N / 512)), nd, nd, 1000.0 * N / 512,
                  1500.0 * N / 512)
    return dict(geom=geom, phantom_seed=0, eta=0.01, noise_seed=3000, iters=100, rule="gcv")
