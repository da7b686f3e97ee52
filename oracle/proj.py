"""ctypes front end of the FP64 C oracle projectors (``projectors.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the benchmark's CPU
baseline, never by the product library.  The shared object is compiled with gcc on first
use (or by ``build_oracle()``), next to this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "projectors.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

KIND = {"parallel2d": 0, "fanflat2d": 1, "cone3d": 2}


def build_oracle(force: bool = False) -> str:
    """Compile projectors.c with gcc (-O2, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", _SRC,
               "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _OGeom(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("h", ctypes.c_double), ("n_views", ctypes.c_int),
                ("angles", ctypes.POINTER(ctypes.c_double)), ("n_det_u", ctypes.c_int),
                ("n_det_v", ctypes.c_int), ("pitch_u", ctypes.c_double),
                ("pitch_v", ctypes.c_double), ("sid", ctypes.c_double), ("sdd", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_oracle())
            dp = ctypes.POINTER(ctypes.c_double)
            gp = ctypes.POINTER(_OGeom)
            lib.og_forward.argtypes = [gp, dp, dp]
            lib.og_back_pixel.argtypes = [gp, dp, dp]
            lib.og_back_adjoint.argtypes = [gp, dp, dp]
            lib.og_forward_ray.argtypes = [gp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.og_forward_ray.restype = ctypes.c_double
            lib.og_back_pixel_one.argtypes = [gp, dp, ctypes.c_long, ctypes.c_long, ctypes.c_long]
            lib.og_back_pixel_one.restype = ctypes.c_double
            lib.og_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().og_num_threads())


class _Bound:
    """Keeps the angle array alive while the C struct points at it."""

    def __init__(self, geom):
        self.angles = np.ascontiguousarray(geom.angles, dtype=np.float64)
        self.s = _OGeom(KIND[geom.kind], geom.nx, geom.ny, geom.nz, float(geom.h),
                        len(self.angles),
                        self.angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        geom.n_det_u, geom.n_det_v, float(geom.pitch_u), float(geom.pitch_v),
                        float(geom.sid), float(geom.sdd))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def forward(geom, x) -> np.ndarray:
    """y = A x (Joseph), FP64, returned with the geometry's sinogram shape."""
    lib = _load()
    g = _Bound(geom)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    assert x.size == geom.n
    y = np.zeros(geom.m, dtype=np.float64)
    lib.og_forward(ctypes.byref(g.s), _dptr(x), _dptr(y))
    return y.reshape(geom.sino_shape)


def back_pixel(geom, y) -> np.ndarray:
    """x = B y (pixel/voxel-driven, unmatched), FP64."""
    lib = _load()
    g = _Bound(geom)
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
    assert y.size == geom.m
    x = np.zeros(geom.n, dtype=np.float64)
    lib.og_back_pixel(ctypes.byref(g.s), _dptr(y), _dptr(x))
    return x.reshape(geom.image_shape)


def back_adjoint(geom, y) -> np.ndarray:
    """x = A^T y, the exact transpose of ``forward`` (matched backprojector), FP64."""
    lib = _load()
    g = _Bound(geom)
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
    assert y.size == geom.m
    x = np.zeros(geom.n, dtype=np.float64)
    lib.og_back_adjoint(ctypes.byref(g.s), _dptr(y), _dptr(x))
    return x.reshape(geom.image_shape)


def forward_ray(geom, x, view: int, iu: int, iv: int = 0) -> float:
    """One entry of A x."""
    lib = _load()
    g = _Bound(geom)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    return float(lib.og_forward_ray(ctypes.byref(g.s), _dptr(x), view, iu, iv))


def back_pixel_one(geom, y, k: int, r: int, c: int) -> float:
    """One entry of B y (pixel (r, c) of slice k)."""
    lib = _load()
    g = _Bound(geom)
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
    return float(lib.og_back_pixel_one(ctypes.byref(g.s), _dptr(y), k, r, c))


def operators(geom, matched: bool = False):
    """(A, B) as callables on flat FP64 vectors; matched=True gives B = A^T."""
    A = lambda v: forward(geom, v).reshape(-1)
    if matched:
        B = lambda v: back_adjoint(geom, v).reshape(-1)
    else:
        B = lambda v: back_pixel(geom, v).reshape(-1)
    return A, B
