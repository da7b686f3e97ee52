"""ctypes binding of libctabba.so: argument marshalling only.

Names follow the C ABI in ``include/ctabba.h``.  Device buffers are PyTorch CUDA tensors
(FP32 or FP64, contiguous); the work is enqueued on PyTorch's current CUDA stream.  Every
numerical step runs in the library's CUDA kernels: there is no CPU or PyTorch fallback, and
loading fails loudly when the shared library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libctabba.so")

CT_OK, CT_EINVAL, CT_ENOMEM, CT_ECUDA, CT_BREAKDOWN, CT_ETIMEOUT, CT_ENONFINITE = range(7)
STATUS_NAMES = {0: "CT_OK", 1: "CT_EINVAL", 2: "CT_ENOMEM", 3: "CT_ECUDA", 4: "CT_BREAKDOWN",
                5: "CT_ETIMEOUT", 6: "CT_ENONFINITE"}
KINDS = {"parallel2d": 0, "fanflat2d": 1, "cone3d": 2}
RULES = {"none": 0, "fixed": 1, "gcv": 2, "dp": 3, "learned": 4, "lcurve": 5}
CT_MLP_NIN, CT_MLP_NPARAMS = 80, 9569
BASIS = {"f32": 0, "bf16": 1, "f16": 2}
STOPS = {"none": 0, "dp": 1, "rns": 2, "ncp": 3}

# the entry points of include/ctabba.h
EXPORTS = ("ct_geom_create", "ct_geom_destroy", "ct_geom_dims", "ct_geom_work", "ct_forward_A", "ct_back_B",
           "ct_hybrid_opts_default", "ab_gmres_hybrid", "ba_gmres_hybrid", "ct_arnoldi_step", "ct_arnoldi_step_noalloc",
           "ct_projected_solve", "ct_status_string", "ct_last_error", "ct_profile_enable",
           "ct_profile_collect", "ct_launch_count", "ct_geom_autotune", "ct_batch_create",
           "ct_batch_solve", "ct_batch_launches", "ct_batch_destroy", "abba_solve", "ct_mlp_forward",
           "ct_mlp_grad", "ct_mlp_adam", "ct_mlp_train", "ct_lambda_samples",
           "ab_gmres_hybrid_restarted", "ba_gmres_hybrid_restarted", "ct_test_drop_tile_copy",
           "ct_probe")
PHASES = ("forward_A", "back_B", "layout", "arnoldi", "small_solve", "other")


class CtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GeomDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("pixel", ctypes.c_double), ("n_views", ctypes.c_int),
                ("angles", ctypes.POINTER(ctypes.c_double)), ("n_det_u", ctypes.c_int),
                ("n_det_v", ctypes.c_int), ("pitch_u", ctypes.c_double),
                ("pitch_v", ctypes.c_double), ("sid", ctypes.c_double), ("sdd", ctypes.c_double)]


class HybridOpts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("rule", ctypes.c_int),
                ("lambda_fixed", ctypes.c_double), ("noise_norm", ctypes.c_double),
                ("tau", ctypes.c_double), ("reorth", ctypes.c_int), ("basis", ctypes.c_int),
                ("lambda_hist", ctypes.POINTER(ctypes.c_double)),
                ("resid_hist", ctypes.POINTER(ctypes.c_double)),
                ("lambda_net_dev", ctypes.c_void_p), ("features_dev", ctypes.c_void_p),
                ("stop_rule", ctypes.c_int), ("stop_tol", ctypes.c_double),
                ("stop_every", ctypes.c_int), ("ncp_hist", ctypes.POINTER(ctypes.c_double))]


class PhaseTime(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("launches", ctypes.c_int64), ("groups", ctypes.c_int64)]


class LaunchShapes(ctypes.Structure):
    _fields_ = [("a_threads", ctypes.c_int), ("a_views", ctypes.c_int), ("a_slab", ctypes.c_int),
                ("b_rows", ctypes.c_int), ("b_views", ctypes.c_int), ("a_rays", ctypes.c_int),
                ("a_warp_views", ctypes.c_int), ("b_warp_rows", ctypes.c_int)]


class HybridInfo(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int), ("beta", ctypes.c_double),
                ("final_lambda", ctypes.c_double), ("final_resid", ctypes.c_double),
                ("status", ctypes.c_int), ("fast_path_steps", ctypes.c_int),
                ("lambda_fallback_steps", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libctabba.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libctabba.so not found at {path}; build it with "
                          "`python -m paper_2602_17892_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.ct_geom_create.argtypes = [ctypes.POINTER(GeomDesc), ctypes.POINTER(vp)]
    lib.ct_geom_destroy.argtypes = [vp]
    lib.ct_geom_destroy.restype = None
    lib.ct_geom_dims.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.ct_geom_work.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.ct_forward_A.argtypes = [vp, vp, vp, vp]
    lib.ct_back_B.argtypes = [vp, vp, vp, vp]
    lib.ct_hybrid_opts_default.argtypes = [ctypes.POINTER(HybridOpts)]
    lib.ct_hybrid_opts_default.restype = None
    for fn in (lib.ab_gmres_hybrid, lib.ba_gmres_hybrid):
        fn.argtypes = [vp, vp, vp, vp, ctypes.POINTER(HybridOpts), ctypes.POINTER(HybridInfo), vp]
    for fn in (lib.ab_gmres_hybrid_restarted, lib.ba_gmres_hybrid_restarted):
        fn.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(HybridOpts),
                       ctypes.POINTER(HybridInfo), vp]
    lib.ct_arnoldi_step.argtypes = [vp, i64, i64, ctypes.c_int, vp, vp, vp]
    lib.ct_arnoldi_step_noalloc.argtypes = [vp, i64, i64, ctypes.c_int, vp, vp, vp]
    lib.ct_arnoldi_step_noalloc.restype = ctypes.c_int
    lib.ct_projected_solve.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double, vp, vp,
                                       vp, vp]
    lib.ct_profile_enable.argtypes = [ctypes.c_int]
    lib.ct_profile_collect.argtypes = [ctypes.POINTER(PhaseTime)]
    lib.ct_launch_count.restype = ctypes.c_int64
    lib.ct_launch_count.argtypes = []
    lib.ct_geom_autotune.argtypes = [vp, vp, ctypes.POINTER(LaunchShapes)]
    lib.ct_geom_set_launch_shapes.argtypes = [vp, ctypes.POINTER(LaunchShapes)]
    lib.ct_back_AT.argtypes = [vp, vp, vp, vp]
    lib.ct_geom_set_backprojector.argtypes = [vp, ctypes.c_int]
    lib.ct_geom_get_launch_shapes.argtypes = [vp, ctypes.POINTER(LaunchShapes)]
    lib.ct_test_drop_tile_copy.argtypes = [ctypes.c_int, i64]
    lib.ct_probe.argtypes = [ctypes.c_int, i64, vp, i64, ctypes.POINTER(i64), vp]
    lib.ct_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(HybridOpts), ctypes.c_int, ctypes.POINTER(vp)]
    lib.ct_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(HybridInfo), vp]
    lib.ct_batch_launches.argtypes = [vp]
    lib.ct_batch_launches.restype = ctypes.c_int64
    lib.ct_batch_destroy.argtypes = [vp]
    lib.ct_batch_destroy.restype = None
    lib.abba_solve.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(HybridOpts),
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(HybridInfo), vp]
    lib.ct_mlp_forward.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int, vp]
    lib.ct_mlp_grad.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp, ctypes.c_int, vp]
    lib.ct_mlp_adam.argtypes = [vp, vp, vp, vp, ctypes.c_float, ctypes.c_int, vp]
    lib.ct_mlp_train.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_float, ctypes.POINTER(ctypes.c_int), vp, ctypes.c_int, vp]
    lib.ct_lambda_samples.argtypes = [vp, vp, vp, ctypes.POINTER(HybridOpts), vp, vp, vp,
                                      ctypes.POINTER(HybridInfo), vp]
    lib.ct_status_string.argtypes = [ctypes.c_int]
    lib.ct_status_string.restype = ctypes.c_char_p
    lib.ct_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        getattr(lib, name).restype = getattr(lib, name).restype or ctypes.c_int
    _lib = lib
    return lib


def _check(st):
    if st != CT_OK:
        raise CtError(st, load().ct_last_error().decode())
    return st


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype_name="float32"):
    if t is None:
        return None
    import torch
    want = getattr(torch, dtype_name)
    if not (t.is_cuda and t.dtype == want and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA {dtype_name} tensor")
    return ctypes.c_void_p(t.data_ptr())


class Geom:
    """Owns a ct_geom handle (ct_geom_create / ct_geom_destroy)."""

    def __init__(self, kind, nx, ny, angles, n_det_u, pitch_u, pixel=1.0, nz=1, n_det_v=1,
                 pitch_v=1.0, sid=0.0, sdd=0.0):
        lib = load()
        self._angles = np.ascontiguousarray(angles, dtype=np.float64)
        d = GeomDesc(KINDS[kind] if isinstance(kind, str) else int(kind), int(nx), int(ny),
                     int(nz), float(pixel), len(self._angles),
                     self._angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(n_det_u),
                     int(n_det_v), float(pitch_u), float(pitch_v), float(sid), float(sdd))
        h = ctypes.c_void_p()
        _check(lib.ct_geom_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        n, m = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.ct_geom_dims(h, ctypes.byref(n), ctypes.byref(m)))
        self.n, self.m = n.value, m.value
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.ct_geom_work(h, ctypes.byref(a), ctypes.byref(b)))
        self.a_samples, self.b_samples = a.value, b.value

    @classmethod
    def from_geometry(cls, g):
        """From any object with the fields of the seeded input module's Geometry."""
        return cls(g.kind, g.nx, g.ny, g.angles, g.n_det_u, g.pitch_u, pixel=g.h, nz=g.nz,
                   n_det_v=g.n_det_v, pitch_v=g.pitch_v, sid=g.sid, sdd=g.sdd)

    def close(self):
        if getattr(self, "handle", None):
            load().ct_geom_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ct_forward_A(g: Geom, x, y, stream=None):
    _check(load().ct_forward_A(g.handle, _ptr(x), _ptr(y), _stream(stream)))


def ct_back_B(g: Geom, y, x, stream=None):
    _check(load().ct_back_B(g.handle, _ptr(y), _ptr(x), _stream(stream)))


def _opts(max_iters, rule, lambda_fixed, noise_norm, tau, reorth, basis, history,
          lambda_net=None, features=None, stop=None, stop_tol=1e-3, stop_every=5):
    o = HybridOpts()
    load().ct_hybrid_opts_default(ctypes.byref(o))
    o.max_iters = int(max_iters)
    o.rule = RULES[rule] if isinstance(rule, str) else int(rule)
    o.lambda_fixed = float(lambda_fixed)
    o.noise_norm = float(noise_norm)
    o.tau = float(tau)
    o.reorth = int(reorth)
    o.basis = BASIS[basis] if isinstance(basis, str) else int(basis)
    o.stop_rule = STOPS[stop] if isinstance(stop, str) else int(stop or 0)
    o.stop_tol = float(stop_tol)
    o.stop_every = int(stop_every)
    o.lambda_net_dev = _ptr(lambda_net).value if lambda_net is not None else None
    o.features_dev = _ptr(features).value if features is not None else None
    lam = res = ncp = None
    if history:
        lam = np.full(int(max_iters), np.nan)
        res = np.full(int(max_iters), np.nan)
        o.lambda_hist = lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        o.resid_hist = res.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if o.stop_rule == STOPS["ncp"]:
            ncp = np.full(int(max_iters), np.nan)
            o.ncp_hist = ncp.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return o, lam, res, ncp


def _solve(fn, g, b, x, x0, max_iters, rule, lambda_fixed, noise_norm, tau, reorth, basis,
           history, stream, lambda_net=None, features=None, stop=None, stop_tol=1e-3,
           stop_every=5):
    o, lam, res, ncp = _opts(max_iters, rule, lambda_fixed, noise_norm, tau, reorth, basis,
                             history, lambda_net, features, stop, stop_tol, stop_every)
    info = HybridInfo()
    st = fn(g.handle, _ptr(b), _ptr(x0), _ptr(x), ctypes.byref(o), ctypes.byref(info),
            _stream(stream))
    _check(st)
    out = _info_dict(info)
    if history:
        out["lambdas"], out["resid"] = lam, res
        if ncp is not None:
            out["ncp"] = ncp
    return out


def ab_gmres_hybrid(g, b, x, u0=None, max_iters=30, rule="gcv", lambda_fixed=0.0,
                    noise_norm=0.0, tau=1.01, reorth=1, basis="f32", history=True, stream=None,
                    lambda_net=None, features=None, stop=None, stop_tol=1e-3, stop_every=5):
    """Hybrid AB-GMRES (Algorithm 1): x <- x0 + B W_K y_K with x0 = B u0."""
    return _solve(load().ab_gmres_hybrid, g, b, x, u0, max_iters, rule, lambda_fixed,
                  noise_norm, tau, reorth, basis, history, stream, lambda_net, features, stop,
                  stop_tol, stop_every)


def ba_gmres_hybrid(g, b, x, x0=None, max_iters=30, rule="gcv", lambda_fixed=0.0,
                    noise_norm=0.0, tau=1.01, reorth=1, basis="f32", history=True, stream=None,
                    lambda_net=None, features=None, stop=None, stop_tol=1e-3, stop_every=5):
    """Hybrid BA-GMRES (Algorithm 2): x <- x0 + W_K y_K."""
    return _solve(load().ba_gmres_hybrid, g, b, x, x0, max_iters, rule, lambda_fixed,
                  noise_norm, tau, reorth, basis, history, stream, lambda_net, features, stop,
                  stop_tol, stop_every)


def _solve_restarted(fn, g, b, x, cycles, max_iters, rule, lambda_fixed, noise_norm, tau,
                     reorth, basis, history, stream, lambda_net):
    o, _, _, _ = _opts(max_iters, rule, lambda_fixed, noise_norm, tau, reorth, basis, False,
                       lambda_net)
    lam = res = None
    if history:
        lam = np.full(int(cycles) * int(max_iters), np.nan)
        res = np.full(int(cycles) * int(max_iters), np.nan)
        o.lambda_hist = lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        o.resid_hist = res.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    info = HybridInfo()
    _check(fn(g.handle, _ptr(b), _ptr(x), int(cycles), ctypes.byref(o), ctypes.byref(info),
              _stream(stream)))
    out = _info_dict(info)
    if history:
        out["lambdas"], out["resid"] = lam, res
    return out


def ab_gmres_hybrid_restarted(g, b, x, cycles, max_iters=10, rule="gcv", lambda_fixed=0.0,
                              noise_norm=0.0, tau=1.01, reorth=1, basis="f32", history=True,
                              stream=None, lambda_net=None):
    """Restarted hybrid AB-GMRES (Sec. 3.3): `cycles` cycles of `max_iters` steps."""
    return _solve_restarted(load().ab_gmres_hybrid_restarted, g, b, x, cycles, max_iters, rule,
                            lambda_fixed, noise_norm, tau, reorth, basis, history, stream,
                            lambda_net)


def ba_gmres_hybrid_restarted(g, b, x, cycles, max_iters=10, rule="gcv", lambda_fixed=0.0,
                              noise_norm=0.0, tau=1.01, reorth=1, basis="f32", history=True,
                              stream=None, lambda_net=None):
    """Restarted hybrid BA-GMRES (Sec. 3.3): `cycles` cycles of `max_iters` steps."""
    return _solve_restarted(load().ba_gmres_hybrid_restarted, g, b, x, cycles, max_iters, rule,
                            lambda_fixed, noise_norm, tau, reorth, basis, history, stream,
                            lambda_net)


def ct_arnoldi_step(W, length, ld, k, q, h, stream=None):
    _check(load().ct_arnoldi_step(_ptr(W), int(length), int(ld), int(k), _ptr(q),
                                  _ptr(h, "float64"), _stream(stream)))


def ct_arnoldi_step_noalloc(W, length, ld, k, q, h, stream=None):
    """As ct_arnoldi_step, with its scratch in a static device array (no allocation)."""
    _check(load().ct_arnoldi_step_noalloc(_ptr(W), int(length), int(ld), int(k), _ptr(q),
                                          _ptr(h, "float64"), _stream(stream)))


def ct_projected_solve(H, ldh, k, beta, rule, lambda_fixed, dp_target, y, lam, resid,
                       stream=None):
    r = RULES[rule] if isinstance(rule, str) else int(rule)
    _check(load().ct_projected_solve(_ptr(H, "float64"), int(ldh), int(k), float(beta), r,
                                     float(lambda_fixed), float(dp_target), _ptr(y, "float64"),
                                     _ptr(lam, "float64"), _ptr(resid, "float64"),
                                     _stream(stream)))


def ct_profile_enable(on: bool = True):
    _check(load().ct_profile_enable(1 if on else 0))


def ct_profile_collect() -> dict:
    """{phase: (ms, launches, groups)} accumulated since the last collect (host-blocking)."""
    arr = (PhaseTime * len(PHASES))()
    _check(load().ct_profile_collect(arr))
    return {name: (arr[i].ms, arr[i].launches, arr[i].groups) for i, name in enumerate(PHASES)}


def ct_launch_count() -> int:
    return int(load().ct_launch_count())


def ct_back_AT(g: Geom, y, x, stream=None):
    """x = A^T y (2D; the matched adjoint of ct_forward_A)."""
    _check(load().ct_back_AT(g.handle, _ptr(y), _ptr(x), _stream(stream)))


def ct_geom_set_backprojector(g: Geom, kind: str):
    """'pixel' (the unmatched B, default) or 'adjoint' (B = A^T, 2D)."""
    k = {"pixel": 0, "adjoint": 1}[kind]
    _check(load().ct_geom_set_backprojector(g.handle, k))


def _shapes_dict(sh) -> dict:
    return {"a_threads": sh.a_threads, "a_views": sh.a_views, "a_slab": sh.a_slab,
            "b_rows": sh.b_rows, "b_views": sh.b_views, "a_rays": sh.a_rays,
            "a_warp_views": sh.a_warp_views, "b_warp_rows": sh.b_warp_rows}


def ct_geom_set_launch_shapes(g: Geom, shapes: dict):
    sh = LaunchShapes(int(shapes["a_threads"]), int(shapes["a_views"]), int(shapes["a_slab"]),
                      int(shapes["b_rows"]), int(shapes["b_views"]), int(shapes.get("a_rays", 1)),
                      int(shapes.get("a_warp_views", 1)), int(shapes.get("b_warp_rows", 1)))
    _check(load().ct_geom_set_launch_shapes(g.handle, ctypes.byref(sh)))


def ct_geom_get_launch_shapes(g: Geom) -> dict:
    sh = LaunchShapes()
    _check(load().ct_geom_get_launch_shapes(g.handle, ctypes.byref(sh)))
    return _shapes_dict(sh)


def ct_geom_autotune(g: Geom, stream=None) -> dict:
    """Time the projector launch shapes on this geometry; returns the chosen shapes."""
    sh = LaunchShapes()
    _check(load().ct_geom_autotune(g.handle, _stream(stream), ctypes.byref(sh)))
    return _shapes_dict(sh)


def _info_dict(inf):
    return dict(iters_done=inf.iters_done, beta=inf.beta, final_lambda=inf.final_lambda,
                final_resid=inf.final_resid, status=STATUS_NAMES[inf.status],
                fast_path_steps=inf.fast_path_steps,
                lambda_fallback_steps=inf.lambda_fallback_steps)


class Batch:
    """ct_batch: many independent problems solved through one captured CUDA graph."""

    def __init__(self, geoms, methods=None, max_iters=30, rule="gcv", lambda_fixed=0.0, tau=1.01,
                 reorth=1, basis="f32", autotune=True, lambda_net=None):
        lib = load()
        self.geoms = list(geoms)
        n = len(self.geoms)
        o, _, _, _ = _opts(max_iters, rule, lambda_fixed, 0.0, tau, reorth, basis, False,
                           lambda_net)
        self._o = o
        self._net = lambda_net
        gh = (ctypes.c_void_p * n)(*[g.handle.value for g in self.geoms])
        mth = None
        if methods is not None:
            m = [{"ab": 0, "ba": 1, "auto": 2}.get(x, x) for x in methods]
            mth = (ctypes.c_int * n)(*m)
        h = ctypes.c_void_p()
        _check(lib.ct_batch_create(n, gh, mth, ctypes.byref(o), 1 if autotune else 0, ctypes.byref(h)))
        self.handle = h
        self.n = n

    def solve(self, b_list, x_list, noise_norms=None, stream=None):
        lib = load()
        n = self.n
        bp = (ctypes.c_void_p * n)(*[_ptr(b).value for b in b_list])
        xp = (ctypes.c_void_p * n)(*[_ptr(x).value for x in x_list])
        nz = (ctypes.c_double * n)(*noise_norms) if noise_norms is not None else None
        infos = (HybridInfo * n)()
        _check(lib.ct_batch_solve(self.handle, bp, xp, nz, infos, _stream(stream)))
        return [_info_dict(infos[i]) for i in range(n)]

    def launches(self) -> int:
        return int(load().ct_batch_launches(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            load().ct_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def abba_solve(geoms, b_list, x_list, methods=None, max_iters=30, rule="gcv", lambda_fixed=0.0,
               noise_norms=None, tau=1.01, basis="f32", stream=None, lambda_net=None):
    """One-shot batched solve (creates, solves and destroys a ct_batch)."""
    lib = load()
    n = len(geoms)
    o, _, _, _ = _opts(max_iters, rule, lambda_fixed, 0.0, tau, 1, basis, False, lambda_net)
    gh = (ctypes.c_void_p * n)(*[g.handle.value for g in geoms])
    mth = None
    if methods is not None:
        mth = (ctypes.c_int * n)(*[{"ab": 0, "ba": 1, "auto": 2}.get(x, x) for x in methods])
    bp = (ctypes.c_void_p * n)(*[_ptr(b).value for b in b_list])
    xp = (ctypes.c_void_p * n)(*[_ptr(x).value for x in x_list])
    nz = (ctypes.c_double * n)(*noise_norms) if noise_norms is not None else None
    infos = (HybridInfo * n)()
    _check(lib.abba_solve(n, gh, bp, xp, mth, ctypes.byref(o), nz, infos, _stream(stream)))
    return [_info_dict(infos[i]) for i in range(n)]


# ------------------------------------------------------------------ learned lambda

def ct_mlp_forward(params, X, out, bf16=True, stream=None):
    """out[i] = net(X[i]) for the n x 80 feature rows X (FP32 CUDA tensors)."""
    _check(load().ct_mlp_forward(_ptr(params), _ptr(X), int(X.shape[0]), _ptr(out),
                                 1 if bf16 else 0, _stream(stream)))


def ct_mlp_grad(params, X, Y, grad, loss=None, bf16=True, stream=None):
    """grad <- d/dparams of mean((net(X) - Y)^2); loss (1-element tensor) <- that mean."""
    _check(load().ct_mlp_grad(_ptr(params), _ptr(X), _ptr(Y), int(X.shape[0]), _ptr(grad),
                              _ptr(loss), 1 if bf16 else 0, _stream(stream)))


def ct_mlp_adam(params, grad, m, v, lr, t, stream=None):
    _check(load().ct_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), float(lr), int(t),
                              _stream(stream)))


def ct_mlp_train(params, m, v, X, Y, batch, epochs, lr, t=0, loss_hist=None, bf16=True,
                 stream=None):
    """Mini-batch Adam training; returns the updated Adam step counter."""
    tc = ctypes.c_int(int(t))
    _check(load().ct_mlp_train(_ptr(params), _ptr(m), _ptr(v), _ptr(X), _ptr(Y),
                               int(X.shape[0]), int(batch), int(epochs), float(lr),
                               ctypes.byref(tc), _ptr(loss_hist), 1 if bf16 else 0,
                               _stream(stream)))
    return tc.value


def ct_lambda_samples(g, b, x_true, x, feats, labels, max_iters=30, rule="gcv", stream=None):
    """Features (K x 80) and labels (K) of the learned lambda rule from one AB solve."""
    o, _, _, _ = _opts(max_iters, rule, 0.0, 0.0, 1.01, 1, "f32", False)
    info = HybridInfo()
    _check(load().ct_lambda_samples(g.handle, _ptr(b), _ptr(x_true), ctypes.byref(o), _ptr(x),
                                    _ptr(feats), _ptr(labels), ctypes.byref(info),
                                    _stream(stream)))
    return _info_dict(info)


def ct_test_drop_tile_copy(enable: bool, wait_cycles: int = 1 << 20):
    """Test hook of the bounded device waits (see include/ctabba.h): armed, the next
    Gram-Schmidt tile pass leaves one tile's copies unissued so its wait runs out."""
    _check(load().ct_test_drop_tile_copy(1 if enable else 0, int(wait_cycles)))


PROBES = {"gather8": 0, "mufu": 1}


def ct_probe(kind, reps, out, stream=None) -> int:
    """Launch one throughput probe ('gather8' or 'mufu'); returns its operation count."""
    ops = ctypes.c_int64(0)
    _check(load().ct_probe(PROBES[kind] if isinstance(kind, str) else int(kind), int(reps),
                           _ptr(out), int(out.numel()), ctypes.byref(ops), _stream(stream)))
    return int(ops.value)
