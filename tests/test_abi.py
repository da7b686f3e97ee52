"""The C-ABI library loads and exports every entry point declared in include/*.h; invalid
arguments are rejected on the host before any CUDA call (no GPU needed)."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_17892_gb300 import build as B
    B.build()
    from paper_2602_17892_gb300 import _binding
    return _binding.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b([A-Za-z_]\w*)\s*\([^;{]*\)\s*;", text, re.M):
            if m.group(1) not in ("if", "while", "for", "sizeof"):
                names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for fn in ("ct_geom_create", "ct_forward_A", "ct_back_B", "ab_gmres_hybrid",
               "ba_gmres_hybrid"):
        assert fn in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = sorted(n for n in _declared() if n not in exported)
    assert not missing, missing
    for n in _declared():
        getattr(lib, n)


def test_invalid_geometry_rejected_without_gpu(lib):
    from paper_2602_17892_gb300 import _binding as Bn
    ang = np.zeros(4)
    with pytest.raises(Bn.CtError) as ei:
        Bn.Geom("parallel2d", 0, 8, ang, 10, 1.0)
    assert ei.value.status == Bn.CT_EINVAL
    with pytest.raises(Bn.CtError):
        Bn.Geom("fanflat2d", 64, 64, ang, 10, 1.0, sid=10.0, sdd=20.0)   # source inside image
    with pytest.raises(Bn.CtError):
        Bn.Geom("parallel2d", 8, 8, ang, 10, -1.0)
    assert lib.ct_status_string(4) == b"CT_BREAKDOWN"


def test_solver_rejects_bad_options(lib):
    from paper_2602_17892_gb300 import _binding as Bn
    o = Bn.HybridOpts()
    lib.ct_hybrid_opts_default(ctypes.byref(o))
    assert o.max_iters == 30 and o.rule == 2 and o.reorth == 1
    st = lib.ab_gmres_hybrid(None, None, None, None, ctypes.byref(o), None, None)
    assert st == Bn.CT_EINVAL
    st = lib.ct_projected_solve(None, 2, 1, 1.0, 0, 0.0, 0.0, None, None, None, None)
    assert st == Bn.CT_EINVAL


def test_launch_shape_entry_points_reject_null_arguments(lib):
    from paper_2602_17892_gb300 import _binding as Bn
    sh = Bn.LaunchShapes(256, 1, 16, 8, 1, 1, 1, 1)
    assert lib.ct_geom_set_launch_shapes(None, ctypes.byref(sh)) == Bn.CT_EINVAL
    assert lib.ct_geom_get_launch_shapes(None, ctypes.byref(sh)) == Bn.CT_EINVAL


def test_learned_lambda_entry_points_reject_bad_arguments(lib):
    from paper_2602_17892_gb300 import _binding as Bn
    o = Bn.HybridOpts()
    lib.ct_hybrid_opts_default(ctypes.byref(o))
    assert o.lambda_net_dev is None and o.features_dev is None
    assert lib.ct_mlp_forward(None, None, 4, None, 1, None) == Bn.CT_EINVAL
    assert lib.ct_mlp_grad(None, None, None, 4, None, None, 1, None) == Bn.CT_EINVAL
    assert lib.ct_mlp_adam(None, None, None, None, 1e-3, 1, None) == Bn.CT_EINVAL
    t = ctypes.c_int(0)
    assert lib.ct_mlp_train(None, None, None, None, None, 4, 4, 1, 1e-3, ctypes.byref(t), None,
                            1, None) == Bn.CT_EINVAL
    assert lib.ct_lambda_samples(None, None, None, ctypes.byref(o), None, None, None, None,
                                 None) == Bn.CT_EINVAL
    # the learned rule without a network is refused before anything is launched
    o.rule = Bn.RULES["learned"]
    st = lib.ab_gmres_hybrid(ctypes.c_void_p(1), ctypes.c_void_p(16), None, ctypes.c_void_p(16),
                             ctypes.byref(o), None, None)
    assert st == Bn.CT_EINVAL and b"lambda_net_dev" in lib.ct_last_error()
    assert Bn.CT_MLP_NPARAMS == 64 * 80 + 64 + 64 * 64 + 64 + 64 + 1 + 2 * 80


def test_ncp_rule_and_test_hook_are_checked_on_the_host(lib):
    from paper_2602_17892_gb300 import _binding as Bn
    o = Bn.HybridOpts()
    lib.ct_hybrid_opts_default(ctypes.byref(o))
    assert not o.ncp_hist
    o.stop_rule = 4                                     # no such rule
    assert lib.ab_gmres_hybrid(ctypes.c_void_p(1), ctypes.c_void_p(16), None,
                               ctypes.c_void_p(16), ctypes.byref(o), None, None) == Bn.CT_EINVAL
    o.stop_rule = Bn.STOPS["ncp"]
    o.stop_every = 0
    assert lib.ba_gmres_hybrid(ctypes.c_void_p(1), ctypes.c_void_p(16), None,
                               ctypes.c_void_p(16), ctypes.byref(o), None, None) == Bn.CT_EINVAL
    assert lib.ct_test_drop_tile_copy(1, 10) == Bn.CT_EINVAL   # limit below 2^16


def test_launch_shape_fields_match_the_header_and_the_bench():
    """ct_launch_shapes in include/ctabba.h, the binding's ctypes structure and the benchmark's
    --launch-shapes keys list the same int fields in the same order; --launch-shapes takes six
    integers (one view per Joseph warp, one pixel row per B warp) or all eight."""
    import bench
    from paper_2602_17892_gb300 import _binding as Bn
    text = open(os.path.join(ROOT, "include", "ctabba.h")).read()
    body = text.split("} ct_launch_shapes;")[0].rsplit("typedef struct {", 1)[1]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\bint\s+(\w+)\s*;", body)
    assert fields == [f[0] for f in Bn.LaunchShapes._fields_]
    assert list(bench.SHAPE_KEYS) == fields
    assert bench.parse_shapes("128,4,16,4,4,1") == [128, 4, 16, 4, 4, 1, 1, 1]
    assert bench.parse_shapes("128,4,16,4,4,1,4,2") == [128, 4, 16, 4, 4, 1, 4, 2]
    with pytest.raises(SystemExit):
        bench.parse_shapes("128,4,16,4,4,1,4")
