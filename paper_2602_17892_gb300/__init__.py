"""GB300-native hybrid AB-/BA-GMRES for X-ray CT with an unmatched projector pair.

The numerical path lives in ``libctabba.so`` (hand-written CUDA for sm_103a, C ABI declared in
``include/ctabba.h``); this package holds its CUDA sources (``csrc/``), the nvcc build script
(``build.py``) and a ctypes binding (``_binding.py``) whose functions carry the C names.
"""
from ._binding import (Batch, CtError, Geom, ab_gmres_hybrid, ab_gmres_hybrid_restarted,
                       abba_solve, ba_gmres_hybrid, ba_gmres_hybrid_restarted,
                       ct_arnoldi_step, ct_back_AT, ct_back_B, ct_forward_A, ct_geom_autotune,
                       ct_geom_set_backprojector,
                       ct_geom_get_launch_shapes, ct_geom_set_launch_shapes, ct_lambda_samples, ct_mlp_adam, ct_mlp_forward, ct_mlp_grad, ct_mlp_train,
                       ct_projected_solve, load)

__all__ = ["Batch", "CtError", "Geom", "ab_gmres_hybrid", "ab_gmres_hybrid_restarted",
           "abba_solve", "ba_gmres_hybrid", "ba_gmres_hybrid_restarted",
           "ct_arnoldi_step", "ct_back_AT", "ct_back_B", "ct_forward_A", "ct_geom_autotune",
           "ct_geom_set_backprojector",
           "ct_geom_get_launch_shapes", "ct_geom_set_launch_shapes", "ct_lambda_samples", "ct_mlp_adam", "ct_mlp_forward", "ct_mlp_grad", "ct_mlp_train",
           "ct_projected_solve", "load"]
