"""FP64 CPU oracle for hybrid AB-/BA-GMRES with an unmatched CT projector pair.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import, call or link anything in this package.  It shares no code with
the CUDA library (``paper_2602_17892_gb300``) and neither imports the other; the only common
dependency is the seeded input module ``synth``.

Contents:
  projectors.c / proj.py   Joseph forward projector A, pixel/voxel-driven backprojector B,
                           matched Joseph adjoint A^T (plain FP64 C, optional OpenMP).
  solver.py                Algorithms 1 and 2 with MGS + one reorthogonalisation pass, the
                           SVD-based projected Tikhonov step, GCV and discrepancy-principle
                           lambda rules, Givens GMRES, Golub-Kahan LSQR/LSMR comparators.

Pins (tests marked "not gpu") tie each function to something other than itself: disc
chords and exact line integrals of affine images, exact special angles, the adjoint
identity, B applied to constants, the Arnoldi relation and orthogonality, the matched-case
equivalences with LSQR/LSMR, brute-force minimisation over explicit Krylov bases, the
full-dimension closed forms and dense evaluation of GCV.
"""
