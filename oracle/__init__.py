"""FP64 CPU oracle of the background-decomposed, preconditioned PSFD method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library.

It is a plain, slow, obviously-correct restatement of the method in complex128
PyTorch CPU ops (library FFTs, matmuls and dense LU serve as steps):

* ``oracle.psfd``   - grid, PML, Gaussian smoothing, transfer-matrix reflection,
                      reflection operator R_ml, operator A, its adjoint, the
                      spectral-damping preconditioner M and the source b
                      (Sec. 2.2, Eqs. bg_source / vector_helmholtz_operator;
                      Sec. 3, Eqs. spectral_damping_action / _mask).
* ``oracle.krylov`` - right-preconditioned BiCGSTAB and GMRES(m) with the
                      affine warm start E = E_base + M y (Eqs.
                      right_preconditioned, right_correction_solution,
                      right_preconditioned_system), relative residual
                      (Eq. relative_residual), dense assembly + LU.
* ``oracle.fno``    - factorised FNO forward (Sec. 2.1, Eqs. 1-4) and the
                      physics-informed loss (Eq. loss).
* ``oracle.metric`` - threshold-contour widths of the scattered-field
                      intensity along scan lines and their deviation from a
                      reference solution (Sec. 4, practical assessment,
                      Eq. logistic_sigmoid).

Parity status of each function is stated in its module header.
"""
