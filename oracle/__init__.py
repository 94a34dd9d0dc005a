"""Plain FP64 CPU oracle for the Ga (Galerkin with exact integration) scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_1412_2033_gb300``) never imports it and
shares no code with it: the oracle has its own DFT/FFT, its own coefficient
formulas, its own projections and its own conjugate gradients, all written from
the paper (Vondrejc, "Improved guaranteed computable bounds on homogenized
properties of periodic media by Fourier-Galerkin method with exact integration",
arXiv:1412.2033):

* ``fourier``       -- index sets Z_N (Def. trig_pol, eq. index_set), the DFT
                       convention of eq. DFT_coef / eq. DFT, a naive DFT and an
                       own recursive mixed-radix + Bluestein FFT.
* ``coefficients``  -- Fourier coefficients of the characteristic functions
                       (Remark anal_Fourier, eq. char_func_Four), the sphere
                       coefficient the paper does not print, and the
                       inclusion-matrix composite table (eq. inclcomp_formula).
* ``image``         -- grid-based (pixel / voxel image) composites (Lemma
                       grid_compos, Remark eval_with_FFT): the coefficient table
                       of a piecewise-constant image and its Ga bounds.
* ``gani``          -- the GaNi scheme (Def. GaNi, Algorithm 1): point samples
                       of the coefficient, the trapezoidal-rule operator, the
                       GaNi matrices and the a-posteriori guaranteed bounds
                       (eq. GaNi_apost).
* ``galerkin``      -- Helmholtz projections (Def. projection), the fully
                       populated Galerkin matrix (Lemma FD_matrix_full), the
                       double-grid values A_M (Lemma integ_eval_VM, eq. MBA_GA),
                       the double-grid operator (Algorithm 2, Cor. Ga_linsys),
                       conjugate gradients (Remark CG) and the guaranteed bounds
                       (Def. Ga, Prop. struct_bounds, eq. spd_inverse_ineq).

Every function is FP64.  Pins (checks against facts the paper and mathematics
fix, not against the oracle itself) live in ``tests/test_oracle_*.py``.
Parity status: the matvec, coefficient tables, double-grid values, CG and
bounds are pinned (closed forms, brute force, library FFT, quadrature,
invariants).  The paper prints no value reproducible without its missing
voxel image, so no absolute bound is pinned to a printed number.
"""
