"""Oracle for the TT-IGA hot path: a plain, slow, obviously correct FP64 CPU code.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
package; only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
reference arm of ``bench.py`` may use it.  It shares no code with the CUDA
library: its own knots, Gauss rule (Newton on Legendre polynomials), Cox-de
Boor basis, NURBS geometry, hyper-dual Laplacian, full-grid element assembly,
Jacobi-PCG and TT definitions.

Modules and the passages they follow:

* spline        -- Section 2 (knots, Cox-de Boor, derivative, NURBS, Fig. 1)
* geometry      -- Section 3.3 (exact geometry map, J, det J) and Eq. (Rxi)
* hyperdual     -- exact second derivatives for f = -Laplace(u) (Section 3.1)
* manufactured  -- manufactured solutions with homogeneous Dirichlet data
* iga           -- Eqs. (Kfinal), (ffinal), Section 3.4 Dirichlet, CG, Eq. (L2norm)
* tt            -- Section 4.1 TT format, TT-matrix format, TT-SVD rank
                   definition, and the Section 4.2 per-direction contraction
                   and Eq. (K = sum K_ij) as plain definitions

Each module's docstring lists its pins (tests/test_oracle_*.py).
"""
