"""Oracle: a plain, slow, CPU FP64 restatement of the space-time IgA heat solver.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path (the CUDA library and its Python binding) never
imports, calls or links anything here, and nothing here imports the product.

Every function follows the paper "An efficient solver for space-time
isogeometric Galerkin methods for parabolic problems" (Loli, Montardini,
Sangalli, Tani) and cites the section / equation it restates:

* ``bspline``  -- open knot vectors and the Cox-de Boor recursion (Sec. 2.1).
* ``matrices`` -- univariate mass / stiffness / time-derivative matrices by
  Gauss quadrature and the initial/boundary reduction (Sec. 2.2, eqs.
  time_mat and space_mat, Sec. 4 univariate factors).
* ``assemble`` -- the space-time system matrix A and preconditioner P
  assembled directly by (d+1)-dimensional quadrature of the bilinear form
  (Sec. 3.1-3.3), never by Kronecker products.
* ``direct``   -- banded Gaussian elimination with partial pivoting, an
  independent check of the sparse direct solves (Sec. 3.3, eq. sys_solve).
* ``kron``     -- m-mode products and the Kronecker form of A (eqs.
  kron_vec_multi, syst_mat).
* ``fd``       -- Algorithm 1 (extended Fast Diagonalization) in complex
  arithmetic exactly as written in Sec. 4.1-4.3.
* ``gmres``    -- right-preconditioned GMRES with modified Gram-Schmidt and
  Givens rotations, zero initial guess (Sec. 4.5 and Sec. 5 set-up).
* ``loads``    -- load vectors and point evaluation of discrete solutions for
  manufactured solutions (Sec. 3.1 linear form F).
* ``geometry`` -- the exact NURBS quarter-annulus map and its Jacobian (the
  domain of Sec. 5, extruded in 3D).
* ``mapped``   -- spatial mass / stiffness matrices on a mapped domain with
  variable coefficients (Sec. 4.6 and 4.6.1), the geometry-aware
  preconditioner (eqs. separation, over_A, prec_geo) and the adjoint gradient
  of a solution misfit (built from the paper's algebra; not in the paper).

Pins (tests marked ``not gpu``) tie each function to facts the paper and the
mathematics fix: partition of unity, closed-form uniform B-spline matrices,
W_t + W_t^T = e_n e_n^T (eq. integral_W), Tables 1 and 3, the arrowhead
identities of eq. time_eig_2, direct sparse solves, a manufactured
polynomial solution that lies in the spline space, the area of the quarter
annulus, the optimal L2 convergence rate of a manufactured solution on it,
exact recovery of separable coefficient data, and central finite differences
of the loss. No function here is "parity unpinned".
"""
