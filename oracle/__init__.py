"""Plain FP64 CPU oracle for the ADR amplitude solver.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of bench.py may import or run anything in this package; the
product path (the CUDA library and its Python binding) never does, and this
package imports nothing from the product.

It restates, slowly and literally, what Treister & Haber compute in "A
multigrid solver to the Helmholtz equation with a point source based on
travel time and amplitude":

* `adr`       -- travel-time coefficients (Eq. travel_time_coeff), the ADR
                 rows with central / first- and second-order upwind advection
                 (Eqs. ADR, londDiff, londUpwindDiff, 1up), the averaging mass
                 of the Delta-tau term (Sec. 2.3), Neumann boundary rows
                 (Eq. BCADR), the standard Helmholtz matrix H
                 (Eq. HelmholtzLinSystem), the point-source right-hand side
                 and the reconstruction u = a exp(-i omega tau) (Eq. new_u).
* `multigrid` -- bilinear/trilinear prolongation, Galerkin coarse operators
                 (Eq. coarseGridMatrix), damped Jacobi, the V-cycle built from
                 the two-grid cycle (Algorithm TwoGrid), the fixed-count
                 Jacobi-preconditioned GMRES coarsest solve (Sec. 3.1).
* `krylov`    -- flexible GMRES with classical Gram-Schmidt applied twice.
* `eikonal`   -- factored-eikonal fast marching (Eq. factoredEikonal).
* `twostage`  -- the two-stage solve of the central ADR system
                 (Algorithm ADRlong): a low-accuracy H_1up solve, then the
                 shifted-Laplacian FGMRES on the system rescaled as Helmholtz.
* `adjoint`   -- receiver misfit and its slowness gradient by the adjoint
                 state of the assembled system (not in the paper).

Every function is FP64 and single-threaded; scipy.sparse supplies the sparse
matrix products and direct solves used as library steps.
"""
