"""Plain FP64 CPU oracle of the matrix-free modal DG + p-multigrid FGMRES step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, calls or links anything here, and nothing here imports the product.

Method: Franciolini, Fidkowski & Crivellini, "Efficient discontinuous Galerkin
implementations and preconditioners for implicit unsteady compressible flow
simulations" (arXiv 1812.04789).  Every function cites the section / equation /
algorithm it follows.  The code is written for a reader checking it against
the paper by eye: whole-mesh numpy arrays, no blocking, no fusion.

Modules
  basis    -- orthonormal Legendre total-degree basis, Gauss-Legendre rules (Sec. 3)
  physics  -- NS closure, inviscid/viscous fluxes, Roe flux (Sec. 2, Sec. 3.1)
  dg       -- mesh, residual R(W) of eq. (dg_ns) with BR2 (eqs. visc_flux, re),
              exact JVP by complex step, FD JVP of eq. (DG-mf)
  blocks   -- Jacobian blocks (diagonal and neighbour), inheritance (Sec. 5.1), PLU
  tri      -- DG on periodic triangulations, full-order Dubiner basis, blocks and pMG (Sec. 3)
  bilu     -- block ILU(0) of the coarsest level, MDF / natural / colour orders (Sec. 6.3)
  solvers  -- GMRES(BJ) smoother, MG_V (Alg. 2), MG_full (Alg. 1), FGMRES,
              BDF2 Newton step

Pins: every function is checked against something other than itself in
``tests/test_oracle_*.py`` (closed forms, invariants, library routines, brute
force on tiny inputs).  Functions with no such pin say "parity unpinned" in
their docstring.
"""
