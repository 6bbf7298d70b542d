"""Independent FP64 CPU oracle for the space-time Biot slab operator and solver.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import or call this
package.  The product path (the CUDA library and its Python binding) never
imports it, and this package imports nothing from the product path except the
seeded input generators (`paper_1801_04984_gb300.inputs`), which hold no
arithmetic of the method.

Everything here is plain numpy/scipy in float64, written from the paper
(Köcher, "Space-Time-Parallel Poroelasticity Simulation"):

* `timebasis` - dG(r) time matrices in a Legendre (modal) basis, the right-Radau
  nodal basis by an exact change of basis, and the stability functions
  (§Discretisation in Time).
* `space`     - Q2 displacement / RT1 flux / DGQ1 pressure matrices assembled by
  cellwise Gauss quadrature on Cartesian meshes (§Poroelasticity strong form,
  §Discretisation in Space).
* `slab`      - the monolithic slab system, loads, constraints, direct solves,
  time marching, the goal functional and its adjoint (§Monolithic Approach).
* `exact`     - closed forms: manufactured solutions and Terzaghi consolidation.
* `dwr`       - dual-weighted residual indicators of the dG(r) time error against
  dG(r+1) for a goal functional (§Abstract: duality-based adaptivity).

Parity status: every function is pinned by `tests/test_oracle_*.py` except the
Krylov/preconditioner iteration counts, which the oracle does not model
("parity unpinned" for iteration counts; the oracle pins solutions only).
"""
