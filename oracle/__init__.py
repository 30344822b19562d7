"""Plain, slow, FP64 CPU oracle of the homogenized-multigrid topology-optimization
hot path (arXiv 2201.12931).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
runs this code: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg (and `bench.py --impl reference`) may use it.  It shares no code
with the CUDA path: it assembles the global stiffness matrix explicitly with
scipy.sparse, solves with dense Cholesky / sparse direct / PCG, and evaluates
the filter and the OC update by their plain definitions.

Modules and the passages of the paper they follow:
  element      hex8 reference stiffness K0 (Alg. 4 "Compute K0"; SIMP Eq. K_mod)
  grid         node / element / DOF numbering of the structured brick grid
  assemble     global K(rho) = sum_e E(rho_e) A_e^T K0 A_e and Dirichlet rows
  solve        direct solve (Sec. 3.1) and PCG (Algorithm 1)
  multigrid    trilinear transfers (Sec. 3.2, restriction matrix), the
               homogenized coarse operators (Sec. 4.2.2, Sec. 6), the V-cycle
               (Algorithm 3) and a Galerkin-coarse-operator MG preconditioner
  filter       neighbourhood weights (Eqs. Neighbourhood, NB_dist) used as a
               density filter, and its transpose
  sensitivity  compliance (Eq. compliance objective) and its adjoint
               sensitivity (Eq. sensitivity)
  oc           optimality-criteria update with bisection (Eqs. OCUp1, bisect)

Where the paper is silent or garbled the oracle takes one reading, stated in
the docstring of the function concerned.
"""
