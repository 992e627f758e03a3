"""Plain, slow CPU FP64 oracle for the non-nested multigrid hot path (TEST INFRASTRUCTURE).

This package is test infrastructure only. It may be imported by ``tests/``, by
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline / reference leg, and by
nothing else; the product path (the CUDA library and its binding) never imports or
calls it, and the two share no code. The only shared module is the seeded input
generator ``paper_2402_12947_gb300.inputs`` (geometry only).

Modules follow the paper (Chen & Wells, "Multigrid on unstructured meshes with regions of
low quality cells"), section by section:
  quadrature  exact simplex quadrature (collapsed Gauss-Legendre) used by the assembly
  fem         Lagrange P1/P2 DoF maps, Dirichlet elimination, stiffness and load (Sec. 6.1)
  quality     normalised radius ratio gamma (Sec. 3, Eq. radius_ratio)
  patches     low-quality regions Omega_b, Omega_B and DoF sets B_d (Sec. 4.4, Sec. 4.1)
  transfer    interpolation prolongation P, R = P^T, Galerkin A_{l+1} (Sec. 2, Eqs. 2-4)
  eig         largest eigenvalue of D^{-1}A, adjusted eigenvalue (Sec. 3.2, Sec. 5)
  smoother    Chebyshev-Jacobi S_g, local correction S_c (Alg. 2), sandwich S_gc (Sec. 4.2)
  mg          V-cycle (Alg. 1), MG-preconditioned CG (Sec. 6.2), stationary MG
  hierarchy   building all of the above for a list of meshes

Parity status of each function is stated in its module header; every function here
is pinned by a ``-m "not gpu"`` test against closed forms, invariants or brute force.
"""
