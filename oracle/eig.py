"""Largest eigenvalue of the Jacobi-scaled operator (oracle; test infrastructure only).

Sec. 3.2 / Sec. 6: the Chebyshev smoother needs lambda_max, estimated in the paper by
Krylov-Schur to 1e-8; lambda_min = lambda_max / 10. Reading: the operator is D^{-1}A
(the values in Table eig_cube, ~2 on good meshes, are those of a Jacobi-scaled
Laplacian), computed here through the similar symmetric matrix D^{-1/2} A D^{-1/2}.
Sec. 5: the adjusted eigenvalue is lambda_max of the block A_gg, g = the DoFs outside
the closure of Omega_B (the complement of the union of the B_d); with no patches it
equals the unadjusted value.

Dense ``eigvalsh`` for n <= 3000, else ARPACK Lanczos (``eigsh``) to 1e-12.

Pinned by tests/test_oracle_smoother.py: dense vs Lanczos agreement, Cauchy interlacing
(adjusted <= unadjusted), and the 1D/2D closed-form spectra of small Laplacians.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

DENSE_MAX = 3000


def _scaled(A: sp.csr_matrix, keep: np.ndarray | None):
    d = A.diagonal()
    s = 1.0 / np.sqrt(d)
    S = sp.diags(s) @ A @ sp.diags(s)
    if keep is not None:
        S = S[keep][:, keep]
    return S.tocsr()


def lambda_max(A: sp.csr_matrix, keep: np.ndarray | None = None) -> float:
    S = _scaled(A, keep)
    n = S.shape[0]
    if n == 0:
        return 0.0
    if n <= DENSE_MAX:
        return float(np.linalg.eigvalsh(S.toarray())[-1])
    v0 = np.random.default_rng(12345).uniform(-1, 1, n)
    val = spla.eigsh(S, k=1, which="LA", tol=1e-12, v0=v0, maxiter=20000, return_eigenvectors=False)
    return float(val[0])


def adjusted_lambda_max(A: sp.csr_matrix, patches: list[np.ndarray]) -> float:
    if not patches:
        return lambda_max(A)
    keep = np.ones(A.shape[0], dtype=bool)
    keep[np.concatenate(patches)] = False
    return lambda_max(A, keep)
