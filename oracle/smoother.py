"""Smoothers of the global-local combined smoother (oracle; test infrastructure only).

S_g, Sec. 3.2 / Sec. 5: Jacobi-preconditioned Chebyshev semi-iteration on D^{-1}A over the
interval [lmin, lmax], lmin = lmax/10 (the three-term recurrence of the Hageman-Young
text the paper cites). With theta = (lmax+lmin)/2, delta = (lmax-lmin)/2, sigma =
theta/delta, one application of degree k is
    r = b - A x;  d = D^{-1} r / theta;  x += d;  rho = 1/sigma
    repeat k-1 times:  r = b - A x;  rho' = 1/(2 sigma - rho);
                       d = rho' rho d + (2 rho'/delta) D^{-1} r;  x += d;  rho = rho'
so that the error is multiplied by T_k((theta - D^{-1}A)/delta) / T_k(theta/delta).

S_c, Sec. 4.1 (Eqs. local_system .. local_update, Alg. 2): with one residual r = b - A x,
x += sum_d I_d (I_d^T A I_d)^{-1} I_d^T r, each local system solved directly (dense
Cholesky). Reading for semi-definite blocks: on coarse levels built from degenerate cells
P can lose column rank, so a Galerkin block P^T A P may be singular (its residuals are
still consistent: orthogonal to P's null space). The direct method is a Cholesky in
which a pivot at or below 1e-10 of its original diagonal marks that DoF as dependent on
the previous ones; dependent DoFs get a zero correction and the others are solved
exactly. For SPD blocks nothing is dropped and this is the plain Cholesky solve.

S_gc, Sec. 4.2: the sandwich S_c, then S_g, then S_c; the explicit form is
S_gc = 2 S_c - S_c A S_c + (I - S_c A) S_g (I - A S_c).
Reading for the smoother order option: "sandwich" (default, the paper's form);
"global_then_local" applies S_g then S_c before the coarse correction and S_c then S_g
after it (still symmetric); "global" is S_g alone (no local correction).

S_g alternative (the paper's other global smoother, Sec. 3.1 and Sec. 6: symmetric
Gauss-Seidel): a multicolour symmetric Gauss-Seidel sweep. Rows are coloured greedily in
index order (the smallest colour not used by an already coloured neighbour; couplings
below 1e-12 sqrt(a_ii a_jj), rounding residue of the Galerkin products, are ignored);
a forward
sweep updates the colours 0..C-1 in turn, each colour's rows at once
(x_i += (b - A x)_i / a_ii), and a backward sweep the colours C-1..0. This is exactly
sequential symmetric Gauss-Seidel in the colour-sorted row order.

Pinned by tests/test_oracle_smoother.py: Chebyshev error polynomial against the
closed form via a dense eigendecomposition; S_c exact when one patch covers all DoFs;
S_gc applied to unit vectors equals the explicit formula and is symmetric; no patches
reduces S_gc to S_g bit for bit.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def chebyshev_coefficients(lmax: float, lmin: float, k: int):
    """Per-step (c_d, c_r): d = c_d d + c_r D^{-1} r (c_d = 0 on the first step)."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    out = [(0.0, 1.0 / theta)]
    for _ in range(1, k):
        rho_new = 1.0 / (2.0 * sigma - rho)
        out.append((rho_new * rho, 2.0 * rho_new / delta))
        rho = rho_new
    return out


def chebyshev(A: sp.csr_matrix, dinv: np.ndarray, b: np.ndarray, x: np.ndarray,
              lmax: float, lmin: float, k: int) -> np.ndarray:
    x = x.copy()
    d = np.zeros_like(x)
    for cd, cr in chebyshev_coefficients(lmax, lmin, k):
        r = b - A @ x
        d = cd * d + cr * (dinv * r)
        x = x + d
    return x


DROP_TOL = 1e-10


def dependent_dofs(Ad: np.ndarray) -> np.ndarray:
    """Column-by-column Cholesky of a symmetric positive semi-definite matrix; returns the
    mask of DoFs whose pivot is <= DROP_TOL times their diagonal (dependent DoFs)."""
    n = Ad.shape[0]
    L = np.zeros_like(Ad)
    drop = np.zeros(n, dtype=bool)
    for j in range(n):
        s = Ad[j, j] - L[j, :j] @ L[j, :j]
        if not Ad[j, j] > 0 or s < -DROP_TOL * Ad[j, j]:
            raise np.linalg.LinAlgError("matrix is not positive semi-definite")
        if s <= DROP_TOL * Ad[j, j]:
            drop[j] = True
            continue
        L[j, j] = np.sqrt(s)
        L[j + 1:, j] = (Ad[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return drop


class DirectSolver:
    """Direct solve with a dense SPD (or consistent semi-definite) matrix, see module doc."""

    def __init__(self, Ad: np.ndarray):
        self.keep = ~dependent_dofs(Ad)
        self.factor = sla.cho_factor(Ad[np.ix_(self.keep, self.keep)], lower=True)

    def solve(self, r: np.ndarray) -> np.ndarray:
        e = np.zeros_like(r)
        e[self.keep] = sla.cho_solve(self.factor, r[self.keep])
        return e


class LocalSolver:
    """Direct solvers for A^{[d]} = A[B_d, B_d] of each patch (Sec. 4.1)."""

    def __init__(self, A: sp.csr_matrix, patches: list[np.ndarray]):
        self.patches = patches
        self.factors = [DirectSolver(A[B][:, B].toarray()) for B in patches]

    def apply(self, A: sp.csr_matrix, b: np.ndarray, x: np.ndarray) -> np.ndarray:
        if not self.patches:
            return x.copy()
        r = b - A @ x
        x = x.copy()
        for B, fac in zip(self.patches, self.factors):
            x[B] += fac.solve(r[B])
        return x


COLOUR_TOL = 1e-12


def greedy_colouring(A: sp.csr_matrix) -> np.ndarray:
    """colour[i] = the smallest colour not taken by a neighbour j < i (index order)."""
    n = A.shape[0]
    d = np.sqrt(np.abs(A.diagonal()))
    colour = -np.ones(n, dtype=np.int64)
    for i in range(n):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        vals = A.data[A.indptr[i]:A.indptr[i + 1]]
        cols = cols[np.abs(vals) > COLOUR_TOL * d[i] * d[cols]]
        used = set(colour[cols].tolist())
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return colour


def multicolour_sgs(A: sp.csr_matrix, dinv: np.ndarray, b: np.ndarray, x: np.ndarray,
                    colour: np.ndarray) -> np.ndarray:
    """One symmetric sweep: colours 0..C-1, then C-1..0."""
    x = x.copy()
    C = int(colour.max()) + 1
    for c in list(range(C)) + list(range(C - 1, -1, -1)):
        rows = np.flatnonzero(colour == c)
        x[rows] += dinv[rows] * (b[rows] - A[rows] @ x)
    return x


def global_smoother(A, dinv, b, x, lmax, lmin, k, kind: str = "chebyshev", colour=None):
    if kind == "chebyshev":
        return chebyshev(A, dinv, b, x, lmax, lmin, k)
    if kind == "sgs":
        return multicolour_sgs(A, dinv, b, x, colour)
    raise ValueError(kind)


def smooth(A, dinv, b, x, lmax, lmin, k, local: LocalSolver | None, order: str, post: bool,
           kind: str = "chebyshev", colour=None):
    """One application of the combined smoother (pre-smoothing unless ``post``)."""
    g = lambda x: global_smoother(A, dinv, b, x, lmax, lmin, k, kind, colour)
    use_local = local is not None and len(local.patches) > 0 and order != "global"
    if not use_local:
        return g(x)
    if order == "sandwich":
        x = local.apply(A, b, x)
        x = g(x)
        return local.apply(A, b, x)
    if order == "global_then_local":
        if not post:
            x = g(x)
            return local.apply(A, b, x)
        x = local.apply(A, b, x)
        return g(x)
    raise ValueError(order)
