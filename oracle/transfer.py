"""Non-nested transfer operators (oracle; test infrastructure only).

Sec. 2, Eq. (2): [P_l]_ij = phi_j^{(l+1)}(x_i), the coarse basis evaluated at the fine
interpolation points; R_l = P_l^T; Eq. (3): A_{l+1} = P_l^T A_l P_l (Galerkin).

Point location (the paper delegates it to FEniCS): for each free fine DoF point x_i,
the containing coarse cell is the lowest-numbered cell whose barycentric coordinates at
x_i are all >= -1e-12 (points on shared edges/vertices give the same row from any
containing cell, up to rounding). Candidates are all cells whose centroid lies within
the largest cell diameter of x_i, which contains every cell that can hold x_i. Barycentric
coordinates within 1e-12 of zero are set to zero (a point on a face, edge or vertex of
its cell then gives exact zeros instead of rounding residue of either sign), the basis is
evaluated there, entries with |value| < 1e-14 are dropped; columns are the coarse free
DoFs (Dirichlet columns vanish with g = 0).

Reading for degenerate coarse cells: a coarse basis function can vanish at every fine
interpolation point (e.g. the P2 edge DoF of a needle edge much shorter than the fine
mesh size), leaving an empty column of P and an empty row/column of P^T A P. Such a DoF
cannot influence the fine level; it is kept in the numbering with a unit diagonal, so it
is decoupled and always receives a zero correction (equivalent to removing it).

Pinned by tests/test_oracle_transfer.py: identical meshes give P = I; P reproduces any
polynomial of degree <= p exactly; rows of the all-DoF P sum to 1; the Galerkin operator
is symmetric positive definite and equals the dense triple product.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.spatial import cKDTree

from .fem import DofMap, basis_values

LOCATE_TOL = 1e-12
DROP_TOL = 1e-14


class PointLocationError(RuntimeError):
    pass


def barycentric(coords: np.ndarray, cells: np.ndarray, cell_ids: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Barycentric coordinates of pts[k] in cell cell_ids[k] -> [k, dim+1]."""
    X = coords[cells[cell_ids].astype(np.int64)]          # [k, d+1, dim]
    J = np.transpose(X[:, 1:] - X[:, :1], (0, 2, 1))       # columns v_i - v0
    rhs = pts - X[:, 0]
    lam = np.linalg.solve(J, rhs[..., None])[..., 0]
    return np.concatenate([1.0 - lam.sum(axis=1, keepdims=True), lam], axis=1)


def locate(coords: np.ndarray, cells: np.ndarray, pts: np.ndarray):
    """(cell id [npts], barycentric [npts, dim+1]) with the lowest-index containing cell."""
    X = coords[cells.astype(np.int64)]
    cent = X.mean(axis=1)
    diam = 0.0
    d1 = cells.shape[1]
    for a in range(d1):
        for b in range(a + 1, d1):
            diam = max(diam, float(np.max(np.linalg.norm(X[:, a] - X[:, b], axis=1))))
    tree = cKDTree(cent)
    found_cell = np.full(len(pts), -1, dtype=np.int64)
    found_lam = np.zeros((len(pts), d1))
    chunk = 20000
    for s in range(0, len(pts), chunk):
        p = pts[s:s + chunk]
        cand = tree.query_ball_point(p, r=diam * (1.0 + 1e-9) + 1e-15)
        lens = np.array([len(c) for c in cand])
        pid = np.repeat(np.arange(len(p)), lens)
        cid = np.concatenate([np.asarray(c, dtype=np.int64) for c in cand]) if lens.sum() else np.zeros(0, np.int64)
        lam = barycentric(coords, cells, cid, p[pid])
        ok = lam.min(axis=1) >= -LOCATE_TOL
        pid, cid, lam = pid[ok], cid[ok], lam[ok]
        order = np.lexsort((cid, pid))                     # by point, then cell id
        pid, cid, lam = pid[order], cid[order], lam[order]
        first = np.ones(len(pid), dtype=bool)
        first[1:] = pid[1:] != pid[:-1]
        found_cell[s + pid[first]] = cid[first]
        found_lam[s + pid[first]] = lam[first]
    if np.any(found_cell < 0):
        raise PointLocationError(f"{int(np.sum(found_cell < 0))} points outside the coarse mesh")
    return found_cell, found_lam


def prolongation(fine: DofMap, coarse_coords: np.ndarray, coarse_cells: np.ndarray,
                 coarse: DofMap, free_only: bool = True) -> sp.csr_matrix:
    """P: coarse -> fine. Rows: free fine DoFs (all fine DoFs if not free_only); columns:
    free coarse DoFs (all coarse DoFs if not free_only)."""
    rows_g = fine.free if free_only else np.arange(fine.ndofs)
    pts = fine.points[rows_g]
    cell, lam = locate(coarse_coords, coarse_cells, pts)
    lam = np.where(np.abs(lam) <= LOCATE_TOL, 0.0, lam)
    vals = basis_values(lam, coarse.degree, coarse.dim)         # [npts, nloc]
    cols = coarse.cell_dofs[cell]                               # [npts, nloc]
    if free_only:
        cols = coarse.free_index[cols]
        ncols = coarse.nfree
    else:
        ncols = coarse.ndofs
    rows = np.repeat(np.arange(len(pts))[:, None], cols.shape[1], axis=1)
    keep = (cols >= 0) & (np.abs(vals) >= DROP_TOL)
    P = sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(len(pts), ncols))
    P.sort_indices()
    return P


def galerkin(A: sp.csr_matrix, P: sp.csr_matrix) -> sp.csr_matrix:
    """A_{l+1} = P^T A P, with a unit diagonal on coarse DoFs that P never reaches."""
    Ac = (P.T @ (A @ P)).tocsr()
    unreached = np.flatnonzero(np.diff(P.tocsc().indptr) == 0)
    if len(unreached):
        Ac = (Ac + sp.csr_matrix((np.ones(len(unreached)), (unreached, unreached)), shape=Ac.shape)).tocsr()
    Ac.sort_indices()
    return Ac
