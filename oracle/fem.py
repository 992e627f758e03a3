"""Lagrange P1/P2 finite elements on simplices (oracle; test infrastructure only).

Follows the paper's discretisation (Sec. 2: A_1 u_1 = b_1 from continuous Lagrange
elements; Sec. 6.1: the Poisson problem -lap u = f with Dirichlet data g = 0 on Gamma_D).

Conventions (the library's numbering, which both sides implement independently):
  * DoFs on a mesh: vertices 0..nv-1 in input order, then (P2) one DoF per edge, edges
    ordered lexicographically by their sorted vertex pair (min, max);
  * Dirichlet DoFs: vertices on a boundary facet (a facet of exactly one cell) that the
    optional vertex mask allows; an edge DoF is Dirichlet when the edge lies in a boundary
    facet and both of its vertices are Dirichlet;
  * free DoFs keep the order above with Dirichlet DoFs removed.
  * local DoF order in a cell: its vertices, then edges (0,1),(0,2),(1,2) in 2D and
    (0,1),(0,2),(0,3),(1,2),(1,3),(2,3) in 3D.

Element integrals use the collapsed Gauss rule of ``quadrature`` (exact for the
polynomial degrees involved on affine cells).

Pinned by tests/test_oracle_fem.py: symmetry, zero row sums of the pre-Dirichlet
stiffness (constants are in the kernel), the 5-point stencil on the unjittered P1 grid,
the P2 reference-element stiffness against exact rational integration (sympy), the
constant-load closed forms, and O(h^2)/O(h^3) L2 convergence of a manufactured solution.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .quadrature import barycentric_of_reference, simplex_rule

LOCAL_EDGES = {1: [(0, 1)],
               2: [(0, 1), (0, 2), (1, 2)],
               3: [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]}


@dataclass
class DofMap:
    degree: int
    dim: int
    cell_dofs: np.ndarray      # [nc, nloc] global DoF ids (all DoFs)
    points: np.ndarray         # [ndofs, dim] interpolation points
    edges: np.ndarray          # [ne, 2] sorted vertex pairs (P2), else empty
    dirichlet: np.ndarray      # [ndofs] bool
    free: np.ndarray           # [nfree] global ids of free DoFs, ascending
    free_index: np.ndarray     # [ndofs] free number or -1

    @property
    def ndofs(self) -> int:
        return int(self.points.shape[0])

    @property
    def nfree(self) -> int:
        return int(self.free.shape[0])


def boundary_facets(cells: np.ndarray) -> np.ndarray:
    """Facets (sorted vertex tuples) that belong to exactly one cell."""
    d1 = cells.shape[1]
    facets = np.concatenate([np.delete(cells, i, axis=1) for i in range(d1)], axis=0)
    facets = np.sort(facets, axis=1)
    uniq, counts = np.unique(facets, axis=0, return_counts=True)
    return uniq[counts == 1]


def dof_map(coords: np.ndarray, cells: np.ndarray, degree: int,
            dirichlet_vertex_mask: np.ndarray | None = None) -> DofMap:
    nv, dim = coords.shape
    nc = cells.shape[0]
    cells = cells.astype(np.int64)
    bf = boundary_facets(cells)
    on_bnd = np.zeros(nv, dtype=bool)
    on_bnd[bf.ravel()] = True
    vdir = on_bnd if dirichlet_vertex_mask is None else (on_bnd & dirichlet_vertex_mask.astype(bool))
    if degree == 1:
        return _finish(degree, dim, cells, coords, np.zeros((0, 2), np.int64), vdir)
    if degree != 2:
        raise ValueError("degree must be 1 or 2")
    le = LOCAL_EDGES[dim]
    e = np.stack([np.sort(cells[:, [a, b]], axis=1) for a, b in le], axis=1)
    uniq, inv = np.unique(e.reshape(-1, 2), axis=0, return_inverse=True)
    inv = inv.reshape(nc, len(le))
    cell_dofs = np.concatenate([cells, nv + inv], axis=1)
    points = np.concatenate([coords, 0.5 * (coords[uniq[:, 0]] + coords[uniq[:, 1]])], axis=0)
    # edges lying in a boundary facet
    bedges = set()
    for f in bf:
        for a in range(len(f)):
            for b in range(a + 1, len(f)):
                bedges.add((int(f[a]), int(f[b])))
    edir = np.array([(int(a), int(b)) in bedges and vdir[a] and vdir[b] for a, b in uniq], dtype=bool)
    dirichlet = np.concatenate([vdir, edir])
    free = np.flatnonzero(~dirichlet)
    free_index = -np.ones(len(dirichlet), dtype=np.int64)
    free_index[free] = np.arange(len(free))
    return DofMap(degree, dim, cell_dofs, points, uniq, dirichlet, free, free_index)


def _finish(degree, dim, cells, coords, edges, vdir):
    free = np.flatnonzero(~vdir)
    free_index = -np.ones(len(vdir), dtype=np.int64)
    free_index[free] = np.arange(len(free))
    return DofMap(degree, dim, cells.copy(), coords.copy(), edges, vdir.copy(), free, free_index)


def jacobians(coords: np.ndarray, cells: np.ndarray):
    """J [nc, dim, dim] with columns x_i - x_0, and |det J|."""
    x0 = coords[cells[:, 0]]
    J = np.stack([coords[cells[:, i]] - x0 for i in range(1, cells.shape[1])], axis=2)
    return J, np.abs(np.linalg.det(J))


def barycentric_gradients(coords: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """[nc, dim+1, dim]: gradient of each barycentric coordinate on each cell."""
    J, _ = jacobians(coords, cells)
    dim = coords.shape[1]
    gref = np.concatenate([-np.ones((1, dim)), np.eye(dim)], axis=0)     # d lambda / d xi
    Jinv = np.linalg.inv(J)                                              # d xi / d x
    return np.einsum("ak,ckx->cax", gref, Jinv)


def basis_values(lam: np.ndarray, degree: int, dim: int) -> np.ndarray:
    """Basis values at barycentric points lam [..., dim+1] -> [..., nloc]."""
    if degree == 1:
        return lam.copy()
    vert = lam * (2.0 * lam - 1.0)
    edge = np.stack([4.0 * lam[..., a] * lam[..., b] for a, b in LOCAL_EDGES[dim]], axis=-1)
    return np.concatenate([vert, edge], axis=-1)


def basis_gradients(lam: np.ndarray, G: np.ndarray, degree: int, dim: int) -> np.ndarray:
    """Gradients at barycentric points lam [nq, dim+1] on cells with barycentric
    gradients G [nc, dim+1, dim] -> [nc, nq, nloc, dim]."""
    nq = lam.shape[0]
    if degree == 1:
        return np.broadcast_to(G[:, None, :, :], (G.shape[0], nq) + G.shape[1:]).copy()
    vert = (4.0 * lam - 1.0)[None, :, :, None] * G[:, None, :, :]
    edges = []
    for a, b in LOCAL_EDGES[dim]:
        ga = G[:, None, a, :]
        gb = G[:, None, b, :]
        edges.append(4.0 * (lam[None, :, b, None] * ga + lam[None, :, a, None] * gb))
    return np.concatenate([vert, np.stack(edges, axis=2)], axis=2)


def element_stiffness(coords: np.ndarray, cells: np.ndarray, degree: int) -> np.ndarray:
    """[nc, nloc, nloc] int_K grad phi_i . grad phi_j by exact quadrature."""
    dim = coords.shape[1]
    pts, w = simplex_rule(dim, max(0, 2 * (degree - 1)))
    lam = barycentric_of_reference(pts)
    G = barycentric_gradients(coords, cells.astype(np.int64))
    _, detJ = jacobians(coords, cells.astype(np.int64))
    dphi = basis_gradients(lam, G, degree, dim)                        # [nc, nq, nloc, dim]
    return np.einsum("q,cqix,cqjx,c->cij", w, dphi, dphi, detJ)


def element_mass(coords: np.ndarray, cells: np.ndarray, degree: int) -> np.ndarray:
    dim = coords.shape[1]
    pts, w = simplex_rule(dim, 2 * degree)
    lam = barycentric_of_reference(pts)
    _, detJ = jacobians(coords, cells.astype(np.int64))
    phi = basis_values(lam, degree, dim)                               # [nq, nloc]
    return np.einsum("q,qi,qj,c->cij", w, phi, phi, detJ)


def scatter_matrix(dm: DofMap, Ke: np.ndarray) -> sp.csr_matrix:
    """Sum element matrices into the full (all-DoF) sparse matrix."""
    nloc = dm.cell_dofs.shape[1]
    rows = np.repeat(dm.cell_dofs, nloc, axis=1).ravel()
    cols = np.tile(dm.cell_dofs, (1, nloc)).ravel()
    A = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(dm.ndofs, dm.ndofs)).tocsr()
    A.sum_duplicates()
    return A


def assemble_stiffness_full(coords, cells, dm: DofMap) -> sp.csr_matrix:
    return scatter_matrix(dm, element_stiffness(coords, cells, dm.degree))


def restrict_free(A: sp.csr_matrix, dm: DofMap) -> sp.csr_matrix:
    """Dirichlet elimination with g = 0: keep the free rows and columns."""
    Af = A[dm.free][:, dm.free].tocsr()
    Af.sort_indices()
    return Af


def load_vector_full(coords, cells, dm: DofMap, f, qdegree: int | None = None) -> np.ndarray:
    """b_i = int f phi_i over all DoFs; f(x [npts, dim]) -> [npts] (or a float constant)."""
    dim = coords.shape[1]
    if qdegree is None:
        qdegree = dm.degree + (0 if np.isscalar(f) else 6)
    pts, w = simplex_rule(dim, qdegree)
    lam = barycentric_of_reference(pts)
    cells64 = cells.astype(np.int64)
    _, detJ = jacobians(coords, cells64)
    phi = basis_values(lam, dm.degree, dim)                            # [nq, nloc]
    if np.isscalar(f):
        fq = np.full((cells.shape[0], len(w)), float(f))
    else:
        xq = np.einsum("qa,cax->cqx", lam, coords[cells64])
        fq = f(xq.reshape(-1, dim)).reshape(cells.shape[0], len(w))
    be = np.einsum("q,cq,qi,c->ci", w, fq, phi, detJ)
    b = np.zeros(dm.ndofs)
    np.add.at(b, dm.cell_dofs.ravel(), be.ravel())
    return b


def interpolate(dm: DofMap, u) -> np.ndarray:
    """Nodal interpolation of u at all DoF points."""
    return u(dm.points)


def l2_error(coords, cells, dm: DofMap, u_all: np.ndarray, u_exact, qdegree: int = 10) -> float:
    """|| u_h - u ||_{L2} with u_h given by all-DoF coefficients."""
    dim = coords.shape[1]
    pts, w = simplex_rule(dim, qdegree)
    lam = barycentric_of_reference(pts)
    cells64 = cells.astype(np.int64)
    _, detJ = jacobians(coords, cells64)
    phi = basis_values(lam, dm.degree, dim)
    uh = np.einsum("qi,ci->cq", phi, u_all[dm.cell_dofs])
    xq = np.einsum("qa,cax->cqx", lam, coords[cells64])
    ue = u_exact(xq.reshape(-1, dim)).reshape(uh.shape)
    return float(np.sqrt(np.einsum("q,cq,c->", w, (uh - ue) ** 2, detJ)))
