"""Linear elasticity with vector Lagrange P1/P2 elements (oracle; test infrastructure only).

Sec. 6.3 of the paper: -div sigma(u) = f in Omega with the isotropic law
sigma(u) = 2 mu eps(u) + lambda tr(eps(u)) I, eps(u) = (grad u + grad u^T) / 2, and the
Lame parameters mu = E / (2 (1 + nu)), lambda = E nu / ((1 + nu) (1 - 2 nu)); u = 0 on
Gamma_1, sigma n = t on Gamma_2 and sigma n = 0 on the rest of the boundary.

Weak form, for trial u = phi_b e_j and test v = phi_a e_i on a cell:
    int  mu (grad phi_a . grad phi_b) delta_ij + mu d_j phi_a d_i phi_b
       + lambda d_i phi_a d_j phi_b,
integrated exactly (degree 2(p-1) on affine cells) with the rule of ``quadrature``.

Numbering (the library's, implemented independently on both sides): vector DoF
dim*k + c is component c of scalar DoF k (components interleaved, node-major); the free
vector DoFs are the free scalar DoFs of ``fem.dof_map`` each expanded to its dim
components, in order (a Dirichlet node fixes every component). Transfer acts
componentwise: P_vec = P (x) I_dim, with P the scalar interpolation of ``transfer``.

Pinned by tests/test_oracle_elasticity.py: symmetry; rigid-body modes (translations and
infinitesimal rotations) in the kernel of the pre-Dirichlet operator; the energy of
affine displacements against the closed form vol (2 mu eps:eps + lambda tr(eps)^2) for a
dilatation and a shear (which separates the mu and lambda terms); the traction load's
total force and first moment; O(h^2) / O(h^3) L2 convergence of a manufactured solution
whose body force is derived symbolically.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from .quadrature import barycentric_of_reference, simplex_rule


def lame(E: float, nu: float):
    """(mu, lambda) from Young's modulus and Poisson's ratio (Sec. 6.3)."""
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def element_elasticity(coords: np.ndarray, cells: np.ndarray, degree: int, mu: float, lam: float) -> np.ndarray:
    """[nc, nloc*dim, nloc*dim] element matrices, local index a*dim + i (node a, component i)."""
    dim = coords.shape[1]
    cells = cells.astype(np.int64)
    pts, w = simplex_rule(dim, max(0, 2 * (degree - 1)))
    lq = barycentric_of_reference(pts)
    G = fem.barycentric_gradients(coords, cells)
    _, detJ = fem.jacobians(coords, cells)
    dphi = fem.basis_gradients(lq, G, degree, dim)                     # [nc, nq, nloc, dim]
    M = np.einsum("q,cqai,cqbj,c->caibj", w, dphi, dphi, detJ)         # int d_i phi_a d_j phi_b
    S = np.einsum("caibi->cab", M)                                     # int grad phi_a . grad phi_b
    eye = np.eye(dim)
    K = (mu * S[:, :, None, :, None] * eye[None, None, :, None, :]
         + mu * np.einsum("cajbi->caibj", M)
         + lam * M)
    nc, nloc = dphi.shape[0], dphi.shape[2]
    return K.reshape(nc, nloc * dim, nloc * dim)


def vector_cell_dofs(dm: fem.DofMap) -> np.ndarray:
    d = dm.dim
    return (dm.cell_dofs[:, :, None] * d + np.arange(d)[None, None, :]).reshape(dm.cell_dofs.shape[0], -1)


def free_vector_dofs(dm: fem.DofMap) -> np.ndarray:
    d = dm.dim
    return (dm.free[:, None] * d + np.arange(d)[None, :]).ravel()


def assemble_full(coords, cells, dm: fem.DofMap, mu: float, lam: float) -> sp.csr_matrix:
    """The operator over all vector DoFs (before Dirichlet elimination)."""
    Ke = element_elasticity(coords, cells, dm.degree, mu, lam)
    cd = vector_cell_dofs(dm)
    nloc = cd.shape[1]
    rows = np.repeat(cd, nloc, axis=1).ravel()
    cols = np.tile(cd, (1, nloc)).ravel()
    n = dm.ndofs * dm.dim
    A = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def restrict_free(A: sp.csr_matrix, dm: fem.DofMap) -> sp.csr_matrix:
    f = free_vector_dofs(dm)
    Af = A[f][:, f].tocsr()
    Af.sort_indices()
    return Af


def expand_patches(patches, dim: int):
    """Scalar free-DoF patches -> the vector DoFs of their nodes (ascending)."""
    return [(np.asarray(p, dtype=np.int64)[:, None] * dim + np.arange(dim)[None, :]).ravel() for p in patches]


def vector_prolongation(P: sp.csr_matrix, dim: int) -> sp.csr_matrix:
    Pv = sp.kron(P, sp.identity(dim, format="csr"), format="csr")
    Pv.sort_indices()
    return Pv


def traction_load_full(coords, cells, dm: fem.DofMap, t, axis: int, value: float, tol: float = 1e-12) -> np.ndarray:
    """b = int_{Gamma_2} t . v over the boundary facets lying in the plane x_axis = value
    (every vertex within tol of it), over all vector DoFs."""
    dim = coords.shape[1]
    t = np.asarray(t, dtype=np.float64)
    bf = fem.boundary_facets(cells.astype(np.int64))
    on = np.all(np.abs(coords[bf][:, :, axis] - value) <= tol, axis=1)
    bf = bf[on]
    b = np.zeros(dm.ndofs * dim)
    if len(bf) == 0:
        return b
    fd = dim - 1
    pts, w = simplex_rule(fd, dm.degree)
    lq = barycentric_of_reference(pts)
    phi = fem.basis_values(lq, dm.degree, fd)                          # [nq, nloc_facet]
    ref = np.einsum("q,qi->i", w, phi)                                 # reference-facet integrals
    edge_id = {(int(a), int(c)): k for k, (a, c) in enumerate(dm.edges)} if dm.degree == 2 else {}
    nv = coords.shape[0]
    fact = 1.0
    for k in range(2, fd + 1):
        fact *= k
    for f in bf:
        X = coords[f]
        J = (X[1:] - X[0]).T                                           # [dim, fd]
        area = np.sqrt(np.linalg.det(J.T @ J)) / fact                  # facet measure
        dofs = list(f)
        if dm.degree == 2:
            dofs += [nv + edge_id[(int(min(f[a], f[c])), int(max(f[a], f[c])))] for a, c in fem.LOCAL_EDGES[fd]]
        for loc, g in enumerate(dofs):
            b[g * dim:(g + 1) * dim] += t * (fact * area * ref[loc])
    return b
