"""Level hierarchy of the non-nested multigrid method (oracle; test infrastructure only).

Builds, for meshes Omega_1 (finest) .. Omega_L (coarsest), per Sec. 2 and Sec. 6:
  * level 1: the Poisson stiffness on free DoFs (fem), level l+1: A_{l+1} = P_l^T A_l P_l;
  * P_l by interpolation at the fine DoF points (transfer), R_l = P_l^T;
  * gamma per cell, Omega_b / Omega_B and the patches B_d on every level (patches),
    with A^{[d]} = A_l[B_d, B_d] factored by dense Cholesky (smoother.LocalSolver);
  * lambda_max of D^{-1}A_l (adjusted per Sec. 5 by default), lambda_min = lmin_ratio
    lambda_max; the option ``lambda_override`` injects given values instead;
  * a dense Cholesky factor of the coarsest operator (the "direct solver" of Alg. 1),
    with the semi-definite reading of ``smoother.DirectSolver``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import eig as _eig
from . import elasticity as _elasticity
from . import fem, patches as _patches, quality, transfer
from . import smoother
from .smoother import DirectSolver, LocalSolver


@dataclass
class Level:
    A: sp.csr_matrix
    dinv: np.ndarray
    dm: fem.DofMap | None = None
    coords: np.ndarray | None = None
    cells: np.ndarray | None = None
    gamma: np.ndarray | None = None
    patches: list = field(default_factory=list)
    local: LocalSolver | None = None
    P: sp.csr_matrix | None = None      # level l+1 -> l
    R: sp.csr_matrix | None = None      # level l -> l+1
    lmax_unadj: float = 0.0
    lmax_adj: float = 0.0
    lmax: float = 0.0
    lmin: float = 0.0
    colour: np.ndarray | None = None    # greedy colouring (multicolour SGS)

    @property
    def n(self) -> int:
        return self.A.shape[0]


@dataclass
class Hierarchy:
    levels: list
    degree: int
    cheb_degree: int = 2
    nu: int = 1
    order: str = "sandwich"
    coarse: DirectSolver | None = None
    smoother_kind: str = "chebyshev"     # global smoother: "chebyshev" or "sgs"

    @property
    def L(self) -> int:
        return len(self.levels)


def build(meshes, degree: int, threshold: float = 0.1, layers: int = 1, adjusted: bool = True,
          lmin_ratio: float = 0.1, cheb_degree: int = 2, nu: int = 1, order: str = "sandwich",
          lambda_override=None, dirichlet_masks=None, local_levels=None,
          compute_eigs: bool = True, smoother_kind: str = "chebyshev", pde: str = "poisson",
          young: float = 6.9e10, poisson_ratio: float = 0.33) -> Hierarchy:
    """``pde``: "poisson" (Sec. 6.1-6.2) or "elasticity" (Sec. 6.3, vector DoFs numbered as
    in ``elasticity``; P acts componentwise and patches hold every component of their nodes)."""
    L = len(meshes)
    levels = []
    vec = pde == "elasticity"
    if pde not in ("poisson", "elasticity"):
        raise ValueError(pde)
    for l, m in enumerate(meshes):
        mask = None if dirichlet_masks is None else dirichlet_masks[l]
        dm = fem.dof_map(m.coords, m.cells, degree, mask)
        gamma = quality.radius_ratio(m.coords, m.cells)
        if l == 0:
            if vec:
                mu, lam = _elasticity.lame(young, poisson_ratio)
                A = _elasticity.restrict_free(_elasticity.assemble_full(m.coords, m.cells, dm, mu, lam), dm)
            else:
                A = fem.restrict_free(fem.assemble_stiffness_full(m.coords, m.cells, dm), dm)
        else:
            prev = levels[-1]
            prev.P = transfer.prolongation(prev.dm, m.coords, m.cells, dm)
            if vec:
                prev.P = _elasticity.vector_prolongation(prev.P, m.coords.shape[1])
            prev.R = prev.P.T.tocsr()
            prev.R.sort_indices()
            A = transfer.galerkin(prev.A, prev.P)
        lev = Level(A=A, dinv=1.0 / A.diagonal(), dm=dm, coords=m.coords, cells=m.cells, gamma=gamma)
        if local_levels is None or l in local_levels:
            lev.patches = _patches.local_patches(m.cells, gamma, threshold, layers, m.nv,
                                                 dm.cell_dofs, dm.free_index)
            if vec:
                lev.patches = _elasticity.expand_patches(lev.patches, m.coords.shape[1])
        levels.append(lev)
    for l, lev in enumerate(levels):
        lev.local = LocalSolver(lev.A, lev.patches)
        if l == L - 1:
            continue
        if smoother_kind == "sgs":
            lev.colour = smoother.greedy_colouring(lev.A)
            continue
        if lambda_override is not None:
            lev.lmax = float(lambda_override[l])
        elif compute_eigs:
            lev.lmax_unadj = _eig.lambda_max(lev.A)
            lev.lmax_adj = _eig.adjusted_lambda_max(lev.A, lev.patches) if lev.patches else lev.lmax_unadj
            lev.lmax = lev.lmax_adj if adjusted else lev.lmax_unadj
        lev.lmin = lmin_ratio * lev.lmax
    coarse = DirectSolver(levels[-1].A.toarray())
    return Hierarchy(levels=levels, degree=degree, cheb_degree=cheb_degree, nu=nu, order=order,
                     coarse=coarse, smoother_kind=smoother_kind)


def from_matrices(As, Ps, patches, lmax, cheb_degree=2, nu=1, order="sandwich", lmin_ratio=0.1):
    """Hierarchy from algebraic data: A_l (L), P_l (L-1, maps l+1 -> l), patches per level."""
    L = len(As)
    levels = []
    for l in range(L):
        lev = Level(A=As[l].tocsr(), dinv=1.0 / As[l].diagonal(), patches=list(patches[l]))
        if l < L - 1:
            lev.P = Ps[l].tocsr()
            lev.R = lev.P.T.tocsr()
            lev.lmax = float(lmax[l])
            lev.lmin = lmin_ratio * lev.lmax
        lev.local = LocalSolver(lev.A, lev.patches)
        levels.append(lev)
    coarse = DirectSolver(levels[-1].A.toarray())
    return Hierarchy(levels=levels, degree=0, cheb_degree=cheb_degree, nu=nu, order=order, coarse=coarse)
