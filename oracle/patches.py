"""Low-quality regions and local-correction DoF sets (oracle; test infrastructure only).

Sec. 4.4, Eq. (identify): Omega_b = {K : gamma(K) < threshold} (0.1 in the paper), and
Omega_B = Omega_b plus every cell sharing a vertex with it (one layer; ``layers`` repeats
the extension). Sec. 4.1: the subdomains Omega_B^d are disjoint and B_d is the set of
DoFs on the closure of Omega_B^d. Reading: the subdomains are the vertex-connected
components of Omega_B (touching regions merge, which keeps the closures disjoint), B_d
holds the free DoFs of the component's cells in ascending free numbering, and patches
are ordered by their smallest DoF. Dirichlet DoFs are excluded (the local problem is a
Dirichlet problem on the patch, Sec. 4.1).

Pinned by tests/test_oracle_smoother.py (patches are disjoint, cover the flagged cells'
DoFs, and A[B_d, B_d] is SPD) and brute-force recomputation on tiny meshes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components


def extend_region(cells: np.ndarray, region: np.ndarray, nv: int, layers: int) -> np.ndarray:
    region = region.copy()
    for _ in range(layers):
        vmark = np.zeros(nv, dtype=bool)
        vmark[cells[region].ravel()] = True
        region = vmark[cells].any(axis=1)
    return region


def local_patches(cells: np.ndarray, gamma: np.ndarray, threshold: float, layers: int,
                  nv: int, cell_dofs: np.ndarray, free_index: np.ndarray) -> list[np.ndarray]:
    bad = gamma < threshold
    if not bad.any():
        return []
    region = extend_region(cells, bad, nv, layers)
    rc = np.flatnonzero(region)
    # bipartite graph cells <-> vertices; components give vertex-connected cell groups
    d1 = cells.shape[1]
    rows = np.repeat(np.arange(len(rc)), d1)
    cols = len(rc) + cells[rc].ravel()
    g = sp.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(len(rc) + nv, len(rc) + nv))
    _, labels = connected_components(g, directed=False)
    comp = labels[:len(rc)]
    patches = []
    for c in np.unique(comp):
        dofs = np.unique(cell_dofs[rc[comp == c]].ravel())
        fd = free_index[dofs]
        fd = np.sort(fd[fd >= 0])
        if len(fd):
            patches.append(fd)
    patches.sort(key=lambda p: int(p[0]))
    return patches
