"""Seeded synthetic inputs: simplex meshes of the unit square / unit cube, and right-hand sides.

The paper's Gmsh meshes are not available, so its workloads (Sec. 6: unstructured,
non-nested meshes of the unit square and unit cube whose levels are generated
independently, with some vertices displaced to create low-quality cells) are stood in
for by structured simplex grids with seeded interior jitter and seeded vertex moves.

This module is shared by the oracle, the tests and the benchmark. It holds geometry
generation only (grids, jitter, vertex displacement and an orientation check that keeps
every cell valid); none of the finite-element or multigrid arithmetic lives here.

Recipe (all seeds derive from ``(seed, level)``):
  * grid: an N^dim grid of squares split into 2 triangles along the (i,j)->(i+1,j+1)
    diagonal, or of cubes split into the 6 Kuhn tetrahedra around the main diagonal;
  * jitter: every interior vertex moves by U(-a h, a h) per coordinate (a = 0.2 in 2D,
    0.15 in 3D); boundary vertices stay fixed, so all levels share the boundary; a move
    that would invert a cell is undone;
  * low-quality clusters: a cluster picks a random interior centre vertex and moves
    vertices within two vertex rings of it. A "cap" move puts a vertex at distance
    ``dist`` above the centroid of the opposite facet of one of its cells (a flattened
    triangle, or in 3D a cap/sliver tetrahedron); a "needle" move (2D) puts it at
    distance ``dist`` from another vertex of that cell along their common edge. ``dist``
    is ``eps*h`` or ``h/AR`` with AR log-uniform in a range. A move is redrawn if any cell
    around the vertex would invert, and moved vertices never share a cell.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh", "structured_mesh", "jitter_mesh", "degrade_mesh", "signed_volumes",
    "hierarchy_meshes", "config_c1", "config_c2", "config_c3", "config_c4", "lattice_mesh", "config_lattice",
    "dumbbell_mesh", "config_dumbbell",
    "serving_request", "uniform_rhs", "CONFIGS",
]


@dataclass
class Mesh:
    """A simplicial mesh: ``coords`` [nv, dim] float64 and ``cells`` [nc, dim+1] int32."""
    coords: np.ndarray
    cells: np.ndarray
    n: int = 0                      # grid squares/cubes per unit length
    moves: list = field(default_factory=list)   # (vertex, kind, dist/h) per degrading move
    boundary: np.ndarray | None = None  # [nv] bool boundary vertices (None: unit square/cube)

    @property
    def dim(self) -> int:
        return int(self.coords.shape[1])

    @property
    def nv(self) -> int:
        return int(self.coords.shape[0])

    @property
    def nc(self) -> int:
        return int(self.cells.shape[0])

    @property
    def h(self) -> float:
        return 1.0 / self.n


def structured_mesh(dim: int, n: int) -> Mesh:
    """Unit square (2 triangles per square) or unit cube (6 Kuhn tets per cube), positively oriented."""
    if dim == 2:
        j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
        coords = np.stack([i.ravel() / n, j.ravel() / n], axis=1).astype(np.float64)
        vid = lambda a, b: b * (n + 1) + a
        jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        ii, jj = ii.ravel(), jj.ravel()
        v00, v10 = vid(ii, jj), vid(ii + 1, jj)
        v01, v11 = vid(ii, jj + 1), vid(ii + 1, jj + 1)
        t1 = np.stack([v00, v10, v11], axis=1)
        t2 = np.stack([v00, v11, v01], axis=1)
        cells = np.stack([t1, t2], axis=1).reshape(-1, 3)
    elif dim == 3:
        k, j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
        coords = np.stack([i.ravel() / n, j.ravel() / n, k.ravel() / n], axis=1).astype(np.float64)
        vid = lambda a, b, c: (c * (n + 1) + b) * (n + 1) + a
        kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        base = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
        tets = []
        for perm in itertools.permutations(range(3)):
            p = base.copy()
            path = [vid(p[:, 0], p[:, 1], p[:, 2])]
            for ax in perm:
                p[:, ax] += 1
                path.append(vid(p[:, 0], p[:, 1], p[:, 2]))
            t = np.stack(path, axis=1)
            # the Kuhn tet along `perm` has orientation sign(perm); swap two vertices if odd
            inv = sum(1 for a, b in itertools.combinations(perm, 2) if a > b)
            if inv % 2 == 1:
                t = t[:, [0, 1, 3, 2]]
            tets.append(t)
        cells = np.stack(tets, axis=1).reshape(-1, 4)
    else:
        raise ValueError("dim must be 2 or 3")
    return Mesh(coords=coords, cells=cells.astype(np.int32), n=n)


def boundary_vertices(mesh: Mesh) -> np.ndarray:
    """Vertices on the boundary of the unit square/cube (exact grid coordinates), or the
    mesh's own boundary mask when it has one."""
    if mesh.boundary is not None:
        return mesh.boundary
    n = mesh.n
    idx = np.rint(mesh.coords * n).astype(np.int64)
    return np.any((idx == 0) | (idx == n), axis=1)


def signed_volumes(coords: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """det of the edge vectors (v_i - v_0); positive for a positively oriented cell."""
    x0 = coords[cells[:, 0]]
    e = np.stack([coords[cells[:, i]] - x0 for i in range(1, cells.shape[1])], axis=1)
    return np.linalg.det(e)


def jitter_mesh(mesh: Mesh, amp: float, rng: np.random.Generator) -> Mesh:
    """Move interior vertices by U(-amp h, amp h) per coordinate; undo moves that invert cells."""
    bnd = boundary_vertices(mesh)
    delta = rng.uniform(-amp * mesh.h, amp * mesh.h, size=mesh.coords.shape)
    delta[bnd] = 0.0
    new = mesh.coords + delta
    for _ in range(64):
        bad = signed_volumes(new, mesh.cells) <= 0.0
        if not bad.any():
            break
        reset = np.unique(mesh.cells[bad].ravel())
        new[reset] = mesh.coords[reset]
    return Mesh(coords=new, cells=mesh.cells, n=mesh.n, boundary=mesh.boundary)


def _vertex_star(cells: np.ndarray, nv: int):
    flat = cells.ravel()
    order = np.argsort(flat, kind="stable")
    owners = (order // cells.shape[1]).astype(np.int64)
    ptr = np.zeros(nv + 1, dtype=np.int64)
    np.cumsum(np.bincount(flat, minlength=nv), out=ptr[1:])
    return ptr, owners


def _facet_normal(pts: np.ndarray) -> np.ndarray:
    """Unit normal of a facet given by its dim vertices (edge in 2D, triangle in 3D)."""
    if pts.shape[0] == 2:
        t = pts[1] - pts[0]
        nrm = np.array([-t[1], t[0]])
    else:
        nrm = np.cross(pts[1] - pts[0], pts[2] - pts[0])
    return nrm / np.linalg.norm(nrm)


def degrade_mesh(mesh: Mesh, rng: np.random.Generator, n_clusters: int,
                 moves_per_cluster=(1, 1), kinds=("cap",), eps: float | None = 1e-3,
                 ar_range=(1e2, 1e4), rings: int = 2, center=None) -> Mesh:
    """Create ``n_clusters`` clusters of low-quality cells by seeded vertex moves (see module doc)."""
    coords = mesh.coords.copy()
    cells = mesh.cells
    nv, dim = coords.shape
    bnd = boundary_vertices(mesh)
    ptr, star = _vertex_star(cells, nv)
    blocked = np.zeros(nv, dtype=bool)
    interior = np.flatnonzero(~bnd)
    h = mesh.h
    moves = []
    if len(interior) == 0:
        n_clusters = 0
    for c in range(n_clusters):
        if center is not None and c == 0:
            ctr = int(center)
        else:
            ctr = int(rng.choice(interior))
        ring = {ctr}
        frontier = {ctr}
        for _ in range(rings):
            nxt = set()
            for v in frontier:
                nxt.update(cells[star[ptr[v]:ptr[v + 1]]].ravel().tolist())
            frontier = nxt - ring
            ring |= nxt
        cand = np.array(sorted(v for v in ring if not bnd[v]), dtype=np.int64)
        rng.shuffle(cand)
        if center is not None and c == 0:
            cand = np.concatenate([[ctr], cand[cand != ctr]])
        target = int(rng.integers(moves_per_cluster[0], moves_per_cluster[1] + 1))
        made = 0
        for v in cand:
            if made >= target:
                break
            if blocked[v]:
                continue
            vstar = star[ptr[v]:ptr[v + 1]]
            for _attempt in range(8):
                k = int(rng.choice(vstar))
                kind = kinds[int(rng.integers(len(kinds)))]
                if eps is not None:
                    dist = eps * h
                else:
                    lo, hi = np.log(ar_range[0]), np.log(ar_range[1])
                    dist = h / float(np.exp(rng.uniform(lo, hi)))
                others = [int(u) for u in cells[k] if u != v]
                if kind == "cap":
                    pts = coords[others]
                    nrm = _facet_normal(pts)
                    cen = pts.mean(axis=0)
                    if np.dot(coords[v] - cen, nrm) < 0:
                        nrm = -nrm
                    pos = cen + dist * nrm
                elif kind == "needle":
                    a = others[int(rng.integers(len(others)))]
                    u = coords[v] - coords[a]
                    pos = coords[a] + dist * u / np.linalg.norm(u)
                else:
                    raise ValueError(kind)
                old = coords[v].copy()
                coords[v] = pos
                if np.all(signed_volumes(coords, cells[vstar]) > 0.0):
                    moves.append((int(v), kind, dist / h))
                    blocked[np.unique(cells[vstar].ravel())] = True
                    made += 1
                    break
                coords[v] = old
    return Mesh(coords=coords, cells=cells, n=mesh.n, moves=moves, boundary=mesh.boundary)


def hierarchy_meshes(dim: int, n_fine: int, levels: int, amp: float, seed: int,
                     cluster_levels=(), n_clusters: int = 0, **degrade_kw) -> list[Mesh]:
    """Independently generated levels n_fine, n_fine/2, ... (non-nested after jitter)."""
    out = []
    for lvl in range(levels):
        n = n_fine >> lvl
        if n < 1:
            raise ValueError("too many levels for this grid")
        rng = np.random.default_rng([seed, lvl])
        m = jitter_mesh(structured_mesh(dim, n), amp, rng)
        if lvl in cluster_levels and n_clusters > 0:
            m = degrade_mesh(m, rng, n_clusters, **degrade_kw)
        out.append(m)
    return out


def _central_vertex(dim: int, n: int) -> int:
    c = n // 2
    return c * (n + 1) + c if dim == 2 else (c * (n + 1) + c) * (n + 1) + c


def config_c1(seed: int = 1, clusters: bool = True) -> list[Mesh]:
    """2D P1 unit square, 64^2 -> 32^2 -> 16^2, one cluster of 4 flattened cells near the
    centre (four cap moves, each vertex 1e-3 h above its opposite edge: min angle ~0.1 deg)."""
    return hierarchy_meshes(2, 64, 3, 0.2, seed, cluster_levels=(0,) if clusters else (),
                            n_clusters=1, moves_per_cluster=(4, 4), kinds=("cap",), eps=1e-3,
                            center=_central_vertex(2, 64))


def config_c2(n_fine: int = 1024, levels: int = 6, seed: int = 2, n_clusters: int = 32,
              cluster_levels=None) -> list[Mesh]:
    """2D P2, clusters of 2-8 flattened/needle cells (AR 1e2-1e4) on fine + intermediate levels."""
    if cluster_levels is None:
        cluster_levels = tuple(range(levels - 1))
    return hierarchy_meshes(2, n_fine, levels, 0.2, seed, cluster_levels=cluster_levels,
                            n_clusters=n_clusters, moves_per_cluster=(2, 8),
                            kinds=("cap", "needle"), eps=None, ar_range=(1e2, 1e4))


def config_c3(n_fine: int = 128, levels: int = 5, seed: int = 3, n_clusters: int = 64,
              cluster_levels=None) -> list[Mesh]:
    """3D P1 unit cube (Kuhn tets), cap slivers at 1e-3 h on the fine and 2nd-coarsest level."""
    if cluster_levels is None:
        cluster_levels = (0, levels - 2)
    return hierarchy_meshes(3, n_fine, levels, 0.15, seed, cluster_levels=cluster_levels,
                            n_clusters=n_clusters, moves_per_cluster=(1, 1), kinds=("cap",),
                            eps=1e-3)


def config_c4(n_fine: int = 64, levels: int = 4, seed: int = 4, n_clusters: int = 256,
              cluster_levels=(0,), moves_per_cluster=(1, 4)) -> list[Mesh]:
    """3D P2 unit cube, 256 clusters of 1-4 cap slivers within two rings on the fine level;
    touching clusters merge into uneven patches (about 100-2000 P2 DoFs)."""
    return hierarchy_meshes(3, n_fine, levels, 0.15, seed, cluster_levels=cluster_levels,
                            n_clusters=n_clusters, moves_per_cluster=moves_per_cluster,
                            kinds=("cap",), eps=1e-3, rings=2)


def lattice_mesh(n: int, size: float = 6.0, bar: float = 1.0) -> Mesh:
    """The truss-like lattice of Sec. 6.3: the cube [0, size]^3 minus three orthogonal square
    channels [bar, size - bar]^2 through it (a cube frame of 12 bars of cross-section
    bar x bar), meshed by 6 Kuhn tetrahedra per grid cube of side 1/n; unused vertices are
    dropped (order kept) and the boundary mask marks the vertices of boundary facets."""
    N = int(round(size * n))
    m = structured_mesh(3, N)
    coords = m.coords * size
    cen = coords[m.cells].mean(axis=1)
    inside = (cen > bar) & (cen < size - bar)
    keep = inside.sum(axis=1) < 2
    cells = m.cells[keep]
    used = np.zeros(m.nv, dtype=bool)
    used[cells.ravel()] = True
    new_id = -np.ones(m.nv, dtype=np.int64)
    new_id[used] = np.arange(int(used.sum()))
    cells = new_id[cells].astype(np.int32)
    coords = coords[used]
    facets = np.sort(np.concatenate([np.delete(cells, i, axis=1) for i in range(4)], axis=0), axis=1)
    uniq, cnt = np.unique(facets, axis=0, return_counts=True)
    bnd = np.zeros(coords.shape[0], dtype=bool)
    bnd[uniq[cnt == 1].ravel()] = True
    return Mesh(coords=coords, cells=cells, n=n, boundary=bnd)


def config_lattice(ns=(13, 6, 3, 2), seed: int = 5, n_clusters: int = 16, cluster_levels=None,
                   eps: float = 1e-4, amp: float = 0.15):
    """Elasticity workload of Sec. 6.3 (four levels of the lattice, generated independently):
    interior vertices jittered U(+-amp h); ``n_clusters`` sliver clusters (1-3 cap moves at
    eps h) on each level in ``cluster_levels`` (default all: Case A; all but the finest:
    Case B). Returns (meshes, Dirichlet vertex masks: the clamped face x = 0)."""
    if cluster_levels is None:
        cluster_levels = tuple(range(len(ns)))
    meshes, masks = [], []
    for lvl, n in enumerate(ns):
        rng = np.random.default_rng([seed, lvl])
        m = jitter_mesh(lattice_mesh(n), amp, rng)
        if lvl in cluster_levels and n_clusters > 0:
            m = degrade_mesh(m, rng, n_clusters, moves_per_cluster=(1, 3), kinds=("cap",), eps=eps)
        meshes.append(m)
        masks.append(np.abs(m.coords[:, 0]) <= 1e-12)
    return meshes, masks


def _box_union_mesh(n: int, extent, boxes) -> Mesh:
    """Kuhn-tetrahedron mesh (grid spacing 1/n) of the union of axis-aligned boxes inside
    [0, extent]^3: a grid cube is kept when its centre lies in some box; unused vertices are
    dropped (order kept) and the boundary mask marks the vertices of boundary facets."""
    N = [int(round(e * n)) for e in extent]
    M = max(N)
    m = structured_mesh(3, M)
    coords = m.coords * (M / n)
    cen = coords[m.cells].mean(axis=1)
    keep = np.zeros(m.nc, dtype=bool)
    for lo, hi in boxes:
        keep |= np.all((cen > np.asarray(lo)) & (cen < np.asarray(hi)), axis=1)
    cells = m.cells[keep]
    used = np.zeros(m.nv, dtype=bool)
    used[cells.ravel()] = True
    new_id = -np.ones(m.nv, dtype=np.int64)
    new_id[used] = np.arange(int(used.sum()))
    cells = new_id[cells].astype(np.int32)
    coords = coords[used]
    facets = np.sort(np.concatenate([np.delete(cells, i, axis=1) for i in range(4)], axis=0), axis=1)
    uniq, cnt = np.unique(facets, axis=0, return_counts=True)
    bnd = np.zeros(coords.shape[0], dtype=bool)
    bnd[uniq[cnt == 1].ravel()] = True
    return Mesh(coords=coords, cells=cells, n=n, boundary=bnd)


# two 1 x 2 x 2 end blocks joined by three 4 x 0.5 x 0.5 bars (grid spacing must divide 0.5)
DUMBBELL_BOXES = [((0.0, 0.0, 0.0), (1.0, 2.0, 2.0)), ((5.0, 0.0, 0.0), (6.0, 2.0, 2.0)),
                  ((1.0, 0.0, 0.0), (5.0, 0.5, 0.5)), ((1.0, 1.5, 0.0), (5.0, 2.0, 0.5)),
                  ((1.0, 0.5, 1.5), (5.0, 1.0, 2.0))]


def dumbbell_mesh(n: int) -> Mesh:
    """A dumbbell-like structure in the spirit of Sec. 6.3 (the paper's has hexagonal ends):
    two end blocks joined by three slender bars, grid spacing 1/n (n even)."""
    if n % 2:
        raise ValueError("n must be even")
    return _box_union_mesh(n, (6.0, 2.0, 2.0), DUMBBELL_BOXES)


def config_dumbbell(ns=(24, 8, 4, 2), seed: int = 6, n_clusters: int = 16, cluster_levels=None,
                    eps: float = 1e-4, amp: float = 0.15):
    """Elasticity workload shaped like the paper's dumbbell example: four independently
    generated levels, interior jitter U(+-amp h), ``n_clusters`` sliver clusters (1-3 cap
    moves at eps h) on each level in ``cluster_levels`` (default all: Case A). Returns
    (meshes, Dirichlet vertex masks: the clamped face x = 0)."""
    if cluster_levels is None:
        cluster_levels = tuple(range(len(ns)))
    meshes, masks = [], []
    for lvl, n in enumerate(ns):
        rng = np.random.default_rng([seed, lvl])
        m = jitter_mesh(dumbbell_mesh(n), amp, rng)
        if lvl in cluster_levels and n_clusters > 0:
            m = degrade_mesh(m, rng, n_clusters, moves_per_cluster=(1, 3), kinds=("cap",), eps=eps)
        meshes.append(m)
        masks.append(np.abs(m.coords[:, 0]) <= 1e-12)
    return meshes, masks


def serving_request(rng: np.random.Generator, seed: int):
    """One request of the mixed serving stream: (meshes, degree, label)."""
    kind = int(rng.integers(3))
    n_cl = int(rng.integers(0, 17))
    if kind < 2:
        n = int(2 ** rng.integers(5, 10))          # 32^2 .. 512^2
        degree = 1 + kind
        levels = max(2, int(np.log2(n)) - 3)
        meshes = hierarchy_meshes(2, n, levels, 0.2, seed, cluster_levels=tuple(range(levels - 1)),
                                  n_clusters=n_cl, moves_per_cluster=(1, 4),
                                  kinds=("cap", "needle"), eps=None, ar_range=(1e2, 1e4))
        return meshes, degree, f"2D P{degree} {n}^2 clusters={n_cl}"
    n = int(2 ** rng.integers(4, 7))               # 16^3 .. 64^3
    levels = max(2, int(np.log2(n)) - 2)
    meshes = hierarchy_meshes(3, n, levels, 0.15, seed, cluster_levels=(0,), n_clusters=n_cl,
                              moves_per_cluster=(1, 1), kinds=("cap",), eps=1e-3)
    return meshes, 1, f"3D P1 {n}^3 clusters={n_cl}"


def uniform_rhs(n: int, seed: int) -> np.ndarray:
    """Algebraic right-hand side, i.i.d. U[-1, 1] (float64)."""
    return np.random.default_rng([seed, 0xB]).uniform(-1.0, 1.0, size=n)


CONFIGS = {
    "c1": dict(dim=2, degree=1, make=config_c1, rtol=1e-10, rhs="f=1", layers=2),
    "c2": dict(dim=2, degree=2, make=config_c2, rtol=1e-8, rhs="uniform", layers=1),
    "c3": dict(dim=3, degree=1, make=config_c3, rtol=1e-8, rhs="uniform", layers=1),
    "c4": dict(dim=3, degree=2, make=config_c4, rtol=1e-8, rhs="uniform", layers=1),
}
