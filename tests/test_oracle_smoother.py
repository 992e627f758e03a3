"""Pins for eigenvalue estimates, Chebyshev S_g, local correction S_c and S_gc (no GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import eig, fem, hierarchy, patches, quality, smoother
from paper_2402_12947_gb300 import inputs


def _level(seed=3, n=10, degree=1, clusters=True):
    m = inputs.jitter_mesh(inputs.structured_mesh(2, n), 0.2, np.random.default_rng(seed))
    if clusters:
        m = inputs.degrade_mesh(m, np.random.default_rng(seed + 1), 2, moves_per_cluster=(1, 2))
    dm = fem.dof_map(m.coords, m.cells, degree)
    A = fem.restrict_free(fem.assemble_stiffness_full(m.coords, m.cells, dm), dm)
    g = quality.radius_ratio(m.coords, m.cells)
    pt = patches.local_patches(m.cells, g, 0.1, 1, m.nv, dm.cell_dofs, dm.free_index)
    return m, dm, A, g, pt


def test_lambda_closed_form_1d_laplacian(monkeypatch):
    for n in (50, 400):
        A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
        exact = 1 + np.cos(np.pi / (n + 1))
        assert abs(eig.lambda_max(A) - exact) < 1e-12
        monkeypatch.setattr(eig, "DENSE_MAX", 10)
        assert abs(eig.lambda_max(A) - exact) < 1e-10
        monkeypatch.setattr(eig, "DENSE_MAX", 3000)


def test_lambda_dense_vs_lanczos_and_interlacing(monkeypatch):
    _, _, A, _, pt = _level(n=24, degree=2)
    assert pt
    dense = eig.lambda_max(A)
    dense_adj = eig.adjusted_lambda_max(A, pt)
    assert dense_adj <= dense + 1e-12
    monkeypatch.setattr(eig, "DENSE_MAX", 10)
    assert abs(eig.lambda_max(A) - dense) < 1e-9 * dense
    assert abs(eig.adjusted_lambda_max(A, pt) - dense_adj) < 1e-9 * dense


def _cheb_poly(mu, lmax, lmin, k):
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    T = lambda x: np.cosh(k * np.arccosh(x)) if np.all(np.abs(x) >= 1) else np.cos(k * np.arccos(x))
    t = (theta - mu) / delta
    num = np.where(np.abs(t) <= 1, np.cos(k * np.arccos(np.clip(t, -1, 1))),
                   np.cosh(k * np.arccosh(np.maximum(np.abs(t), 1))) * np.sign(t) ** k)
    return num / T(np.array(theta / delta))


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_chebyshev_error_polynomial(k):
    _, _, A, _, _ = _level(n=8, clusters=False)
    Ad = A.toarray()
    d = np.diag(Ad)
    S = Ad / np.sqrt(np.outer(d, d))
    mu, V = np.linalg.eigh(S)
    lmax = mu[-1] * 1.05
    lmin = lmax / 10
    rng = np.random.default_rng(k)
    b = rng.normal(size=len(d))
    x0 = rng.normal(size=len(d))
    xs = np.linalg.solve(Ad, b)
    xk = smoother.chebyshev(A, 1 / d, b, x0, lmax, lmin, k)
    e0h = np.sqrt(d) * (xs - x0)
    ek = (V @ (_cheb_poly(mu, lmax, lmin, k) * (V.T @ e0h))) / np.sqrt(d)
    assert np.max(np.abs((xs - xk) - ek)) < 1e-12 * np.max(np.abs(xs - x0))


def test_local_correction_single_patch_is_exact():
    _, dm, A, _, _ = _level(n=8)
    ls = smoother.LocalSolver(A, [np.arange(A.shape[0])])
    b = np.random.default_rng(1).normal(size=A.shape[0])
    x = ls.apply(A, b, np.zeros_like(b))
    assert np.max(np.abs(A @ x - b)) < 1e-12 * np.max(np.abs(b))


def test_patches_disjoint_spd_and_cover_bad_cells():
    m, dm, A, g, pt = _level(n=16, degree=2)
    allp = np.concatenate(pt)
    assert len(np.unique(allp)) == len(allp)
    bad_dofs = dm.free_index[np.unique(dm.cell_dofs[g < 0.1])]
    assert set(bad_dofs[bad_dofs >= 0]) <= set(allp.tolist())
    for B in pt:
        assert np.linalg.eigvalsh(A[B][:, B].toarray())[0] > 0
    # brute force: a free DoF is in a patch iff one of its cells touches a vertex of a bad cell
    badv = np.zeros(m.nv, bool)
    badv[m.cells[g < 0.1].ravel()] = True
    region = badv[m.cells].any(axis=1)
    expect = dm.free_index[np.unique(dm.cell_dofs[region])]
    assert sorted(expect[expect >= 0].tolist()) == sorted(allp.tolist())


def _bfs_components(cells, region_cells):
    """Connected components of a set of cells under shared-vertex adjacency, by breadth-first
    search over pairs of cells (brute force)."""
    left = set(int(c) for c in region_cells)
    comps = []
    while left:
        start = left.pop()
        comp, queue = {start}, [start]
        while queue:
            c = queue.pop()
            vc = set(cells[c].tolist())
            for o in list(left):
                if vc & set(cells[o].tolist()):
                    left.discard(o)
                    comp.add(o)
                    queue.append(o)
        comps.append(sorted(comp))
    return comps


@pytest.mark.parametrize("layers", [1, 2])
def test_patch_components_are_vertex_connected_components(layers):
    """Sec. 4.1/4.4: the subdomains are the vertex-connected components of the extended
    region. Bad cells are planted through gamma on a 14^2 P2 mesh: two far-apart cells (two
    patches), and two cells that share only a vertex (one merged patch); every patch equals the
    free DoFs of one brute-force component."""
    m = inputs.jitter_mesh(inputs.structured_mesh(2, 14), 0.2, np.random.default_rng(7))
    dm = fem.dof_map(m.coords, m.cells, 2)
    cents = m.coords[m.cells].mean(axis=1)
    far_a = int(np.argmin(np.linalg.norm(cents - [0.2, 0.2], axis=1)))
    far_b = int(np.argmin(np.linalg.norm(cents - [0.8, 0.8], axis=1)))
    # a cell touching far_b's region only through one vertex, two layers away from far_a
    vb = set(m.cells[far_b].tolist())
    touch = [c for c in range(len(m.cells)) if len(vb & set(m.cells[c].tolist())) == 1]
    g = np.ones(len(m.cells))
    for bad, expect in (([far_a, far_b], 2), ([far_b, touch[0]], 1)):
        g[:] = 1.0
        g[bad] = 1e-3
        pt = patches.local_patches(m.cells, g, 0.1, layers, m.nv, dm.cell_dofs, dm.free_index)
        # the extended region by its definition: cells sharing a vertex with the region, repeated
        region = set(bad)
        for _ in range(layers):
            verts = set(m.cells[sorted(region)].ravel().tolist())
            region = {c for c in range(len(m.cells)) if verts & set(m.cells[c].tolist())}
        comps = _bfs_components(m.cells, sorted(region))
        assert len(comps) == expect == len(pt), (bad, len(comps), len(pt))
        want = []
        for comp in comps:
            f = dm.free_index[np.unique(dm.cell_dofs[comp].ravel())]
            want.append(np.sort(f[f >= 0]))
        want.sort(key=lambda p: int(p[0]))
        assert all(np.array_equal(a, b) for a, b in zip(pt, want))


def _dense_operator(fn, n):
    return np.stack([fn(np.eye(n)[i]) for i in range(n)], axis=1)


@pytest.mark.parametrize("order", ["sandwich", "global_then_local"])
def test_combined_smoother_closed_form_and_symmetry(order):
    _, dm, A, _, pt = _level(n=8, degree=1)
    assert pt
    n = A.shape[0]
    Ad = A.toarray()
    dinv = 1 / A.diagonal()
    lmax = eig.lambda_max(A)
    lmin = lmax / 10
    ls = smoother.LocalSolver(A, pt)
    Sc = np.zeros((n, n))
    for B in pt:
        Sc[np.ix_(B, B)] = np.linalg.inv(Ad[np.ix_(B, B)])
    Sg = _dense_operator(lambda e: smoother.chebyshev(A, dinv, e, np.zeros(n), lmax, lmin, 2), n)
    pre = _dense_operator(lambda e: smoother.smooth(A, dinv, e, np.zeros(n), lmax, lmin, 2, ls, order, False), n)
    post = _dense_operator(lambda e: smoother.smooth(A, dinv, e, np.zeros(n), lmax, lmin, 2, ls, order, True), n)
    I = np.eye(n)
    if order == "sandwich":
        Sgc = 2 * Sc - Sc @ Ad @ Sc + (I - Sc @ Ad) @ Sg @ (I - Ad @ Sc)
        assert np.max(np.abs(pre - Sgc)) < 1e-10 * np.max(np.abs(Sgc))
        assert np.max(np.abs(pre - pre.T)) < 1e-10 * np.max(np.abs(pre))
    else:
        # pre = S_g then S_c, post = S_c then S_g: the error operators are adjoints in the A-inner product
        Epre = I - pre @ Ad
        Epost = I - post @ Ad
        assert np.max(np.abs(Ad @ Epre - (Ad @ Epost).T)) < 1e-10 * np.max(np.abs(Ad))


def test_no_patches_reduces_to_chebyshev_bitwise():
    _, _, A, _, _ = _level(n=8, clusters=False)
    ls = smoother.LocalSolver(A, [])
    b = np.random.default_rng(2).normal(size=A.shape[0])
    x0 = np.random.default_rng(3).normal(size=A.shape[0])
    dinv = 1 / A.diagonal()
    a = smoother.smooth(A, dinv, b, x0, 2.1, 0.21, 2, ls, "sandwich", False)
    c = smoother.chebyshev(A, dinv, b, x0, 2.1, 0.21, 2)
    assert np.array_equal(a, c)


def test_high_quality_lambda_in_paper_range():
    # Table eig_cube: lambda_max(D^-1 A) of P1 on good unit-cube meshes is 2.0-2.4
    m = inputs.jitter_mesh(inputs.structured_mesh(3, 8), 0.15, np.random.default_rng(1))
    dm = fem.dof_map(m.coords, m.cells, 1)
    A = fem.restrict_free(fem.assemble_stiffness_full(m.coords, m.cells, dm), dm)
    assert 1.8 < eig.lambda_max(A) < 2.6


def test_adjusted_lambda_recovers_high_quality_value():
    """Sec. 5 / Table eig_cube pattern: low-quality cells inflate lambda_max(D^-1 A); the
    adjusted value (the A_gg block, g outside the patches) returns to the clean mesh's."""
    clean = inputs.config_c1(clusters=False)[0]
    bad = inputs.config_c1()[0]
    lam = {}
    for key, m in (("clean", clean), ("bad", bad)):
        dm = fem.dof_map(m.coords, m.cells, 1)
        A = fem.restrict_free(fem.assemble_stiffness_full(m.coords, m.cells, dm), dm)
        g = quality.radius_ratio(m.coords, m.cells)
        pt = patches.local_patches(m.cells, g, 0.1, 1, m.nv, dm.cell_dofs, dm.free_index)
        lam[key] = (eig.lambda_max(A), eig.adjusted_lambda_max(A, pt))
    assert lam["clean"][0] == lam["clean"][1]
    assert lam["bad"][0] > 1.3 * lam["clean"][0]
    assert abs(lam["bad"][1] - lam["clean"][0]) < 0.05 * lam["clean"][0]


def test_direct_solver_spd_is_plain_solve():
    rng = np.random.default_rng(11)
    M = rng.normal(size=(40, 40))
    A = M @ M.T + 40 * np.eye(40)
    r = rng.normal(size=40)
    ds = smoother.DirectSolver(A)
    assert ds.keep.all()
    assert np.max(np.abs(ds.solve(r) - np.linalg.solve(A, r))) < 1e-12


def test_direct_solver_semidefinite_consistent():
    """A Gram matrix of k < n vectors has rank k: exactly n - k DoFs are dependent, and
    every consistent right-hand side (in the range) is solved exactly."""
    rng = np.random.default_rng(12)
    for n, k in ((30, 22), (50, 49), (12, 3)):
        V = rng.normal(size=(n, k))
        A = V @ V.T
        ds = smoother.DirectSolver(A)
        assert int((~ds.keep).sum()) == n - k
        r = A @ rng.normal(size=n)
        e = ds.solve(r)
        assert np.max(np.abs(A @ e - r)) < 1e-10 * np.max(np.abs(r))
    with pytest.raises(np.linalg.LinAlgError):
        smoother.DirectSolver(-np.eye(3))


def test_multicolour_sgs_is_sequential_sgs_in_colour_order():
    """The multicolour sweep equals plain sequential symmetric Gauss-Seidel over the rows
    sorted by colour (brute-force row-by-row loop), the colouring is valid, and the SGS
    error operator is self-adjoint in the A inner product."""
    _, _, A, _, _ = _level(n=8, degree=2)
    n = A.shape[0]
    colour = smoother.greedy_colouring(A)
    Ac = A.tocoo()
    dg = np.sqrt(A.diagonal())
    strong = (Ac.row != Ac.col) & (np.abs(Ac.data) > smoother.COLOUR_TOL * dg[Ac.row] * dg[Ac.col])
    assert np.all(colour[Ac.row[strong]] != colour[Ac.col[strong]])
    Ad = A.toarray()
    d = np.diag(Ad)
    rng = np.random.default_rng(9)
    b, x0 = rng.normal(size=n), rng.normal(size=n)
    order = np.argsort(colour, kind="stable")
    x = x0.copy()
    for i in list(order) + list(order[::-1]):
        x[i] += (b[i] - Ad[i] @ x) / d[i]
    y = smoother.multicolour_sgs(A, 1 / d, b, x0, colour)
    assert np.max(np.abs(x - y)) < 1e-12 * np.max(np.abs(x))
    E = np.stack([smoother.multicolour_sgs(A, 1 / d, np.zeros(n), np.eye(n)[i], colour) for i in range(n)], axis=1)
    AE = Ad @ E
    assert np.max(np.abs(AE - AE.T)) < 1e-10 * np.max(np.abs(AE))


def test_sgs_vcycle_symmetric_and_correction_claim(c1_meshes):
    from oracle import mg
    H = hierarchy.build(c1_meshes, 1, layers=2, smoother_kind="sgs")
    Hn = hierarchy.build(c1_meshes, 1, layers=2, smoother_kind="sgs", order="global")
    n = H.levels[0].n
    rng = np.random.default_rng(4)
    x, y = rng.normal(size=n), rng.normal(size=n)
    assert abs(x @ mg.vcycle(H, y) - y @ mg.vcycle(H, x)) < 1e-12 * abs(x @ mg.vcycle(H, x))
    b = inputs.uniform_rhs(n, 6)
    sc = mg.stationary(H, b, 1e-10)[1]
    sn = mg.stationary(Hn, b, 1e-10, maxit=400)[1]
    assert sn > sc, (sc, sn)
