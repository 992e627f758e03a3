"""Pins of the oracle's linear elasticity discretisation (Sec. 6.3) against invariants and
closed forms: symmetry, rigid-body kernel, affine-field energies, traction load moments,
and convergence rates of a manufactured solution."""
import numpy as np
import pytest

from oracle import elasticity, fem
from paper_2402_12947_gb300 import inputs

MU, LAM = 1.3, 0.7


def _mesh(dim, n, seed=0, amp=0.2):
    m = inputs.structured_mesh(dim, n)
    return inputs.jitter_mesh(m, amp, np.random.default_rng(seed))


def _affine(dm, G, c=None):
    """Coefficients of u(x) = G x + c at every DoF point, vector-numbered."""
    c = np.zeros(dm.dim) if c is None else c
    return (dm.points @ G.T + c).ravel()


@pytest.mark.parametrize("dim,degree", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_symmetric_and_rigid_body_kernel(dim, degree):
    m = _mesh(dim, 4 if dim == 2 else 3)
    dm = fem.dof_map(m.coords, m.cells, degree)
    K = elasticity.assemble_full(m.coords, m.cells, dm, MU, LAM)
    assert abs(K - K.T).max() <= 1e-13 * abs(K).max()
    scale = abs(K).max()
    for c in range(dim):                                   # translations
        t = np.zeros(dim)
        t[c] = 1.0
        r = _affine(dm, np.zeros((dim, dim)), t)
        assert np.abs(K @ r).max() <= 1e-12 * scale
    for a in range(dim):                                   # infinitesimal rotations
        for b in range(a + 1, dim):
            W = np.zeros((dim, dim))
            W[a, b], W[b, a] = 1.0, -1.0
            r = _affine(dm, W)
            assert np.abs(K @ r).max() <= 1e-12 * scale
    # a stretch is not in the kernel
    assert np.abs(K @ _affine(dm, np.eye(dim))).max() > 1e-3 * scale


@pytest.mark.parametrize("dim,degree", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_affine_energies(dim, degree):
    """u^T K u = vol (2 mu eps:eps + lambda tr(eps)^2) for u = G x on the unit square/cube."""
    m = _mesh(dim, 3, seed=1)
    dm = fem.dof_map(m.coords, m.cells, degree)
    K = elasticity.assemble_full(m.coords, m.cells, dm, MU, LAM)
    dil = np.eye(dim)                                      # eps = I: 2 mu d + lambda d^2
    u = _affine(dm, dil)
    assert np.isclose(u @ K @ u, 2 * MU * dim + LAM * dim ** 2, rtol=1e-12)
    sh = np.zeros((dim, dim))
    sh[0, 1] = 1.0                                         # eps:eps = 1/2, tr = 0: mu
    u = _affine(dm, sh)
    assert np.isclose(u @ K @ u, MU, rtol=1e-12)
    G = np.arange(dim * dim, dtype=float).reshape(dim, dim) / 7.0 - 0.3
    eps = 0.5 * (G + G.T)
    u = _affine(dm, G)
    assert np.isclose(u @ K @ u, 2 * MU * np.sum(eps * eps) + LAM * np.trace(eps) ** 2, rtol=1e-12)


@pytest.mark.parametrize("dim,degree", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_traction_load_force_and_moment(dim, degree):
    """On the face x_0 = 1 of the unit square/cube: sum b = t |face|, and the moment
    sum_i b_i x_{i,1} = t int x_1 = t |face| / 2 (basis functions reproduce x_1)."""
    m = _mesh(dim, 4, seed=2)
    dm = fem.dof_map(m.coords, m.cells, degree)
    t = np.array([3.0, -1.0, 0.5][:dim])
    b = elasticity.traction_load_full(m.coords, m.cells, dm, t, axis=0, value=1.0).reshape(-1, dim)
    assert np.allclose(b.sum(axis=0), t, rtol=1e-13, atol=1e-14)
    mom = (b * dm.points[:, 1:2]).sum(axis=0)
    assert np.allclose(mom, 0.5 * t, rtol=1e-12, atol=1e-14)
    # nothing lands off the face
    off = np.abs(dm.points[:, 0] - 1.0) > 1e-12
    assert np.all(b[off] == 0)


def test_lame_parameters():
    """E = 2 mu (1 + nu) and the bulk modulus lambda + 2 mu / 3 = E / (3 (1 - 2 nu))."""
    E, nu = 6.9e10, 0.33
    mu, lam = elasticity.lame(E, nu)
    assert np.isclose(2 * mu * (1 + nu), E, rtol=1e-15)
    assert np.isclose(lam + 2 * mu / 3, E / (3 * (1 - 2 * nu)), rtol=1e-14)


def _manufactured(dim):
    import sympy as s
    X = s.symbols("x0:%d" % dim)
    bump = 1
    for x in X:
        bump = bump * s.sin(s.pi * x)
    u = [bump * (1 + k + X[0] * (k + 1) ** 2 * 0.5) for k in range(dim)]
    grad = [[s.diff(u[i], X[j]) for j in range(dim)] for i in range(dim)]
    eps = [[(grad[i][j] + grad[j][i]) / 2 for j in range(dim)] for i in range(dim)]
    tr = sum(eps[i][i] for i in range(dim))
    sig = [[2 * MU * eps[i][j] + (LAM * tr if i == j else 0) for j in range(dim)] for i in range(dim)]
    f = [-sum(s.diff(sig[i][j], X[j]) for j in range(dim)) for i in range(dim)]
    fu = [s.lambdify(X, e, "numpy") for e in u]
    ff = [s.lambdify(X, e, "numpy") for e in f]
    U = lambda P, c: np.broadcast_to(fu[c](*P.T), (P.shape[0],)).astype(float)
    F = lambda P, c: np.broadcast_to(ff[c](*P.T), (P.shape[0],)).astype(float)
    return U, F


@pytest.mark.parametrize("degree,rate", [(1, 2.0), (2, 3.0)])
def test_manufactured_solution_rates(degree, rate):
    pytest.importorskip("sympy")
    dim = 2
    U, F = _manufactured(dim)
    errs = []
    for n in (8, 16):
        m = _mesh(dim, n, seed=3, amp=0.1)
        dm = fem.dof_map(m.coords, m.cells, degree)
        K = elasticity.restrict_free(elasticity.assemble_full(m.coords, m.cells, dm, MU, LAM), dm)
        b = np.stack([fem.load_vector_full(m.coords, m.cells, dm, lambda P, c=c: F(P, c)) for c in range(dim)],
                     axis=1).ravel()
        fv = elasticity.free_vector_dofs(dm)
        import scipy.sparse.linalg as spl
        u = np.zeros(dm.ndofs * dim)
        u[fv] = spl.spsolve(K.tocsc(), b[fv])
        u = u.reshape(-1, dim)
        e2 = sum(fem.l2_error(m.coords, m.cells, dm, u[:, c], lambda P, c=c: U(P, c)) ** 2 for c in range(dim))
        errs.append(np.sqrt(e2))
    observed = np.log2(errs[0] / errs[1])
    assert observed > rate - 0.25, (errs, observed)


@pytest.mark.parametrize("kind", ["chebyshev", "sgs"])
def test_mg_pcg_solves_the_clamped_lattice(kind):
    """MG-PCG on the elasticity hierarchy (Sec. 6.3: clamped face, traction on the opposite
    face) reaches the sparse direct solution; the V-cycle stays symmetric."""
    import scipy.sparse.linalg as spl
    from oracle import hierarchy, mg
    ms, masks = inputs.config_lattice(ns=(3, 2, 1), n_clusters=3)
    H = hierarchy.build(ms, 1, pde="elasticity", dirichlet_masks=masks, smoother_kind=kind, nu=2)
    lo = H.levels[0]
    b = elasticity.traction_load_full(ms[0].coords, ms[0].cells, lo.dm, [1e3, 0, 0], 0, 6.0)
    b = b[elasticity.free_vector_dofs(lo.dm)]
    x, it, hist, true = mg.pcg(H, b, 1e-10)
    xd = spl.spsolve(lo.A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
    assert it < 60
    r = np.random.default_rng(0)
    u, v = r.standard_normal(lo.n), r.standard_normal(lo.n)
    Bu, Bv = mg.vcycle(H, u), mg.vcycle(H, v)
    assert abs(v @ Bu - u @ Bv) <= 1e-10 * abs(v @ Bu)
