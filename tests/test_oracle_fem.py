"""Pins for the oracle's quadrature, DoF map and assembly (no GPU).

Each test checks the oracle against something other than itself: closed-form
integrals, exact rational integration (sympy), textbook stencils, invariants of the
Laplacian, and the convergence order of a manufactured solution.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem
from oracle.quadrature import simplex_rule
from paper_2402_12947_gb300 import inputs


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("degree", [0, 2, 4, 6])
def test_quadrature_monomials(dim, degree):
    pts, w = simplex_rule(dim, degree)
    for a in itertools.product(range(degree + 1), repeat=dim):
        if sum(a) > degree:
            continue
        got = np.sum(w * np.prod(pts ** np.array(a), axis=1))
        exact = np.prod([math.factorial(k) for k in a]) / math.factorial(dim + sum(a))
        assert abs(got - exact) <= 1e-15 + 1e-13 * exact


def test_p1_five_point_stencil():
    m = inputs.structured_mesh(2, 8)
    dm = fem.dof_map(m.coords, m.cells, 1)
    A = fem.restrict_free(fem.assemble_stiffness_full(m.coords, m.cells, dm), dm).toarray()
    # interior free vertex (i, j) = (3, 4); free numbering is row-major over interior vertices
    n = 7
    r = 3 * n + 2
    row = A[r]
    assert abs(row[r] - 4.0) < 1e-14
    for c in (r - 1, r + 1, r - n, r + n):
        assert abs(row[c] + 1.0) < 1e-14
    mask = np.ones(len(row), bool)
    mask[[r, r - 1, r + 1, r - n, r + n]] = False
    assert np.max(np.abs(row[mask])) < 1e-14


def _sympy_p2_stiffness(dim):
    sympy = pytest.importorskip("sympy")
    xs = sympy.symbols("x0:%d" % dim)
    lam = [1 - sum(xs)] + list(xs)
    edges = fem.LOCAL_EDGES[dim]
    basis = [l * (2 * l - 1) for l in lam] + [4 * lam[a] * lam[b] for a, b in edges]
    grads = [[sympy.diff(p, x) for x in xs] for p in basis]

    def integrate(expr):
        if dim == 2:
            return sympy.integrate(sympy.integrate(expr, (xs[1], 0, 1 - xs[0])), (xs[0], 0, 1))
        return sympy.integrate(sympy.integrate(sympy.integrate(
            expr, (xs[2], 0, 1 - xs[0] - xs[1])), (xs[1], 0, 1 - xs[0])), (xs[0], 0, 1))

    n = len(basis)
    K = np.zeros((n, n))
    for i in range(n):
        for j in range(i, n):
            v = integrate(sum(gi * gj for gi, gj in zip(grads[i], grads[j])))
            K[i, j] = K[j, i] = float(v)
    return K


@pytest.mark.parametrize("dim", [2, 3])
def test_p2_reference_stiffness_exact(dim):
    K = _sympy_p2_stiffness(dim)
    coords = np.concatenate([np.zeros((1, dim)), np.eye(dim)])
    cells = np.arange(dim + 1, dtype=np.int32)[None]
    Ko = fem.element_stiffness(coords, cells, 2)[0]
    assert np.max(np.abs(Ko - K)) < 1e-13


@pytest.mark.parametrize("dim,degree", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_full_stiffness_symmetric_zero_rowsum(dim, degree):
    n = 6 if dim == 2 else 3
    m = inputs.jitter_mesh(inputs.structured_mesh(dim, n), 0.2, np.random.default_rng(7))
    dm = fem.dof_map(m.coords, m.cells, degree)
    A = fem.assemble_stiffness_full(m.coords, m.cells, dm)
    assert abs(A - A.T).max() < 1e-13
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) < 1e-12
    Af = fem.restrict_free(A, dm).toarray()
    assert np.linalg.eigvalsh(Af)[0] > 0


@pytest.mark.parametrize("dim,degree", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_constant_load_closed_form(dim, degree):
    n = 5 if dim == 2 else 2
    m = inputs.jitter_mesh(inputs.structured_mesh(dim, n), 0.15, np.random.default_rng(3))
    dm = fem.dof_map(m.coords, m.cells, degree)
    b = fem.load_vector_full(m.coords, m.cells, dm, 1.0)
    vol = np.abs(inputs.signed_volumes(m.coords, m.cells)) / math.factorial(dim)
    expect = np.zeros(dm.ndofs)
    if degree == 1:
        per_vertex, per_edge = 1.0 / (dim + 1), 0.0
    elif dim == 2:
        per_vertex, per_edge = 0.0, 1.0 / 3.0
    else:
        per_vertex, per_edge = -1.0 / 20.0, 1.0 / 5.0
    nvl = dim + 1
    for c in range(m.nc):
        for i, g in enumerate(dm.cell_dofs[c]):
            expect[g] += vol[c] * (per_vertex if i < nvl else per_edge)
    assert np.max(np.abs(b - expect)) < 1e-14


def test_p2_free_dof_count():
    for n in (4, 8, 16):
        m = inputs.structured_mesh(2, n)
        dm = fem.dof_map(m.coords, m.cells, 2)
        assert dm.nfree == (2 * n - 1) ** 2
        dm1 = fem.dof_map(m.coords, m.cells, 1)
        assert dm1.nfree == (n - 1) ** 2


def test_dirichlet_mask_partial_boundary():
    m = inputs.structured_mesh(2, 4)
    mask = (m.coords[:, 0] == 0.0) | (m.coords[:, 0] == 1.0)
    dm = fem.dof_map(m.coords, m.cells, 2, mask)
    # Dirichlet DoFs: 2 sides x (5 vertices + 4 edges)
    assert int(dm.dirichlet.sum()) == 18


def _solve_manufactured(dim, degree, n, seed=11):
    m = inputs.jitter_mesh(inputs.structured_mesh(dim, n), 0.15, np.random.default_rng(seed))
    dm = fem.dof_map(m.coords, m.cells, degree)
    A = fem.restrict_free(fem.assemble_stiffness_full(m.coords, m.cells, dm), dm)
    u = lambda x: np.prod(np.sin(np.pi * x), axis=1)
    f = lambda x: dim * np.pi ** 2 * np.prod(np.sin(np.pi * x), axis=1)
    b = fem.load_vector_full(m.coords, m.cells, dm, f)[dm.free]
    uf = spla.spsolve(A.tocsc(), b)
    uall = np.zeros(dm.ndofs)
    uall[dm.free] = uf
    return fem.l2_error(m.coords, m.cells, dm, uall, u)


@pytest.mark.parametrize("dim,degree,sizes,rate", [
    (2, 1, (8, 16, 32), 1.85), (2, 2, (8, 16, 32), 2.8),
    (3, 1, (4, 8), 1.6), (3, 2, (3, 6), 2.6)])
def test_manufactured_solution_rate(dim, degree, sizes, rate):
    errs = [_solve_manufactured(dim, degree, n) for n in sizes]
    rates = [math.log2(errs[i] / errs[i + 1]) * (math.log(2) / math.log(sizes[i + 1] / sizes[i]))
             for i in range(len(errs) - 1)]
    assert min(rates) > rate, (errs, rates)
