"""Pins for the non-nested transfer operators (Sec. 2, Eqs. 2-4) (no GPU)."""
import numpy as np
import pytest

from oracle import fem, transfer
from paper_2402_12947_gb300 import inputs


def _mesh(dim, n, seed):
    return inputs.jitter_mesh(inputs.structured_mesh(dim, n), 0.2 if dim == 2 else 0.15,
                              np.random.default_rng(seed))


@pytest.mark.parametrize("dim,degree", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_identical_meshes_give_identity(dim, degree):
    m = _mesh(dim, 5 if dim == 2 else 3, 1)
    dm = fem.dof_map(m.coords, m.cells, degree)
    P = transfer.prolongation(dm, m.coords, m.cells, dm)
    assert P.shape == (dm.nfree, dm.nfree)
    assert abs(P - np.eye(dm.nfree)).max() < 1e-12


@pytest.mark.parametrize("dim,degree", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_polynomial_reproduction_and_partition_of_unity(dim, degree):
    nf, nc = (12, 5) if dim == 2 else (6, 3)
    mf, mc = _mesh(dim, nf, 2), _mesh(dim, nc, 3)
    dmf = fem.dof_map(mf.coords, mf.cells, degree)
    dmc = fem.dof_map(mc.coords, mc.cells, degree)
    P = transfer.prolongation(dmf, mc.coords, mc.cells, dmc, free_only=False)
    assert np.max(np.abs(P @ np.ones(dmc.ndofs) - 1.0)) < 1e-13
    rng = np.random.default_rng(4)
    for _ in range(3):
        c = rng.normal(size=10)
        def poly(x):
            v = c[0] + c[1:1 + dim] @ x.T
            if degree == 2:
                v = v + c[4] * x[:, 0] ** 2 + c[5] * x[:, 0] * x[:, 1] + c[6] * x[:, dim - 1] ** 2
            return v
        assert np.max(np.abs(P @ poly(dmc.points) - poly(dmf.points))) < 1e-12


def test_point_location_brute_force():
    mf, mc = _mesh(2, 9, 5), _mesh(2, 4, 6)
    dmf = fem.dof_map(mf.coords, mf.cells, 2)
    pts = dmf.points
    cell, lam = transfer.locate(mc.coords, mc.cells, pts)
    for i, x in enumerate(pts):
        for k, tri in enumerate(mc.cells):
            X = mc.coords[tri]
            T = np.array([X[1] - X[0], X[2] - X[0]]).T
            l12 = np.linalg.solve(T, x - X[0])
            l = np.array([1 - l12.sum(), *l12])
            if l.min() >= -1e-12:
                assert cell[i] == k
                assert np.allclose(lam[i], l, atol=1e-13)
                break
        else:
            raise AssertionError("point not found")


@pytest.mark.parametrize("dim,degree", [(2, 1), (2, 2), (3, 1)])
def test_galerkin_spd_and_dense_triple_product(dim, degree):
    nf, nc = (10, 5) if dim == 2 else (5, 3)
    mf, mc = _mesh(dim, nf, 7), _mesh(dim, nc, 8)
    dmf = fem.dof_map(mf.coords, mf.cells, degree)
    dmc = fem.dof_map(mc.coords, mc.cells, degree)
    A = fem.restrict_free(fem.assemble_stiffness_full(mf.coords, mf.cells, dmf), dmf)
    P = transfer.prolongation(dmf, mc.coords, mc.cells, dmc)
    Ac = transfer.galerkin(A, P).toarray()
    dense = P.toarray().T @ A.toarray() @ P.toarray()
    assert np.max(np.abs(Ac - dense)) < 1e-12 * np.max(np.abs(dense))
    assert np.max(np.abs(Ac - Ac.T)) < 1e-13 * np.max(np.abs(Ac))
    assert np.linalg.eigvalsh(Ac)[0] > 0
