"""Pins for the V-cycle (Alg. 1), MG-PCG (Sec. 6.2) and the paper's claims (no GPU)."""
import json
import os

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem, hierarchy, mg
from paper_2402_12947_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def test_two_level_identity_transfer_exact():
    m = inputs.jitter_mesh(inputs.structured_mesh(2, 8), 0.2, np.random.default_rng(1))
    dm = fem.dof_map(m.coords, m.cells, 1)
    A = fem.restrict_free(fem.assemble_stiffness_full(m.coords, m.cells, dm), dm)
    n = A.shape[0]
    b = np.random.default_rng(2).normal(size=n)
    H = hierarchy.from_matrices([A, A], [sp.identity(n, format="csr")], [[], []], [2.5])
    assert np.max(np.abs(A @ mg.vcycle(H, b) - b)) < 1e-12 * np.max(np.abs(b))
    # the same through the geometric build: identical meshes give P = I and A_2 = A_1
    for degree in (1, 2):
        Hg = hierarchy.build([m, m], degree)
        A1 = Hg.levels[0].A
        bg = np.random.default_rng(3).normal(size=A1.shape[0])
        assert np.max(np.abs(A1 @ mg.vcycle(Hg, bg) - bg)) < 1e-11 * np.max(np.abs(bg))


def test_pcg_iterates_minimise_energy_over_krylov_space():
    """PCG's k-th iterate is the A-norm-closest point to A^{-1}b in span{(BA)^j B b, j<k},
    B the (symmetric) V-cycle operator: checked against the brute-force projection."""
    meshes = inputs.hierarchy_meshes(2, 12, 3, 0.2, 9, cluster_levels=(0,), n_clusters=1)
    H = hierarchy.build(meshes, 1)
    A = H.levels[0].A.toarray()
    n = A.shape[0]
    B = np.stack([mg.vcycle(H, np.eye(n)[i]) for i in range(n)], axis=1)
    b = np.random.default_rng(4).normal(size=n)
    xs = np.linalg.solve(A, b)
    K = [B @ b]
    for k in range(1, 6):
        x_k = mg.pcg(H, b, 0.0, maxit=k)[0]
        Q, _ = np.linalg.qr(np.stack(K, axis=1))
        y = np.linalg.solve(Q.T @ A @ Q, Q.T @ b)
        ref = Q @ y
        assert np.sqrt((x_k - ref) @ A @ (x_k - ref)) < 1e-9 * np.sqrt(xs @ A @ xs), k
        K.append(B @ (A @ K[-1]))


def test_vcycle_linear_and_symmetric(c1_meshes):
    for order in ("sandwich", "global_then_local", "global"):
        H = hierarchy.build(c1_meshes, 1, layers=2, order=order)
        n = H.levels[0].n
        rng = np.random.default_rng(3)
        x, y = rng.normal(size=n), rng.normal(size=n)
        Bx, By = mg.vcycle(H, x), mg.vcycle(H, y)
        assert abs(x @ By - y @ Bx) < 1e-12 * abs(x @ Bx)
        assert np.max(np.abs(mg.vcycle(H, 2 * x + y) - (2 * Bx + By))) < 1e-10 * np.max(np.abs(Bx))


def test_pcg_matches_direct_solve(c1_meshes):
    H = hierarchy.build(c1_meshes, 1, layers=2)
    lev = H.levels[0]
    b = fem.load_vector_full(c1_meshes[0].coords, c1_meshes[0].cells, lev.dm, 1.0)[lev.dm.free]
    x, it, hist, true_rel = mg.pcg(H, b, 1e-10)
    xd = spla.spsolve(lev.A.tocsc(), b)
    assert true_rel < 2e-10
    assert np.linalg.norm(x - xd) < 1e-8 * np.linalg.norm(xd)
    assert it == len(hist) - 1


def test_correction_restores_iteration_count(c1_meshes):
    """The paper's claim (Sec. 6, Table number_struct): with the local correction and the
    adjusted eigenvalue the iteration count returns to the high-quality reference (+1 at
    most in the table); without the correction it is markedly higher."""
    gold = json.load(open(GOLDEN))["number_struct"]
    margin = max(gold["with_correction_adjusted"]["P1"]["A"] - gold["reference"]["P1"],
                 gold["with_correction_adjusted"]["P2"]["A"] - gold["reference"]["P2"])
    clean = inputs.config_c1(clusters=False)
    for degree in (1, 2):
        Hr = hierarchy.build(clean, degree, layers=2)
        Hc = hierarchy.build(c1_meshes, degree, layers=2)
        Hn = hierarchy.build(c1_meshes, degree, layers=2, order="global", adjusted=False)
        b = inputs.uniform_rhs(Hr.levels[0].n, 5)
        itr = mg.pcg(Hr, b, 1e-10)[1]
        itc = mg.pcg(Hc, b, 1e-10)[1]
        itn = mg.pcg(Hn, b, 1e-10)[1]
        assert itc <= itr + margin + 1, (degree, itr, itc, itn)
        assert itn >= itc + 4, (degree, itr, itc, itn)
        sr = mg.stationary(Hr, b, 1e-10)[1]
        sc = mg.stationary(Hc, b, 1e-10)[1]
        sn = mg.stationary(Hn, b, 1e-10, maxit=400)[1]
        assert sc <= sr + 2 and sn >= 2 * sc, (degree, sr, sc, sn)
