"""The set-up's batched dense inverse on the GPU against the oracle's direct solver (Sec. 4.1,
Alg. 2; Alg. 1's coarsest solve), including singular blocks.

The library inverts every patch block A[B_d, B_d] and the coarsest operator by a batched
Gauss-Jordan sweep: blocks of at most 128 DoFs in one thread block each (shared memory),
larger ones one launch per pivot. A pivot whose Schur complement falls to 1e-10 of its
diagonal marks a dependent DoF, which is dropped (its row and column of the inverse are
zero), the same rule as the oracle's column-by-column Cholesky: for a consistent right-hand
side both give the solution that is zero on the dependent DoFs. A pivot below -1e-10 of its
diagonal means the block is not positive semi-definite (MG_ERR_NOT_SPD). Blocks here are
Gram matrices V V^T whose dependent rows of V (combinations of earlier rows) sit in the
middle of the ordering, so drops happen between kept pivots.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import smoother

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def nnmg():
    from paper_2402_12947_gb300 import build
    build.build()
    from paper_2402_12947_gb300 import nnmg as mod
    return mod


def gram_with_dependents(n, seed):
    """V V^T where every fifth row of V (from row 10 on) is a combination of two earlier rows
    and the others are random in as many dimensions as there are of them: the dependent DoFs
    are exactly those rows."""
    rng = np.random.default_rng(seed)
    dep_rows = list(range(10, n, 5))
    k = n - len(dep_rows)
    V = rng.normal(size=(n, k))
    dep = []
    for j in dep_rows:
        a, c = rng.integers(0, j, size=2)
        V[j] = 0.7 * V[a] - 1.3 * V[c]
        dep.append(j)
    G = V @ V.T
    return 0.5 * (G + G.T), np.array(dep)


def laplace_1d(m):
    return sp.diags([-np.ones(m - 1), 2.0 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1], format="csr")


def bar(A, keep):
    """Forward-error bar of two backward-stable solves (Cholesky vs explicit inverse)."""
    Ak = A[np.ix_(keep, keep)]
    return max(1e-10, 8.0 * np.linalg.cond(Ak) * U64)


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("sizes", [(60, 100), (128, 129), (100, 300)], ids=["small", "edge", "mixed"])
def test_singular_blocks_match_the_oracle(nnmg, sizes):
    na, nb = sizes
    Ga, _ = gram_with_dependents(na, 1)
    Gb, depb = gram_with_dependents(nb, 2)
    m = 200
    A0 = sp.block_diag([sp.csr_matrix(Ga), sp.csr_matrix(Gb), laplace_1d(m)], format="csr")
    n0 = A0.shape[0]
    G1, dep1 = gram_with_dependents(nb, 3)     # coarsest operator: singular, dense
    n1 = G1.shape[0]
    rng = np.random.default_rng(4)
    P = sp.random(n0, n1, density=0.02, random_state=5, format="csr")
    patches = [[np.arange(na), na + np.arange(nb)], []]
    with nnmg.Hierarchy.from_csr([A0, sp.csr_matrix(G1)], [P], patches, [float(abs(A0).sum(axis=1).max())]) as H:
        # coarsest solve on a consistent right-hand side
        for seed in (6, 7):
            b1 = G1 @ np.random.default_rng(seed).normal(size=n1)
            x1 = torch.zeros(n1, dtype=torch.float64, device="cuda")
            H.coarse_solve(torch.from_numpy(b1).cuda(), x1)
            ds = smoother.DirectSolver(G1)
            assert np.array_equal(np.flatnonzero(~ds.keep), dep1)
            ref = ds.solve(b1)
            assert rel(x1.cpu().numpy(), ref) < bar(G1, ds.keep), seed
        # the local correction on both patches (Alg. 2) from a random iterate
        x0 = rng.normal(size=n0)
        y = rng.normal(size=n0)
        b0 = A0 @ (x0 + y)
        x = torch.from_numpy(x0.copy()).cuda()
        H.local_correction(0, torch.from_numpy(b0).cuda(), x)
        xh = x.cpu().numpy()
        r = b0 - A0 @ x0
        for B, G in ((patches[0][0], Ga), (patches[0][1], Gb)):
            ds = smoother.DirectSolver(G)
            ref = x0[B] + ds.solve(r[B])
            assert rel(xh[B], ref) < bar(G, ds.keep), len(B)
        rest = np.arange(na + nb, n0)
        assert np.array_equal(xh[rest], x0[rest])


@pytest.mark.parametrize("n", [60, 300], ids=["one-block", "per-pivot"])
def test_indefinite_block_is_rejected(nnmg, n):
    """I - 0.9 J/(n/10) (J all ones): positive diagonal, one negative eigenvalue."""
    B = np.eye(n) - 0.9 * np.ones((n, n)) / (n / 10.0)
    assert np.linalg.eigvalsh(B)[0] < 0 and B.diagonal().min() > 0
    m = 50
    A0 = sp.block_diag([laplace_1d(m), laplace_1d(m)], format="csr")
    P = sp.random(2 * m, n, density=0.05, random_state=1, format="csr")
    with pytest.raises(nnmg.NnmgError) as e:
        nnmg.Hierarchy.from_csr([A0, sp.csr_matrix(B)], [P], [[], []], [4.0])
    assert e.value.code == nnmg.ERR_NOT_SPD
