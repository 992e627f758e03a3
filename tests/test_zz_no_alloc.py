"""The allocation-free dense product mg_dense_symv_static.

Some callers cannot allocate device memory at the point where they need this product: all
device memory was handed to another allocator up front (a framework's pre-reserved pool, a
service that forbids allocation after start-up), or the call sits on a latency-critical
path where a cudaMalloc/cudaFree would stall or synchronise the device. The entry point
keeps its split-K scratch in a static device array instead. Here it must reproduce:
  * mg_coarse_solve (the coarsest-level direct solve, which uses the hierarchy's allocated
    scratch), on two calls in a row with X the inverse of the exported coarsest operator;
  * x = X b computed on the host in FP64, for sizes across the whole admitted range
    1 <= n <= 65536, within the rounding bound of a length-n dot product,
    |x - X b| <= gamma_{n+1} (|X| |b|) elementwise (gamma_k = k u / (1 - k u), u = 2^-53).
This file is collected last and also passes alone in a fresh process (the first call sets
the array's address up).
"""
import numpy as np
import pytest

from _util import TOL64, case, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def nnmg():
    from paper_2402_12947_gb300 import build
    build.build()
    from paper_2402_12947_gb300 import nnmg as mod
    return mod


def gamma(k):
    return k * U64 / (1.0 - k * U64)


@pytest.mark.parametrize("name", ["c1_p1", "c1_p2"])
def test_static_scratch_matches_coarse_solve_twice(nnmg, name):
    meshes, Ho, degree, layers = case(name)
    lam = [lv.lmax for lv in Ho.levels[:-1]]
    with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, lambda_override=lam) as H:
        lc = H.num_levels - 1
        n = H.num_dofs(lc)
        rp, ci, v = H.export_level(lc)
        A = np.zeros((n, n))
        for i in range(n):
            A[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
        X = torch.from_numpy(np.ascontiguousarray(np.linalg.inv(A))).cuda()
        for seed in (1, 2):   # two calls in a row share (and overwrite) the static array
            b = torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, n)).cuda()
            x_ref = torch.zeros_like(b)
            x_static = torch.full_like(b, float("nan"))
            H.coarse_solve(b, x_ref)
            nnmg.dense_symv_static(X, b, x_static)
            torch.cuda.synchronize()
            assert rel_err(x_static.cpu().numpy(), x_ref.cpu().numpy()) < TOL64


@pytest.mark.parametrize("n", [1, 100, 4097, 8192])
def test_static_scratch_dense_random(nnmg, n):
    """A random dense symmetric X (mixed signs) against X @ b on the host, twice in a row."""
    rng = np.random.default_rng(n)
    M = rng.uniform(-1, 1, (n, n))
    X = np.ascontiguousarray(M + M.T)
    Xd = torch.from_numpy(X).cuda()
    for seed in (1, 2):
        b = np.random.default_rng(seed).uniform(-1, 1, n)
        x = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        nnmg.dense_symv_static(Xd, torch.from_numpy(b).cuda(), x)
        torch.cuda.synchronize()
        bound = gamma(n + 1) * (np.abs(X) @ np.abs(b))
        assert np.all(np.abs(x.cpu().numpy() - X @ b) <= bound), (n, seed)


@pytest.mark.parametrize("n", [25857, 40000, 65535, 65536])
def test_static_scratch_large_sizes(nnmg, n):
    """Sizes up to the limit (X up to 34 GB, built on the device in row blocks):
    X = diag(d) + f g^T + g f^T, whose product X b = d b + f (g.b) + g (f.b) and whose bound
    |X| |b| <= |d||b| + |f| (|g|.|b|) + |g| (|f|.|b|) the host computes in O(n)."""
    rng = np.random.default_rng(n)
    d, f, g = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    free, _ = torch.cuda.mem_get_info()
    if free < 8 * n * n + (2 << 30):
        pytest.skip("not enough device memory for X")
    fd, gd = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    X = torch.empty((n, n), dtype=torch.float64, device="cuda")
    for i0 in range(0, n, 2048):
        i1 = min(n, i0 + 2048)
        X[i0:i1] = torch.outer(fd[i0:i1], gd) + torch.outer(gd[i0:i1], fd)
    X.diagonal().add_(torch.from_numpy(d).cuda())
    try:
        for seed in (1, 2):
            b = np.random.default_rng(seed).uniform(-1, 1, n)
            x = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            nnmg.dense_symv_static(X, torch.from_numpy(b).cuda(), x)
            torch.cuda.synchronize()
            ref = d * b + f * (g @ b) + g * (f @ b)
            ab = np.abs(b)
            bound = gamma(n + 1) * (np.abs(d) * ab + np.abs(f) * (np.abs(g) @ ab) + np.abs(g) * (np.abs(f) @ ab))
            # plus the host's own rounding of the O(n) reference (two dot products of length n)
            bound += gamma(n + 3) * (np.abs(d) * ab + np.abs(f) * (np.abs(g) @ ab) + np.abs(g) * (np.abs(f) @ ab))
            assert np.all(np.abs(x.cpu().numpy() - ref) <= bound), (n, seed)
    finally:
        del X
        torch.cuda.empty_cache()


def test_static_scratch_rejects_sizes_beyond_the_limit(nnmg):
    import ctypes
    code = nnmg.lib.mg_dense_symv_static(ctypes.c_void_p(1), 65537, ctypes.c_void_p(1), ctypes.c_void_p(1), None)
    assert code == nnmg.ERR_INVALID_ARG
    msg = nnmg.lib.mg_last_error(None).decode()
    assert "65537" in msg and "65536" in msg
    assert nnmg.lib.mg_dense_symv_static(None, 10, None, None, None) == nnmg.ERR_INVALID_ARG
