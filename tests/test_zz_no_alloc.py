"""The allocation-free dense product mg_dense_symv_static against the existing entry point.

mg_dense_symv_static serves callers that cannot allocate device memory at the point of the
call (memory pre-reserved by another allocator, latency-critical paths): it keeps its
split-K scratch in a static device array. Here it must reproduce mg_coarse_solve (the
coarsest-level direct solve, which uses the hierarchy's allocated scratch) on two calls in
a row, with X the inverse of the exported coarsest operator. This file is collected last
and also passes alone in a fresh process (the first call sets the array's address up).
"""
import numpy as np
import pytest

from _util import TOL64, case, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nnmg():
    from paper_2402_12947_gb300 import build
    build.build()
    from paper_2402_12947_gb300 import nnmg as mod
    return mod


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


def test_static_scratch_rejects_sizes_beyond_the_limit(nnmg):
    import ctypes
    code = nnmg.lib.mg_dense_symv_static(ctypes.c_void_p(1), 65537, ctypes.c_void_p(1), ctypes.c_void_p(1), None)
    assert code == nnmg.ERR_INVALID_ARG
    assert "65536" in nnmg.lib.mg_last_error(None).decode()
    assert nnmg.lib.mg_dense_symv_static(None, 10, None, None, None) == nnmg.ERR_INVALID_ARG
