"""Shared helpers for the library tests: oracle hierarchies and comparison metrics."""
import numpy as np
import scipy.sparse as sp

from oracle import hierarchy
from paper_2402_12947_gb300 import inputs

# FP64 parity bar (relative, infinity norm) for every step of the hot path
TOL64 = 1e-10


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = max(float(np.max(np.abs(b))), 1e-300)
    return float(np.max(np.abs(a - b))) / scale


def small_3d(seed=5, n=8, levels=3, clusters=3):
    return inputs.hierarchy_meshes(3, n, levels, 0.15, seed, cluster_levels=(0, 1), n_clusters=clusters,
                                   moves_per_cluster=(1, 1), kinds=("cap",), eps=1e-3)


CASES = {
    # name: (meshes factory, degree, patch layers)
    "c1_p1": (lambda: inputs.config_c1(), 1, 2),
    "c1_p2": (lambda: inputs.config_c1(), 2, 2),
    "c2_p2_128": (lambda: inputs.config_c2(n_fine=128, levels=4, n_clusters=8), 2, 1),
    "cube_p1": (lambda: small_3d(n=12), 1, 1),
    "cube_p2": (lambda: small_3d(n=6), 2, 1),
    # fine level 146,689 DoFs: its slices span more than 2^16 columns, so the operators there
    # store 32-bit column indices (the kernels of the 1024^2 benchmark); coarser levels 16-bit
    "c2_p2_192": (lambda: inputs.config_c2(n_fine=192, levels=4, n_clusters=8), 2, 1),
}

_cache = {}


def case(name, order="sandwich"):
    """(meshes, oracle hierarchy, degree, layers) for a named case (cached)."""
    key = (name, order)
    if key not in _cache:
        make, degree, layers = CASES[name]
        meshes = make()
        H = hierarchy.build(meshes, degree, layers=layers, order=order)
        _cache[key] = (meshes, H, degree, layers)
    return _cache[key]


def csr_arrays(H):
    As = [lv.A for lv in H.levels]
    Ps = [lv.P for lv in H.levels[:-1]]
    patches = [lv.patches for lv in H.levels]
    lam = [lv.lmax for lv in H.levels[:-1]]
    return As, Ps, patches, lam


def to_csr(rp, ci, v, shape):
    return sp.csr_matrix((v, ci, rp), shape=shape)


_lmin = {}


def lambda_min(A) -> float:
    """Smallest eigenvalue of the SPD matrix A (shift-invert Lanczos about 0)."""
    import scipy.sparse.linalg as sla
    key = (A.shape, A.nnz, float(A.data[:64].sum()))
    if key not in _lmin:
        _lmin[key] = float(sla.eigsh(A.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0])
    return _lmin[key]


def solution_gap_bound(A, b, x1, x2) -> float:
    """Bound on ||x1 - x2||_2 for two approximate solutions of A x = b:
    A (x1 - x2) = (b - A x2) - (b - A x1), so ||x1 - x2|| <= (||b - A x1|| + ||b - A x2||) / lambda_min(A).
    Two solves stopped at the same relative residual need not agree more closely than this."""
    r1 = np.linalg.norm(b - A @ x1)
    r2 = np.linalg.norm(b - A @ x2)
    return (r1 + r2) / lambda_min(A)


def fp32_flags(H):
    """Per level, per patch: 1 where the library hierarchy H applies the inverse in FP32."""
    return [H.export_patch_precision(l) for l in range(H.num_levels)]
