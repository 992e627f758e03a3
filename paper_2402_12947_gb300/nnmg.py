"""Thin ctypes binding over the nnmg C ABI (``include/nnmg.h``): argument marshalling only.

Every step of the solver runs in the shared library (``lib/libnnmg.so``: C++ set-up and
sm_103a CUDA kernels). Device vectors are PyTorch CUDA tensors (float64, contiguous);
host arrays are NumPy. If the library has not been built, importing this module raises:
there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libnnmg.so")

OK, ERR_INVALID_ARG, ERR_DEGENERATE_CELL, ERR_POINT_LOCATION, ERR_NOT_SPD = 0, 1, 2, 3, 4
ERR_NO_CONVERGENCE, ERR_BREAKDOWN, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NO_DEVICE = 5, 6, 7, 8, 9, 10
SMOOTHER = {"sandwich": 0, "global_then_local": 1, "global": 2}
GLOBAL_SMOOTHER = {"chebyshev": 0, "sgs": 1}
PDE = {"poisson": 0, "elasticity": 1}
PRECISION = {"fp64": 0, "mixed": 1}


class NnmgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"nnmg error {code}: {msg}")
        self.code = code


class MgMesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("reserved", C.c_int32), ("nv", C.c_int64), ("nc", C.c_int64),
                ("coords", C.c_void_p), ("cells", C.c_void_p), ("dirichlet_vertex_mask", C.c_void_p)]


class MgOptions(C.Structure):
    _fields_ = [("cheb_degree", C.c_int32), ("nu", C.c_int32), ("patch_layers", C.c_int32),
                ("smoother", C.c_int32), ("adjusted_lambda", C.c_int32), ("precision", C.c_int32),
                ("host_only", C.c_int32), ("eig_maxit", C.c_int32), ("lmin_ratio", C.c_double),
                ("lmax_safety", C.c_double), ("eig_tol", C.c_double), ("lambda_override", C.c_void_p),
                ("use_graph", C.c_int32), ("local_levels_mask", C.c_int32), ("quality_threshold", C.c_double),
                ("sell_sigma", C.c_int32), ("reorder", C.c_int32), ("global_smoother", C.c_int32),
                ("pde", C.c_int32), ("young", C.c_double), ("poisson_ratio", C.c_double),
                ("small_level_dofs", C.c_int32), ("fp32_patch_kappa", C.c_int32), ("tune_min_nnz", C.c_int32),
                ("reserved", C.c_int32 * 1)]


class MgSolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double)]

    def as_dict(self):
        return {"iterations": self.iterations, "converged": bool(self.converged),
                "rel_residual": self.rel_residual, "true_rel_residual": self.true_rel_residual}


class MgCsr(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("ncols", C.c_int64), ("rowptr", C.c_void_p), ("colidx", C.c_void_p),
                ("values", C.c_void_p)]


class MgRequest(C.Structure):
    _fields_ = [("levels", C.c_void_p), ("L", C.c_int32), ("degree", C.c_int32), ("quality_threshold", C.c_double),
                ("opt", C.c_void_p), ("b", C.c_void_p), ("n_b", C.c_int64), ("rtol", C.c_double),
                ("maxit", C.c_int32), ("tune", C.c_int32)]


class MgRequestResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double), ("n", C.c_int64), ("device_bytes", C.c_int64),
                ("t_queue_ms", C.c_double), ("t_setup_ms", C.c_double), ("t_wait_ms", C.c_double),
                ("t_device_ms", C.c_double), ("t_total_ms", C.c_double), ("t_solve_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MgServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("bytes_in_use", C.c_int64), ("peak_bytes", C.c_int64), ("active", C.c_int32),
                ("peak_active", C.c_int32), ("queued", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_P = C.c_void_p
_SIGS = {
    "mg_default_options": (None, [C.POINTER(MgOptions)]),
    "mg_setup": (C.c_int, [C.POINTER(MgMesh), C.c_int32, C.c_int32, C.c_double, C.POINTER(MgOptions), C.POINTER(_P)]),
    "mg_setup_csr": (C.c_int, [C.POINTER(MgCsr), C.POINTER(MgCsr), C.c_int32, _P, _P, _P, C.POINTER(MgOptions),
                               C.POINTER(_P)]),
    "mg_free": (None, [_P]),
    "mg_last_error": (C.c_char_p, [_P]),
    "mg_num_levels": (C.c_int32, [_P]),
    "mg_num_dofs": (C.c_int64, [_P, C.c_int32]),
    "mg_level_nnz": (C.c_int64, [_P, C.c_int32]),
    "mg_transfer_nnz": (C.c_int64, [_P, C.c_int32]),
    "mg_num_patches": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "mg_export_level": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "mg_export_transfer": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "mg_export_patches": (C.c_int, [_P, C.c_int32, _P, _P]),
    "mg_export_patch_precision": (C.c_int, [_P, C.c_int32, _P]),
    "mg_export_colouring": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int32), _P]),
    "mg_eigs": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mg_dof_coords": (C.c_int, [_P, C.c_int32, _P]),
    "mg_cell_quality": (C.c_int, [_P, C.c_int32, _P]),
    "mg_load_constant": (C.c_int, [_P, C.c_double, _P]),
    "mg_load_traction": (C.c_int, [_P, C.c_int32, C.c_double, _P, _P]),
    "mg_load_body": (C.c_int, [_P, _P, _P]),
    "mg_vcycle": (C.c_int, [_P, _P, _P, _P]),
    "mg_solve": (C.c_int, [_P, _P, _P, C.c_double, C.c_int32, C.POINTER(MgSolveInfo), _P]),
    "mg_solve_host": (C.c_int, [_P, _P, _P, C.c_double, C.c_int32, C.POINTER(MgSolveInfo), _P]),
    "mg_solve_stationary": (C.c_int, [_P, _P, _P, C.c_double, C.c_int32, C.POINTER(MgSolveInfo), _P]),
    "mg_solve_batch": (C.c_int, [_P, _P, _P, C.c_int32, C.c_double, C.c_int32, C.POINTER(MgSolveInfo), _P]),
    "mg_apply_A": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "mg_chebyshev": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "mg_time_vcycle": (C.c_int, [_P, C.c_int32, C.c_int32, _P, C.POINTER(C.c_double)]),
    "mg_sgs": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "mg_local_correction": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "mg_smooth": (C.c_int, [_P, C.c_int32, C.c_int32, _P, _P, _P]),
    "mg_residual_restrict": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P]),
    "mg_prolong_correct": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "mg_coarse_solve": (C.c_int, [_P, _P, _P, _P]),
    "mg_time_smoother_kernel": (C.c_int, [_P, C.c_int32, _P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mg_device_bytes": (C.c_int64, [_P]),
    "mg_time_cg_product": (C.c_int, [_P, C.c_int32, _P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mg_measure_fp64_fma": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "mg_time_patch_solve": (C.c_int, [_P, C.c_int32, C.c_int32, _P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mg_server_create": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.POINTER(_P)]),
    "mg_server_submit": (C.c_int, [_P, C.POINTER(MgRequest), C.POINTER(C.c_int64)]),
    "mg_server_poll": (C.c_int, [_P, C.c_int64, C.POINTER(MgRequestResult)]),
    "mg_server_wait": (C.c_int, [_P, C.c_int64, C.c_double, C.POINTER(MgRequestResult)]),
    "mg_server_fetch": (C.c_int, [_P, C.c_int64, _P, C.c_int64]),
    "mg_server_stats": (C.c_int, [_P, C.POINTER(MgServerStats)]),
    "mg_server_last_error": (C.c_char_p, []),
    "mg_server_destroy": (None, [_P]),
    "mg_launch_counts": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mg_dense_symv_static": (C.c_int, [_P, C.c_int64, _P, _P, _P]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"nnmg library not built ({LIB_PATH} missing): run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()
EXPORTED = tuple(_SIGS)


def _err(h):
    msg = lib.mg_last_error(h)
    return msg.decode() if msg else ""


def _check(code, h=None):
    if code != OK:
        raise NnmgError(code, _err(h))


def default_options(**kw) -> MgOptions:
    o = MgOptions()
    lib.mg_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "smoother" and isinstance(v, str):
            v = SMOOTHER[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k == "global_smoother" and isinstance(v, str):
            v = GLOBAL_SMOOTHER[v]
        if k == "pde" and isinstance(v, str):
            v = PDE[v]
        if k == "lambda_override":
            continue
        setattr(o, k, v)
    return o


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _dev_ptr(t, n=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} entries, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class Hierarchy:
    """Owns one mg_hierarchy_t. Levels are numbered 0 (finest) .. L-1 (coarsest)."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle
        self._keep = []

    # ---- construction ----
    @classmethod
    def from_meshes(cls, meshes, degree: int, quality_threshold: float = 0.1, dirichlet_masks=None,
                    lambda_override=None, **opts) -> "Hierarchy":
        o = default_options(**opts)
        arr = (MgMesh * len(meshes))()
        keep = []
        for i, m in enumerate(meshes):
            coords = _np(m.coords, np.float64)
            cells = _np(m.cells, np.int32)
            keep += [coords, cells]
            arr[i].dim = coords.shape[1]
            arr[i].nv = coords.shape[0]
            arr[i].nc = cells.shape[0]
            arr[i].coords = coords.ctypes.data
            arr[i].cells = cells.ctypes.data
            if dirichlet_masks is not None and dirichlet_masks[i] is not None:
                mk = _np(dirichlet_masks[i], np.uint8)
                keep.append(mk)
                arr[i].dirichlet_vertex_mask = mk.ctypes.data
        if lambda_override is not None:
            lo = _np(lambda_override, np.float64)
            keep.append(lo)
            o.lambda_override = lo.ctypes.data
        h = C.c_void_p()
        code = lib.mg_setup(arr, len(meshes), degree, quality_threshold, C.byref(o), C.byref(h))
        if code != OK:
            raise NnmgError(code, _err(None))
        return cls(h)

    @classmethod
    def from_csr(cls, As, Ps, patches, lambdas, **opts) -> "Hierarchy":
        """As: L scipy CSR matrices; Ps: L-1 (level l+1 -> l); patches: per level list of
        index arrays; lambdas: lambda_max per level (L-1)."""
        L = len(As)
        o = default_options(**opts)
        keep = []
        def csr(M, out):
            M = M.tocsr()
            rp = _np(M.indptr, np.int32)
            ci = _np(M.indices, np.int32)
            v = _np(M.data, np.float64)
            keep.extend([rp, ci, v])
            out.nrows, out.ncols = M.shape
            out.rowptr, out.colidx, out.values = rp.ctypes.data, ci.ctypes.data, v.ctypes.data
        Aa = (MgCsr * L)()
        Pa = (MgCsr * max(1, L - 1))()
        for l in range(L):
            csr(As[l], Aa[l])
        for l in range(L - 1):
            csr(Ps[l], Pa[l])
        pp = (C.c_void_p * L)()
        pd = (C.c_void_p * L)()
        npt = (C.c_int32 * L)()
        for l in range(L):
            pl = list(patches[l]) if patches is not None and l < len(patches) else []
            if pl:
                ptr = _np(np.concatenate([[0], np.cumsum([len(p) for p in pl])]), np.int32)
                dofs = _np(np.concatenate(pl), np.int32)
                keep.extend([ptr, dofs])
                pp[l], pd[l], npt[l] = ptr.ctypes.data, dofs.ctypes.data, len(pl)
        lo = _np(lambdas, np.float64)
        keep.append(lo)
        o.lambda_override = lo.ctypes.data
        h = C.c_void_p()
        code = lib.mg_setup_csr(Aa, Pa, L, C.cast(pp, C.c_void_p), C.cast(pd, C.c_void_p),
                                C.cast(npt, C.c_void_p), C.byref(o), C.byref(h))
        if code != OK:
            raise NnmgError(code, _err(None))
        return cls(h)

    def close(self):
        if self._h:
            lib.mg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- queries / exports ----
    @property
    def num_levels(self) -> int:
        return lib.mg_num_levels(self._h)

    def num_dofs(self, l: int = 0) -> int:
        return int(lib.mg_num_dofs(self._h, l))

    def export_level(self, l: int):
        n, nnz = self.num_dofs(l), int(lib.mg_level_nnz(self._h, l))
        rp, ci, v = np.zeros(n + 1, np.int32), np.zeros(nnz, np.int32), np.zeros(nnz, np.float64)
        _check(lib.mg_export_level(self._h, l, rp.ctypes.data, ci.ctypes.data, v.ctypes.data), self._h)
        return rp, ci, v

    def export_transfer(self, l: int):
        n, nnz = self.num_dofs(l), int(lib.mg_transfer_nnz(self._h, l))
        rp, ci, v = np.zeros(n + 1, np.int32), np.zeros(nnz, np.int32), np.zeros(nnz, np.float64)
        _check(lib.mg_export_transfer(self._h, l, rp.ctypes.data, ci.ctypes.data, v.ctypes.data), self._h)
        return rp, ci, v

    def export_patches(self, l: int):
        num, tot = C.c_int32(), C.c_int64()
        _check(lib.mg_num_patches(self._h, l, C.byref(num), C.byref(tot)), self._h)
        ptr, dofs = np.zeros(num.value + 1, np.int32), np.zeros(tot.value, np.int32)
        _check(lib.mg_export_patches(self._h, l, ptr.ctypes.data, dofs.ctypes.data), self._h)
        return [dofs[ptr[i]:ptr[i + 1]].copy() for i in range(num.value)]

    def export_patch_precision(self, l: int):
        """1 per patch whose inverse is applied in FP32, else 0 (order of export_patches)."""
        num = C.c_int32()
        tot = C.c_int64()
        _check(lib.mg_num_patches(self._h, l, C.byref(num), C.byref(tot)), self._h)
        flags = np.zeros(max(num.value, 1), dtype=np.int32)
        _check(lib.mg_export_patch_precision(self._h, l, flags.ctypes.data), self._h)
        return flags[:num.value]

    def export_colouring(self, l: int):
        num = C.c_int32()
        _check(lib.mg_export_colouring(self._h, l, C.byref(num), None), self._h)
        colour = np.zeros(self.num_dofs(l), np.int32)
        _check(lib.mg_export_colouring(self._h, l, C.byref(num), colour.ctypes.data), self._h)
        return colour

    def eigs(self, l: int):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        _check(lib.mg_eigs(self._h, l, C.byref(a), C.byref(b), C.byref(c)), self._h)
        return a.value, b.value, c.value

    def dof_coords(self, l: int, dim: int):
        out = np.zeros((self.num_dofs(l), dim))
        _check(lib.mg_dof_coords(self._h, l, out.ctypes.data), self._h)
        return out

    def cell_quality(self, l: int, nc: int):
        out = np.zeros(nc)
        _check(lib.mg_cell_quality(self._h, l, out.ctypes.data), self._h)
        return out

    def load_constant(self, f: float = 1.0):
        out = np.zeros(self.num_dofs(0))
        _check(lib.mg_load_constant(self._h, f, out.ctypes.data), self._h)
        return out

    def time_vcycle(self, level: int = 0, reps: int = 20, stream=None) -> float:
        ms = C.c_double()
        _check(lib.mg_time_vcycle(self._h, level, reps, _stream(stream), C.byref(ms)), self._h)
        return ms.value

    def load_body(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros(self.num_dofs(0))
        _check(lib.mg_load_body(self._h, f.ctypes.data, out.ctypes.data), self._h)
        return out

    def load_traction(self, axis: int, value: float, t):
        t = np.ascontiguousarray(t, dtype=np.float64)
        out = np.zeros(self.num_dofs(0))
        _check(lib.mg_load_traction(self._h, axis, value, t.ctypes.data, out.ctypes.data), self._h)
        return out

    def device_bytes(self) -> int:
        return int(lib.mg_device_bytes(self._h))

    def launch_counts(self):
        a, b = C.c_int32(), C.c_int32()
        _check(lib.mg_launch_counts(self._h, C.byref(a), C.byref(b)), self._h)
        return a.value, b.value

    # ---- hot path (torch CUDA float64 tensors) ----
    def vcycle(self, b, x, stream=None):
        n = self.num_dofs(0)
        _check(lib.mg_vcycle(self._h, _dev_ptr(b, n), _dev_ptr(x, n), _stream(stream)), self._h)

    def solve(self, b, x, rtol=1e-8, maxit=500, stream=None, raise_on_fail=True):
        n = self.num_dofs(0)
        info = MgSolveInfo()
        code = lib.mg_solve(self._h, _dev_ptr(b, n), _dev_ptr(x, n), rtol, maxit, C.byref(info), _stream(stream))
        if code != OK and (raise_on_fail or code not in (ERR_NO_CONVERGENCE, ERR_BREAKDOWN)):
            raise NnmgError(code, _err(self._h))
        d = info.as_dict()
        d["status"] = code
        return d

    def solve_host(self, b: np.ndarray, rtol=1e-8, maxit=500, stream=None, out=None):
        b = _np(b, np.float64)
        x = np.zeros_like(b) if out is None else out
        info = MgSolveInfo()
        code = lib.mg_solve_host(self._h, b.ctypes.data, x.ctypes.data, rtol, maxit, C.byref(info), _stream(stream))
        if code != OK:
            raise NnmgError(code, _err(self._h))
        return x, info.as_dict()

    def solve_stationary(self, b, x, rtol=1e-8, maxit=200, stream=None):
        n = self.num_dofs(0)
        info = MgSolveInfo()
        code = lib.mg_solve_stationary(self._h, _dev_ptr(b, n), _dev_ptr(x, n), rtol, maxit, C.byref(info),
                                       _stream(stream))
        if code not in (OK, ERR_NO_CONVERGENCE):
            raise NnmgError(code, _err(self._h))
        d = info.as_dict()
        d["status"] = code
        return d

    def apply_A(self, l, x, y, stream=None):
        n = self.num_dofs(l)
        _check(lib.mg_apply_A(self._h, l, _dev_ptr(x, n), _dev_ptr(y, n), _stream(stream)), self._h)

    def chebyshev(self, l, b, x, stream=None):
        n = self.num_dofs(l)
        _check(lib.mg_chebyshev(self._h, l, _dev_ptr(b, n), _dev_ptr(x, n), _stream(stream)), self._h)

    def sgs(self, l, b, x, stream=None):
        n = self.num_dofs(l)
        _check(lib.mg_sgs(self._h, l, _dev_ptr(b, n), _dev_ptr(x, n), _stream(stream)), self._h)

    def local_correction(self, l, b, x, stream=None):
        n = self.num_dofs(l)
        _check(lib.mg_local_correction(self._h, l, _dev_ptr(b, n), _dev_ptr(x, n), _stream(stream)), self._h)

    def smooth(self, l, b, x, post=False, stream=None):
        n = self.num_dofs(l)
        _check(lib.mg_smooth(self._h, l, int(post), _dev_ptr(b, n), _dev_ptr(x, n), _stream(stream)), self._h)

    def residual_restrict(self, l, b, x, r, bc, stream=None):
        n, nc = self.num_dofs(l), self.num_dofs(l + 1)
        _check(lib.mg_residual_restrict(self._h, l, _dev_ptr(b, n), _dev_ptr(x, n), _dev_ptr(r, n),
                                        _dev_ptr(bc, nc), _stream(stream)), self._h)

    def prolong_correct(self, l, xc, x, stream=None):
        n, nc = self.num_dofs(l), self.num_dofs(l + 1)
        _check(lib.mg_prolong_correct(self._h, l, _dev_ptr(xc, nc), _dev_ptr(x, n), _stream(stream)), self._h)

    def coarse_solve(self, b, x, stream=None):
        n = self.num_dofs(self.num_levels - 1)
        _check(lib.mg_coarse_solve(self._h, _dev_ptr(b, n), _dev_ptr(x, n), _stream(stream)), self._h)

    def time_patch_solve(self, l=0, reps=20, stream=None):
        """(ms per launch, FMAs with FP64 inverses, FMAs with FP32 inverses, inverse bytes) of
        one S_c solve launch on level l."""
        v = [C.c_double() for _ in range(4)]
        _check(lib.mg_time_patch_solve(self._h, l, reps, _stream(stream), *[C.byref(x) for x in v]), self._h)
        return tuple(x.value for x in v)

    def time_cg_product(self, reps=20, stream=None):
        """(ms per launch, algorithmic bytes per launch) of the FP64 CG product q = A p."""
        ms, by = C.c_double(), C.c_double()
        _check(lib.mg_time_cg_product(self._h, reps, _stream(stream), C.byref(ms), C.byref(by)), self._h)
        return ms.value, by.value

    def time_smoother_kernel(self, reps=20, stream=None):
        ms, nbytes = C.c_double(), C.c_double()
        _check(lib.mg_time_smoother_kernel(self._h, reps, _stream(stream), C.byref(ms), C.byref(nbytes)), self._h)
        return ms.value, nbytes.value


def measure_fp64_fma(stream=None) -> float:
    """FP64 FMAs per second of the current device (see mg_measure_fp64_fma)."""
    v = C.c_double()
    _check(lib.mg_measure_fp64_fma(_stream(stream), C.byref(v)))
    return v.value


def dense_symv_static(X, b, x, stream=None):
    """x = X b (dense symmetric FP64, n <= 65536) without any device allocation: the
    split-K partial sums use the library's static device array (see mg_dense_symv_static)."""
    n = b.numel()
    _check(lib.mg_dense_symv_static(_dev_ptr(X, n * n), n, _dev_ptr(b, n), _dev_ptr(x, n), _stream(stream)))


def solve_batch(hs, bs, xs, rtol=1e-8, maxit=500, stream=None):
    n = len(hs)
    H = (C.c_void_p * n)(*[h._h.value for h in hs])
    B = (C.c_void_p * n)(*[_dev_ptr(b).value for b in bs])
    X = (C.c_void_p * n)(*[_dev_ptr(x).value for x in xs])
    infos = (MgSolveInfo * n)()
    code = lib.mg_solve_batch(C.cast(H, C.c_void_p), C.cast(B, C.c_void_p), C.cast(X, C.c_void_p), n, rtol, maxit,
                              infos, _stream(stream))
    if code not in (OK, ERR_NO_CONVERGENCE):
        raise NnmgError(code, _err(None))
    return [infos[i].as_dict() for i in range(n)]


class Server:
    """Continuous-batching solve server (see mg_server_* in include/nnmg.h)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 8, setup_threads: int = 4):
        self._s = C.c_void_p()
        code = lib.mg_server_create(int(hbm_budget_bytes), max_active, setup_threads, C.byref(self._s))
        if code != OK:
            raise NnmgError(code, lib.mg_server_last_error().decode())

    def submit(self, meshes, degree, b=None, rtol=1e-8, maxit=500, quality_threshold=0.1, tune=False,
               **opts) -> int:
        arr = (MgMesh * len(meshes))()
        keep = []
        for i, m in enumerate(meshes):
            coords = _np(m.coords, np.float64)
            cells = _np(m.cells, np.int32)
            keep += [coords, cells]
            arr[i].dim, arr[i].nv, arr[i].nc = coords.shape[1], coords.shape[0], cells.shape[0]
            arr[i].coords, arr[i].cells = coords.ctypes.data, cells.ctypes.data
        o = default_options(**opts)
        q = MgRequest()
        q.levels = C.cast(arr, C.c_void_p)
        q.L, q.degree, q.quality_threshold = len(meshes), degree, quality_threshold
        q.opt = C.cast(C.pointer(o), C.c_void_p)
        if b is not None:
            bb = _np(b, np.float64)
            keep.append(bb)
            q.b, q.n_b = bb.ctypes.data, bb.size
        q.rtol, q.maxit, q.tune = rtol, maxit, int(bool(tune))
        rid = C.c_int64()
        code = lib.mg_server_submit(self._s, C.byref(q), C.byref(rid))
        if code != OK:
            raise NnmgError(code, lib.mg_server_last_error().decode())
        return rid.value

    def poll(self, rid: int) -> dict:
        r = MgRequestResult()
        _check(lib.mg_server_poll(self._s, rid, C.byref(r)))
        return r.as_dict()

    def wait(self, rid: int, timeout: float = 600.0) -> dict:
        r = MgRequestResult()
        code = lib.mg_server_wait(self._s, rid, timeout, C.byref(r))
        if code not in (OK, ERR_TIMEOUT):
            raise NnmgError(code, "wait failed")
        d = r.as_dict()
        d["timed_out"] = code == ERR_TIMEOUT
        return d

    def fetch(self, rid: int, n: int) -> np.ndarray:
        x = np.zeros(n)
        _check(lib.mg_server_fetch(self._s, rid, x.ctypes.data, n))
        return x

    def stats(self) -> dict:
        st = MgServerStats()
        _check(lib.mg_server_stats(self._s, C.byref(st)))
        return st.as_dict()

    def close(self):
        if self._s:
            lib.mg_server_destroy(self._s)
            self._s = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
