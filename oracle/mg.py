"""V-cycle, MG-preconditioned CG and stationary MG (oracle; test infrastructure only).

Alg. 1 (V-cycle): on each level l < L pre-smooth nu times, form b_{l+1} = P_l^T (b_l -
A_l u_l), recurse, solve directly on the coarsest level, then u_l += P_l u_{l+1} and
post-smooth nu times. Reading: the coarse unknown starts from u_{l+1} = 0 (the printed
u_{l+1} = P_l^T u_l is inconsistent with a residual-correction cycle), and the coarse
operators A_{l+1} = P^T A P are built once at setup, not per cycle.

Sec. 6.2: multigrid as a preconditioner for CG, one V-cycle per iteration. Standard
PCG from x_0 = 0; it stops when the l2 norm of the recurrence residual relative to
||b||_2 falls to rtol (Sec. 6: relative residual in the l2 norm), and the iteration count
is the number of CG updates (= V-cycle applications). Sec. 6.1 uses multigrid as a
stationary solver: repeated V-cycles until ||b - A x|| / ||b|| <= rtol.

Pinned by tests/test_oracle_mg.py: P = I two-level cycle with exact coarse solve is
exact; the V-cycle operator is symmetric; PCG agrees with a sparse direct solve; the
local correction restores the iteration count of the high-quality hierarchy.
"""
from __future__ import annotations

import numpy as np

from .hierarchy import Hierarchy
from .smoother import smooth


def vcycle(H: Hierarchy, b: np.ndarray, x: np.ndarray | None = None, l: int = 0) -> np.ndarray:
    lev = H.levels[l]
    if l == H.L - 1:
        return H.coarse.solve(b)
    x = np.zeros_like(b) if x is None else x.copy()
    for _ in range(H.nu):
        x = smooth(lev.A, lev.dinv, b, x, lev.lmax, lev.lmin, H.cheb_degree, lev.local, H.order, post=False,
                   kind=H.smoother_kind, colour=lev.colour)
    r = b - lev.A @ x
    bc = lev.R @ r
    xc = vcycle(H, bc, None, l + 1)
    x = x + lev.P @ xc
    for _ in range(H.nu):
        x = smooth(lev.A, lev.dinv, b, x, lev.lmax, lev.lmin, H.cheb_degree, lev.local, H.order, post=True,
                   kind=H.smoother_kind, colour=lev.colour)
    return x


def pcg(H: Hierarchy, b: np.ndarray, rtol: float, maxit: int = 500):
    """Returns (x, iterations, relative residual history, true final relative residual)."""
    A = H.levels[0].A
    bnorm = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, [0.0], 0.0
    r = b.copy()
    hist = [1.0]
    z = vcycle(H, r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < maxit:
        q = A @ p
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rel = float(np.linalg.norm(r)) / bnorm
        hist.append(rel)
        if rel <= rtol:
            break
        z = vcycle(H, r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    true_rel = float(np.linalg.norm(b - A @ x)) / bnorm
    return x, it, hist, true_rel


def stationary(H: Hierarchy, b: np.ndarray, rtol: float, maxit: int = 500, x0=None):
    A = H.levels[0].A
    bnorm = float(np.linalg.norm(b))
    x = np.zeros_like(b) if x0 is None else x0.copy()
    hist = [float(np.linalg.norm(b - A @ x)) / bnorm]
    it = 0
    while hist[-1] > rtol and it < maxit:
        x = vcycle(H, b, x)
        it += 1
        hist.append(float(np.linalg.norm(b - A @ x)) / bnorm)
    return x, it, hist
