"""Rounding-error bounds for the library's FP32 (mixed-precision) results.

Test infrastructure: the parity bar of an FP32 result of the library, derived from the
arithmetic instead of measured. The FP32 form stores A_l, P_l, R_l, D^{-1} and the
Chebyshev coefficients in FP32 and runs every sparse product, residual and vector update of
the V-cycle in FP32; the patch residuals and solves (explicit FP64 inverses) and the
coarsest solve run in FP64 on FP32 inputs, their results rounded to FP32.

Method: first-order running error analysis on a tape. The library's schedule is replayed in
exact (FP64) arithmetic as a list of linear operations out = sum_j M_j in_j with the exact
matrices M_j; each operation also records a bound rho >= |local rounding error| of its FP32
output (u = 2^-24):
  * a length-m dot product with FP32-stored coefficients: (m + 1) u (|M| |v|)_i (one u for
    the storage, m for the sum, in any summation order); a product or sum rounded once adds
    u times its magnitude; FP64 parts add u64 = 2^-53 terms, the explicit inverses times
    their order and condition number.
To first order the final error is sum_k M_k^tail delta_k, where M_k^tail is the exact map
from operation k's output to the result and |delta_k| <= rho_k. For an output component i,
the adjoint vectors lambda_k = (M_k^tail)^T e_i are computed by one reverse sweep of the tape
(transposed matrices), and
    |error_i| <= sum_k |lambda_k|^T rho_k,
the tightest bound that holds for every sign pattern of the rounding errors. Unlike
bounding each step by the absolute values of its matrices, this keeps the cancellation
inside the exact composite maps (the P2 operators' |I - c D^{-1} A| row sums of 4-10 would
otherwise compound over the cycle). Bounds are computed for chosen components (the ones
with the largest observed error and random ones).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from oracle import smoother

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def _abs(M):
    M = sp.csr_matrix(M, copy=True)
    M.data = np.abs(M.data)
    return M


class Tape:
    """Linear operations out = sum_j c_j M_j in_j on vectors, with a local rounding bound per
    output. A term is (var, M) or (var, M, c); M is a scipy sparse matrix, a dense array, or
    None for the identity; c a scalar (default 1)."""

    def __init__(self):
        self.val = []      # exact value of each variable
        self.rho = []      # local rounding bound of each variable
        self.ops = []      # (out, [(in, M), ...]) in creation order; inputs have no op

    def input(self, v, rho):
        self.val.append(np.asarray(v, dtype=np.float64))
        self.rho.append(np.asarray(rho, dtype=np.float64))
        return len(self.val) - 1

    def op(self, terms, rho_fn):
        """terms: [(var, M or None)]; rho_fn(value) -> local rounding bound of the output."""
        out = None
        for term in terms:
            v, M = term[0], term[1]
            c = term[2] if len(term) > 2 else 1.0
            t = self.val[v] if M is None else M @ self.val[v]
            t = t * c if c != 1.0 else t
            out = t.copy() if out is None else out + t
        self.val.append(out)
        self.rho.append(np.asarray(rho_fn(out), dtype=np.float64))
        self.ops.append((len(self.val) - 1, terms))
        return len(self.val) - 1

    def bound(self, out, comps):
        """First-order bounds on |fl(x) - x| of components comps of variable out."""
        comps = np.asarray(comps)
        k = len(comps)
        lam = {out: np.zeros((len(self.val[out]), k))}
        lam[out][comps, np.arange(k)] = 1.0
        bnd = np.zeros(k)
        op_of = {o: terms for o, terms in self.ops}
        for var in range(out, -1, -1):
            L = lam.pop(var, None)
            if L is None:
                continue
            bnd += np.abs(L).T @ self.rho[var]
            for term in op_of.get(var, ()):
                v, M = term[0], term[1]
                c = term[2] if len(term) > 2 else 1.0
                contrib = np.asarray(L if M is None else M.T @ L)
                if c != 1.0:
                    contrib = contrib * c
                if v in lam:
                    lam[v] += contrib
                else:
                    lam[v] = contrib.copy()
        return bnd


class _Patches:
    """S_c data of one level: K = sum_d E_d X_d E_d^T (block-diagonal, X_d = A[B_d, B_d]^{-1}
    with zero rows and columns on dependent DoFs), the FP64 rounding scale of each block and,
    for the patches applied in FP32 (fp32[d] = 1: FP32 copy of X_d, residual staged in FP32,
    FP32 products and sums), their rows' FP32 scale n_B + 3 (X_d and the residual rounded, n_B
    sums; the result is added in FP64 and rounded as for an FP64 patch)."""

    def __init__(self, A, patches, fp32=None):
        n = A.shape[0]
        rows, cols, vals = [], [], []
        self.mask = np.zeros(n, dtype=bool)
        self.scale = np.zeros(n)       # n_B * kappa_B on the rows of B
        self.scale32 = np.zeros(n)     # n_B + 3 on the rows of an FP32 patch
        blocks = []
        for d, B in enumerate(patches):
            B = np.asarray(B)
            Abb = A[B][:, B].toarray()
            keep = ~smoother.dependent_dofs(Abb)
            Xk = np.linalg.inv(Abb[np.ix_(keep, keep)])
            X = np.zeros_like(Abb)
            X[np.ix_(keep, keep)] = Xk
            kappa = float(np.linalg.norm(Abb[np.ix_(keep, keep)], 1) * np.linalg.norm(Xk, 1))
            r, c = np.meshgrid(B, B, indexing="ij")
            rows.append(r.ravel())
            cols.append(c.ravel())
            vals.append(X.ravel())
            self.mask[B] = True
            self.scale[B] = len(B) * kappa
            if fp32 is not None and fp32[d]:
                self.scale32[B] = len(B) + 3
            blocks.append((B, X))
        self.K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)) \
            if patches else sp.csr_matrix((n, n))
        self.absK = _abs(self.K)


class _Level:
    def __init__(self, lev, cheb_degree, fp32=None):
        self.A = lev.A.tocsr()
        self.absA = _abs(self.A)
        self.m = np.diff(self.A.indptr).astype(np.float64)
        self.dinv = lev.dinv
        self.n = self.A.shape[0]
        self.P = None
        if lev.P is not None:
            self.coef = smoother.chebyshev_coefficients(lev.lmax, lev.lmin, cheb_degree)
            self.D = sp.diags(lev.dinv).tocsr()
            self.DA = (self.D @ self.A).tocsr()
            self.P = lev.P.tocsr()
            self.absP = _abs(self.P)
            self.mP = np.diff(self.P.indptr).astype(np.float64)
            self.R = lev.R.tocsr()
            self.absR = _abs(self.R)
            self.mR = np.diff(self.R.indptr).astype(np.float64)
        self.pt = _Patches(self.A, lev.patches, fp32) if lev.patches else None
        if self.pt is not None:
            self.KA = (self.pt.K @ self.A).tocsr()          # non-zero on the patch rows only
            if self.P is not None:
                self.KAP = (self.KA @ self.P).tocsr()


class Fp32Schedule:
    """Replays the library's FP32 V-cycle schedule (orders sandwich / global_then_local /
    global, nu, Chebyshev degree of the oracle hierarchy H) on a tape."""

    def __init__(self, H, u=U32, fp32=None):
        """fp32: per level, per patch 1 where the library applies the inverse in FP32
        (Hierarchy.export_patch_precision), or None (every patch FP64)."""
        self.H = H
        self.u = u
        self.lv = [_Level(lev, H.cheb_degree, None if fp32 is None else fp32[l]) for l, lev in enumerate(H.levels)]
        Ac = H.levels[-1].A.toarray()
        keep = ~smoother.dependent_dofs(Ac)
        Xk = np.linalg.inv(Ac[np.ix_(keep, keep)])
        self.Xc = np.zeros_like(Ac)
        self.Xc[np.ix_(keep, keep)] = Xk
        self.absXc = np.abs(self.Xc)
        self.kappa_c = float(np.linalg.norm(Ac[np.ix_(keep, keep)], 1) * np.linalg.norm(Xk, 1))

    # ---- steps (t: the tape; variables are tape ids) ----
    def cheb_step(self, t, L, j, x, d, b):
        """r = b - A x; d = cd d + cr D^{-1} r (j = 0: cd = 0, d unused); x + d."""
        u = self.u
        cd, cr = L.coef[j]
        xv = t.val[x]
        crd = np.abs(cr * L.dinv)
        ax_abs = L.absA @ np.abs(xv)
        r = t.val[b] - L.A @ xv
        dprev = t.val[d] if (j > 0) else np.zeros_like(xv)
        terms = [(b, L.D, cr), (x, L.DA, -cr)]
        if j > 0:
            terms.append((d, None, cd))
        # A x (m + 1 roundings incl. the FP32 storage of A), r = b - A x (1), D^{-1} r (2: the
        # FP32 storage of D^{-1} and the product), cr (...) (2), cd d (1), the sum (1)
        dn = t.op(terms, lambda v: u * (crd * ((L.m + 1) * ax_abs + 5.0 * np.abs(r)) + abs(cd) * np.abs(dprev)
                                        + np.abs(v)))
        xo = t.op([(x, None), (dn, None)], lambda v: u * np.abs(v))
        return xo, dn

    def cheb(self, t, L, x, b):
        d = None
        for j in range(len(L.coef)):
            x, d = self.cheb_step(t, L, j, x, d, b)
        return x

    def local(self, t, L, x, b):
        """S_c: x + K (b - A x) with the residual and the solves in FP64, rounded to FP32 on the
        patch rows."""
        u = self.u
        pt = L.pt
        xv, bv = t.val[x], t.val[b]
        fp64 = U64 * pt.scale * (pt.absK @ (np.abs(bv) + L.absA @ np.abs(xv)))
        fp64 = fp64 + u * pt.scale32 * (pt.absK @ np.abs(bv - L.A @ xv))
        return t.op([(x, None), (x, L.KA, -1.0), (b, pt.K)],
                     lambda v: np.where(pt.mask, u * np.abs(v), 0.0) + fp64)

    def residual(self, t, L, x, b):
        u = self.u
        ax_abs = L.absA @ np.abs(t.val[x])
        return t.op([(b, None), (x, -L.A)], lambda v: u * ((L.m + 1) * ax_abs + np.abs(v)))

    def restrict(self, t, L, res):
        u = self.u
        rabs = L.absR @ np.abs(t.val[res])
        return t.op([(res, L.R)], lambda v: u * (L.mR + 1) * rabs)

    def coarse(self, t, bc):
        u = self.u
        bv = t.val[bc]
        fp64 = U64 * len(bv) * self.kappa_c * (self.absXc @ np.abs(bv))
        return t.op([(bc, self.Xc)], lambda v: u * np.abs(v) + fp64)

    def prolong(self, t, L, x, xc):
        u = self.u
        pabs = L.absP @ np.abs(t.val[xc])
        return t.op([(x, None), (xc, L.P)], lambda v: u * ((L.mP + 1) * pabs + np.abs(v)))

    def local_after_prolong(self, t, L, xhat, res, xc, b):
        """The S_c that opens the post-smoothing: r_B = res_B - (A P)_B x_c in FP64 from the
        restriction's FP32 residual, x_B = xhat_B + X r_B rounded to FP32."""
        u = self.u
        pt = L.pt
        xv, bv = t.val[xhat], t.val[b]
        fp64 = U64 * pt.scale * (pt.absK @ (np.abs(bv) + L.absA @ np.abs(xv)))
        fp64 = fp64 + u * pt.scale32 * (pt.absK @ np.abs(bv - L.A @ xv))
        return t.op([(xhat, None), (res, pt.K), (xc, -L.KAP)],
                    lambda v: np.where(pt.mask, u * np.abs(v), 0.0) + fp64)

    # ---- the cycle ----
    def _smooth(self, t, l, x, b, post):
        L = self.lv[l]
        order = self.H.order
        if L.pt is None or order == "global":
            return self.cheb(t, L, x, b)
        if order == "sandwich":
            x = self.local(t, L, x, b)
            x = self.cheb(t, L, x, b)
            return self.local(t, L, x, b)
        if not post:
            x = self.cheb(t, L, x, b)
            return self.local(t, L, x, b)
        x = self.local(t, L, x, b)
        return self.cheb(t, L, x, b)

    def cycle(self, t, b, l=0):
        """z = V b from z = 0 on level l (tape variable of z)."""
        if l == len(self.lv) - 1:
            return self.coarse(t, b)
        L = self.lv[l]
        H = self.H
        x = t.input(np.zeros_like(t.val[b]), np.zeros_like(t.val[b]))
        for _ in range(H.nu):
            x = self._smooth(t, l, x, b, post=False)
        res = self.residual(t, L, x, b)
        bc = self.restrict(t, L, res)
        xc = self.cycle(t, bc, l + 1)
        xh = self.prolong(t, L, x, xc)
        post_local_first = L.pt is not None and H.order != "global"
        for k in range(H.nu):
            if k == 0 and post_local_first:
                xh = self.local_after_prolong(t, L, xh, res, xc, b)
                xh = self.cheb(t, L, xh, b)
                if H.order == "sandwich":
                    xh = self.local(t, L, xh, b)
            else:
                xh = self._smooth(t, l, xh, b, post=True)
        return xh

    # ---- what the ABI entry points compute ----
    def vcycle(self, b, x0):
        """mg_vcycle: x0 + V(b - A x0), the residual in FP64, rounded to FP32 for the cycle, the
        correction added in FP64. Returns (tape, output variable)."""
        t = Tape()
        L = self.lv[0]
        bi = t.input(b, np.zeros_like(b))
        xi = t.input(x0, np.zeros_like(x0))
        axa = L.absA @ np.abs(x0)
        r = t.op([(bi, None), (xi, -L.A)], lambda v: U64 * ((L.m + 1) * axa + np.abs(v)))
        r32 = t.op([(r, None)], lambda v: self.u * np.abs(v))
        z = self.cycle(t, r32)
        x = t.op([(xi, None), (z, None)], lambda v: U64 * np.abs(v))
        return t, x

    def apply(self, l, x):
        """mg_apply_A on a level of the FP32 engine: y = A x with x rounded to FP32."""
        t = Tape()
        L = self.lv[l]
        (xi,) = self._inputs(t, x)
        axa = L.absA @ np.abs(x)
        return t, t.op([(xi, L.A)], lambda v: self.u * (L.m + 1) * axa)

    def _inputs(self, t, *vecs):
        return [t.input(v, self.u * np.abs(v)) for v in vecs]   # FP64 arguments rounded to FP32

    def chebyshev(self, l, b, x0):
        t = Tape()
        bi, xi = self._inputs(t, b, x0)
        return t, self.cheb(t, self.lv[l], xi, bi)

    def local_correction(self, l, b, x0):
        t = Tape()
        bi, xi = self._inputs(t, b, x0)
        return t, self.local(t, self.lv[l], xi, bi)

    def smooth(self, l, b, x0, post=False):
        t = Tape()
        bi, xi = self._inputs(t, b, x0)
        return t, self._smooth(t, l, xi, bi, post)

    def residual_restrict(self, l, b, x0):
        t = Tape()
        bi, xi = self._inputs(t, b, x0)
        L = self.lv[l]
        res = self.residual(t, L, xi, bi)
        return t, res, self.restrict(t, L, res)

    def prolong_correct(self, l, xc, x0):
        t = Tape()
        ci, xi = self._inputs(t, xc, x0)
        return t, self.prolong(t, self.lv[l], xi, ci)


def components(got, ref, k_worst=48, k_random=48, seed=0):
    """The components with the largest error, the largest error relative to |ref|, and random
    ones."""
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref)
    rel = err / (np.abs(ref) + 1e-30 * max(1.0, float(np.abs(ref).max())))
    n = len(ref)
    pick = set(np.argsort(err)[-k_worst:].tolist()) | set(np.argsort(rel)[-k_worst:].tolist())
    pick |= set(np.random.default_rng(seed).choice(n, min(n, k_random), replace=False).tolist())
    return np.array(sorted(pick))


def check(tape, var, got, what="", **kw):
    """|got - exact| <= first-order bound at the chosen components; returns the largest
    error-to-bound ratio seen."""
    ref = tape.val[var]
    comps = components(got, ref, **kw)
    bnd = tape.bound(var, comps)
    err = np.abs(np.asarray(got, dtype=np.float64)[comps] - ref[comps])
    ratio = err / np.maximum(bnd, 1e-300)
    worst = int(np.argmax(ratio))
    assert np.all(err <= bnd), (what, int(comps[worst]), float(err[worst]), float(bnd[worst]))
    return float(ratio.max())
