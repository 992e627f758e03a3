"""Pins of the FP32 rounding-error bounds (tests/_fp32_bound.py) used as the parity bars of
the library's mixed-precision results, on the CPU.

1. The exact values replayed on the tape equal the oracle's (the schedule is the oracle's
   V-cycle, Alg. 1 with the combined smoother of Sec. 4.2).
2. An independent FP32 emulation of the schedule (NumPy/SciPy in float32: FP32 storage of
   the operators, FP32 sums; FP64 patch and coarsest solves rounded to FP32) stays within the
   bounds at every checked component, for every smoother order: the bounds are not too tight.
3. The bounds are not vacuous: a single step's bound stays below 1e-5 of the result's size;
   a V-cycle's, dominated by the worst case (m + 1) u |A||x| of the FP32 fine-level residual
   b - A x after the pre-smoothing (which cancels), below 5e-2; and a planted mistake in the
   emulation (one patch skipped; the last entry of every row dropped from one level's
   Chebyshev product) breaks them.
"""
import numpy as np
import pytest

from _fp32_bound import Fp32Schedule, check
from _util import case
from oracle import hierarchy, mg, smoother

f32 = np.float32


def emulate_vcycle(H, b, x0, plant=None, fp32_patches=False):
    """mg_vcycle's arithmetic in float32 with FP64 patch/coarse solves (the library's mixed form).
    plant: None, "skip_patch" (level 0's first patch gets no correction) or "drop_last" (the
    Chebyshev SpMV of level 1 skips the last entry of every row, a loop-bound mistake).
    fp32_patches: every patch applies an FP32 copy of its inverse to the FP32-rounded residual
    in FP32 arithmetic, the result added in FP64 and rounded to FP32."""
    L = len(H.levels)
    A32 = [lv.A.astype(f32) for lv in H.levels]
    Acheb = list(A32)
    if plant == "drop_last":
        M = Acheb[1].copy()
        M.data[M.indptr[1:] - 1] = 0.0
        Acheb[1] = M
    P32 = [lv.P.astype(f32) if lv.P is not None else None for lv in H.levels]
    R32 = [lv.R.astype(f32) if lv.R is not None else None for lv in H.levels]
    D32 = [lv.dinv.astype(f32) for lv in H.levels]
    Ainv = {}

    def X(l, B):
        key = (l, tuple(B))
        if key not in Ainv:
            Ainv[key] = smoother.DirectSolver(H.levels[l].A[B][:, B].toarray())
        return Ainv[key]

    def solve(l, B, r):
        if not fp32_patches:
            return X(l, B).solve(r)
        key = ("32", l, tuple(B))
        if key not in Ainv:
            Ainv[key] = np.linalg.inv(H.levels[l].A[B][:, B].toarray()).astype(f32)
        return (Ainv[key] @ r.astype(f32)).astype(np.float64)

    def patches(l):
        ps = H.levels[l].patches
        return ps[1:] if (plant == "skip_patch" and l == 0) else ps

    def local(l, x, b):
        r = b.astype(np.float64) - H.levels[l].A @ x.astype(np.float64)
        x = x.copy()
        for B in patches(l):
            x[B] = (x[B].astype(np.float64) + solve(l, B, r[B])).astype(f32)
        return x

    def cheb(l, x, b):
        d = np.zeros_like(x)
        for j, (cd, cr) in enumerate(smoother.chebyshev_coefficients(H.levels[l].lmax, H.levels[l].lmin,
                                                                     H.cheb_degree)):
            r = b - Acheb[l] @ x
            t = D32[l] * r
            d = f32(cr) * t if j == 0 else f32(cd) * d + f32(cr) * t
            x = x + d
        return x

    def smooth(l, x, b, post):
        has = len(H.levels[l].patches) > 0 and H.order != "global"
        if not has:
            return cheb(l, x, b)
        if H.order == "sandwich":
            return local(l, cheb(l, local(l, x, b), b), b)
        if not post:
            return local(l, cheb(l, x, b), b)
        return cheb(l, local(l, x, b), b)

    def cycle(l, b):
        if l == L - 1:
            return (H.coarse.solve(b.astype(np.float64))).astype(f32)
        x = np.zeros_like(b)
        for _ in range(H.nu):
            x = smooth(l, x, b, False)
        res = b - A32[l] @ x
        xc = cycle(l + 1, R32[l] @ res)
        xh = x + P32[l] @ xc
        for k in range(H.nu):
            if k == 0 and len(H.levels[l].patches) > 0 and H.order != "global":
                # S_c from the residual formed at the prolongation: res - (A P) x_c in FP64
                rb = res.astype(np.float64) - (H.levels[l].A @ H.levels[l].P) @ xc.astype(np.float64)
                xh = xh.copy()
                for B in patches(l):
                    xh[B] = (xh[B].astype(np.float64) + solve(l, B, rb[B])).astype(f32)
                xh = cheb(l, xh, b)
                if H.order == "sandwich":
                    xh = local(l, xh, b)
            else:
                xh = smooth(l, xh, b, True)
        return xh

    r = b - H.levels[0].A @ x0
    return x0 + cycle(0, r.astype(f32)).astype(np.float64)


@pytest.mark.parametrize("name,order", [("c1_p1", "sandwich"), ("c1_p2", "sandwich"), ("c2_p2_128", "sandwich"),
                                        ("c1_p2", "global_then_local"), ("c1_p2", "global"), ("cube_p2", "sandwich")])
def test_fp32_emulation_within_bounds(name, order):
    _, Ho, _, _ = case(name, order)
    n = Ho.levels[0].n
    b = np.random.default_rng(1).uniform(-1, 1, n)
    x0 = np.random.default_rng(2).uniform(-1, 1, n)
    sch = Fp32Schedule(Ho)
    tape, var = sch.vcycle(b, x0)
    ref = x0 + mg.vcycle(Ho, b - Ho.levels[0].A @ x0)
    # explicit inverses here, Cholesky in the oracle: equal up to kappa u64 on the patch blocks
    assert np.max(np.abs(tape.val[var] - ref)) <= 1e-10 * np.max(np.abs(ref))
    got = emulate_vcycle(Ho, b, x0)
    ratio = check(tape, var, got, name)
    assert ratio > 1e-3          # the emulation's error is a visible fraction of the bound
    comps = np.arange(0, n, max(1, n // 64))
    assert np.max(tape.bound(var, comps)) < 5e-2 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", ["c1_p2", "c2_p2_128", "cube_p2"])
def test_fp32_patch_inverses_within_bounds(name):
    """Every patch applied in FP32 (the mixed form's well-conditioned patches): the emulation
    within the bound of the schedule told so (n_B + 3 roundings of |X| |r| per patch row)."""
    _, Ho, _, _ = case(name)
    n = Ho.levels[0].n
    b = np.random.default_rng(6).uniform(-1, 1, n)
    x0 = np.zeros(n)
    flags = [np.ones(len(lv.patches), dtype=np.int32) for lv in Ho.levels]
    tape, var = Fp32Schedule(Ho, fp32=flags).vcycle(b, x0)
    check(tape, var, emulate_vcycle(Ho, b, x0, fp32_patches=True), name)


def test_fp32_bounds_nu2_degree3():
    meshes, _, degree, layers = case("c1_p2")
    Ho = hierarchy.build(meshes, degree, layers=layers, nu=2, cheb_degree=3)
    n = Ho.levels[0].n
    b = np.random.default_rng(3).uniform(-1, 1, n)
    x0 = np.zeros(n)
    tape, var = Fp32Schedule(Ho).vcycle(b, x0)
    check(tape, var, emulate_vcycle(Ho, b, x0), "nu2k3")


@pytest.mark.parametrize("plant", ["skip_patch", "drop_last"])
def test_fp32_bound_catches_a_planted_mistake(plant):
    _, Ho, _, _ = case("c1_p2")
    n = Ho.levels[0].n
    b = np.random.default_rng(4).uniform(-1, 1, n)
    x0 = np.zeros(n)
    tape, var = Fp32Schedule(Ho).vcycle(b, x0)
    check(tape, var, emulate_vcycle(Ho, b, x0), "clean")
    with pytest.raises(AssertionError):
        check(tape, var, emulate_vcycle(Ho, b, x0, plant=plant), plant)


def test_single_step_bounds():
    """Chebyshev application, S_c, residual + restriction and prolongation: FP32 emulations
    within the bounds of the corresponding tape (level 0 and 1 of the 128^2 P2 case)."""
    _, Ho, _, _ = case("c2_p2_128")
    sch = Fp32Schedule(Ho)
    rng = np.random.default_rng(5)
    for l in (0, 1):
        lv = Ho.levels[l]
        A32 = lv.A.astype(f32)
        b = rng.uniform(-1, 1, lv.n)
        x0 = rng.uniform(-1, 1, lv.n)
        b32, x32 = b.astype(f32), x0.astype(f32)
        # Chebyshev (degree 2)
        x, d = x32.copy(), np.zeros(lv.n, dtype=f32)
        for j, (cd, cr) in enumerate(smoother.chebyshev_coefficients(lv.lmax, lv.lmin, Ho.cheb_degree)):
            t = lv.dinv.astype(f32) * (b32 - A32 @ x)
            d = f32(cr) * t if j == 0 else f32(cd) * d + f32(cr) * t
            x = x + d
        tape, var = sch.chebyshev(l, b, x0)
        check(tape, var, x, ("cheb", l))
        comps = np.arange(0, lv.n, max(1, lv.n // 64))
        assert np.max(tape.bound(var, comps)) < 1e-5 * np.max(np.abs(tape.val[var]))
        # residual + restriction
        res = b32 - A32 @ x32
        bc = lv.R.astype(f32) @ res
        tape, rv, bv = sch.residual_restrict(l, b, x0)
        check(tape, rv, res, ("res", l))
        check(tape, bv, bc, ("restrict", l))
        # prolongation
        xc = rng.uniform(-1, 1, Ho.levels[l + 1].n)
        xp = x32 + lv.P.astype(f32) @ xc.astype(f32)
        tape, pv = sch.prolong_correct(l, xc, x0)
        check(tape, pv, xp, ("prolong", l))
        # S_c
        r = b32.astype(np.float64) - lv.A @ x32.astype(np.float64)
        xs = x32.copy()
        for B in lv.patches:
            xs[B] = (xs[B].astype(np.float64) + smoother.DirectSolver(lv.A[B][:, B].toarray()).solve(r[B])).astype(f32)
        tape, sv = sch.local_correction(l, b, x0)
        check(tape, sv, xs, ("local", l))
