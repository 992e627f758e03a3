"""GPU parity: every step of the hot path through the C ABI against the CPU oracle.

Bars:
  * FP64 steps and V-cycles: relative max-norm difference <= 1e-10 (TOL64) on the same
    inputs, with the oracle's own operators (mg_setup_csr) and through the geometric set-up
    with identical eigenvalues (mg_setup + lambda_override);
  * FP32 (mixed-precision) V-cycles: the first-order rounding-error bound of the FP32
    schedule at every checked component (tests/_fp32_bound.py);
  * solutions of solves stopped at a relative residual: ||x - x_oracle||_2 <=
    (||b - A x|| + ||b - A x_oracle||) / lambda_min(A), which any two solutions meeting the
    stopping test satisfy (_util.solution_gap_bound); FP64 solves take the oracle's iteration
    count exactly, mixed ones at most one more.
"""
import numpy as np
import pytest

from _fp32_bound import Fp32Schedule, check as check32
from _util import TOL64, case, csr_arrays, fp32_flags, rel_err, solution_gap_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mg, smoother  # noqa: E402

CASES = ["c1_p1", "c1_p2", "c2_p2_128", "cube_p1", "cube_p2"]
ORDERS = ["sandwich", "global_then_local", "global"]


@pytest.fixture(scope="module")
def nnmg():
    from paper_2402_12947_gb300 import build
    build.build()
    from paper_2402_12947_gb300 import nnmg as mod
    assert torch.cuda.is_available()
    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


_lib_cache = {}


def lib_csr(nnmg, name, order="sandwich", precision="fp64"):
    key = ("csr", name, order, precision)
    if key not in _lib_cache:
        _, Ho, _, _ = case(name, order)
        As, Ps, patches, lam = csr_arrays(Ho)
        _lib_cache[key] = nnmg.Hierarchy.from_csr(As, Ps, patches, lam, smoother=order, precision=precision)
    return _lib_cache[key]


def lib_geo(nnmg, name, order="sandwich", precision="fp64"):
    key = ("geo", name, order, precision)
    if key not in _lib_cache:
        meshes, Ho, degree, layers = case(name, order)
        lam = [lv.lmax for lv in Ho.levels[:-1]]
        _lib_cache[key] = nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, smoother=order,
                                                     precision=precision, lambda_override=lam)
    return _lib_cache[key]


def rng_vec(n, seed):
    return np.random.default_rng(seed).uniform(-1, 1, n)


@pytest.mark.parametrize("name", CASES)
def test_apply_A_every_level(nnmg, name):
    _, Ho, _, _ = case(name)
    H = lib_csr(nnmg, name)
    for l, lo in enumerate(Ho.levels):
        x = rng_vec(lo.n, l)
        y = torch.zeros(lo.n, dtype=torch.float64, device="cuda")
        H.apply_A(l, dev(x), y)
        assert rel_err(host(y), lo.A @ x) < TOL64, l


@pytest.mark.parametrize("name", CASES)
def test_chebyshev_and_local_correction(nnmg, name):
    _, Ho, _, _ = case(name)
    H = lib_csr(nnmg, name)
    for l, lo in enumerate(Ho.levels[:-1]):
        b, x0 = rng_vec(lo.n, 10 + l), rng_vec(lo.n, 20 + l)
        x = dev(x0)
        H.chebyshev(l, dev(b), x)
        ref = smoother.chebyshev(lo.A, lo.dinv, b, x0, lo.lmax, lo.lmin, Ho.cheb_degree)
        assert rel_err(host(x), ref) < TOL64, ("cheb", l)
        x = dev(x0)
        H.local_correction(l, dev(b), x)
        ref = lo.local.apply(lo.A, b, x0)
        assert rel_err(host(x), ref) < TOL64, ("local", l)


@pytest.mark.parametrize("name", ["c1_p1", "c2_p2_128", "cube_p2"])
@pytest.mark.parametrize("order", ORDERS)
def test_combined_smoother(nnmg, name, order):
    _, Ho, _, _ = case(name, order)
    H = lib_csr(nnmg, name, order)
    for l, lo in enumerate(Ho.levels[:-1]):
        b, x0 = rng_vec(lo.n, 30 + l), rng_vec(lo.n, 40 + l)
        for post in (False, True):
            x = dev(x0)
            H.smooth(l, dev(b), x, post=post)
            ref = smoother.smooth(lo.A, lo.dinv, b, x0, lo.lmax, lo.lmin, Ho.cheb_degree, lo.local, order, post)
            assert rel_err(host(x), ref) < TOL64, (l, post)


@pytest.mark.parametrize("name", CASES)
def test_transfer_and_coarse_solve(nnmg, name):
    _, Ho, _, _ = case(name)
    H = lib_csr(nnmg, name)
    for l, lo in enumerate(Ho.levels[:-1]):
        nc = Ho.levels[l + 1].n
        b, x0, xc = rng_vec(lo.n, 50 + l), rng_vec(lo.n, 60 + l), rng_vec(nc, 70 + l)
        r = torch.zeros(lo.n, dtype=torch.float64, device="cuda")
        bc = torch.zeros(nc, dtype=torch.float64, device="cuda")
        H.residual_restrict(l, dev(b), dev(x0), r, bc)
        rr = b - lo.A @ x0
        assert rel_err(host(r), rr) < TOL64
        assert rel_err(host(bc), lo.R @ rr) < TOL64
        x = dev(x0)
        H.prolong_correct(l, dev(xc), x)
        assert rel_err(host(x), x0 + lo.P @ xc) < TOL64
    lc = Ho.levels[-1]
    b = rng_vec(lc.n, 80)
    x = torch.zeros(lc.n, dtype=torch.float64, device="cuda")
    H.coarse_solve(dev(b), x)
    assert rel_err(host(x), Ho.coarse.solve(b)) < TOL64


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("setup", ["csr", "geo"])
def test_vcycle(nnmg, name, setup):
    _, Ho, _, _ = case(name)
    H = lib_csr(nnmg, name) if setup == "csr" else lib_geo(nnmg, name)
    n = Ho.levels[0].n
    b, x0 = rng_vec(n, 90), rng_vec(n, 91)
    x = dev(x0)
    H.vcycle(dev(b), x)
    ref = x0 + mg.vcycle(Ho, b - Ho.levels[0].A @ x0)
    assert rel_err(host(x), ref) < TOL64
    # Alg. 1 with the initial guess inside the cycle gives the same iterate
    assert rel_err(host(x), mg.vcycle(Ho, b, x0)) < TOL64


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("graph", [1, 0])
def test_pcg_solve(nnmg, name, graph):
    meshes, Ho, degree, layers = case(name)
    lam = [lv.lmax for lv in Ho.levels[:-1]]
    H = nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, lambda_override=lam, use_graph=graph)
    try:
        n = Ho.levels[0].n
        b = rng_vec(n, 100)
        rtol = 1e-10
        xr, itr, hist, tr = mg.pcg(Ho, b, rtol)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = H.solve(dev(b), x, rtol=rtol, maxit=200)
        assert info["converged"] and info["iterations"] == itr, (info, itr)
        assert abs(info["rel_residual"] - hist[-1]) <= 1e-3 * hist[-1] + 1e-14
        assert info["true_rel_residual"] < 2 * rtol
        A = Ho.levels[0].A
        xh = host(x)
        assert np.linalg.norm(xh - xr) <= solution_gap_bound(A, b, xh, xr)
    finally:
        H.close()


@pytest.mark.parametrize("name", ["c1_p1", "c1_p2", "c2_p2_128", "cube_p1"])
def test_mixed_precision_solve(nnmg, name):
    meshes, Ho, degree, layers = case(name)
    H = lib_geo(nnmg, name, precision="mixed")
    n = Ho.levels[0].n
    b = rng_vec(n, 110)
    rtol = 1e-8
    xr, itr, _, _ = mg.pcg(Ho, b, rtol)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = H.solve(dev(b), x, rtol=rtol, maxit=200)
    assert info["converged"] and info["iterations"] <= itr + 1, (info, itr)
    assert info["true_rel_residual"] < 1.5 * rtol
    xh = host(x)
    A = Ho.levels[0].A
    assert np.linalg.norm(b - A @ xh) < 1.5 * rtol * np.linalg.norm(b)
    # the error against the FP64 oracle's solution, within what the two residuals allow
    assert np.linalg.norm(xh - xr) <= solution_gap_bound(A, b, xh, xr)
    # one FP32 V-cycle against its rounding-error bound around the exact (oracle) cycle
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    H.vcycle(dev(b), z)
    tape, var = Fp32Schedule(Ho, fp32=fp32_flags(H)).vcycle(b, np.zeros(n))
    assert rel_err(tape.val[var], mg.vcycle(Ho, b)) < TOL64
    check32(tape, var, host(z), name)


def test_stationary_multigrid(nnmg):
    _, Ho, _, _ = case("c1_p1")
    H = lib_geo(nnmg, "c1_p1")
    n = Ho.levels[0].n
    b = rng_vec(n, 120)
    xr, itr, hist = mg.stationary(Ho, b, 1e-10)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = H.solve_stationary(dev(b), x, rtol=1e-10, maxit=100)
    assert info["converged"] and info["iterations"] == itr
    xh = host(x)
    assert np.linalg.norm(xh - xr) <= solution_gap_bound(Ho.levels[0].A, b, xh, xr)


def test_edge_cases(nnmg):
    _, Ho, _, _ = case("c1_p1")
    H = lib_geo(nnmg, "c1_p1")
    n = Ho.levels[0].n
    # zero right-hand side: zero solution, no iterations
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    info = H.solve(torch.zeros(n, dtype=torch.float64, device="cuda"), x, rtol=1e-8)
    assert info["converged"] and info["iterations"] == 0 and float(x.abs().max()) == 0.0
    # maxit reached: status and info are reported
    b = rng_vec(n, 130)
    info = H.solve(dev(b), torch.zeros(n, dtype=torch.float64, device="cuda"), rtol=1e-14, maxit=2,
                   raise_on_fail=False)
    assert info["status"] == nnmg.ERR_NO_CONVERGENCE and info["iterations"] == 2 and not info["converged"]
    # the same solve twice is bitwise reproducible (deterministic reductions)
    x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    x2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    H.solve(dev(b), x1, rtol=1e-10)
    H.solve(dev(b), x2, rtol=1e-10)
    assert torch.equal(x1, x2)
    # wrong sizes and types are rejected before any launch
    with pytest.raises(ValueError):
        H.vcycle(dev(b[:-1]), x1)
    with pytest.raises(TypeError):
        H.vcycle(dev(b).float(), x1)


def test_clean_mesh_smoother_reduces_to_chebyshev(nnmg):
    from paper_2402_12947_gb300 import inputs
    from oracle import hierarchy
    meshes = inputs.config_c1(clusters=False)
    Ho = hierarchy.build(meshes, 1, layers=2)
    assert all(len(lv.patches) == 0 for lv in Ho.levels)
    lam = [lv.lmax for lv in Ho.levels[:-1]]
    with nnmg.Hierarchy.from_meshes(meshes, 1, 0.1, patch_layers=2, lambda_override=lam) as H:
        lo = Ho.levels[0]
        b, x0 = rng_vec(lo.n, 140), rng_vec(lo.n, 141)
        xs, xc = dev(x0), dev(x0)
        H.smooth(0, dev(b), xs)
        H.chebyshev(0, dev(b), xc)
        assert torch.equal(xs, xc)


def test_batch_matches_individual_solves(nnmg):
    names = ["c1_p1", "c1_p2", "cube_p1"]
    hs = [lib_geo(nnmg, nm) for nm in names]
    bs = [dev(rng_vec(h.num_dofs(0), 150 + i)) for i, h in enumerate(hs)]
    alone = []
    for h, b in zip(hs, bs):
        x = torch.zeros_like(b)
        h.solve(b, x, rtol=1e-9)
        alone.append(x)
    xs = [torch.zeros_like(b) for b in bs]
    infos = nnmg.solve_batch(hs, bs, xs, rtol=1e-9)
    for a, x, inf in zip(alone, xs, infos):
        assert inf["converged"]
        assert torch.equal(a, x)


@pytest.mark.parametrize("name", ["c1_p1", "c1_p2", "c2_p2_128", "cube_p1"])
def test_device_lanczos_eigenvalues(nnmg, name):
    """lambda_max of D^-1 A (Sec. 3.2) and the adjusted value (Sec. 5), estimated by the
    device Lanczos, agree with the oracle's dense/ARPACK values to 1e-8."""
    meshes, Ho, degree, layers = case(name)
    with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers) as H:
        for l, lo in enumerate(Ho.levels[:-1]):
            lu, la, used = H.eigs(l)
            assert abs(lu - lo.lmax_unadj) < 1e-8 * lo.lmax_unadj, (l, lu, lo.lmax_unadj)
            assert abs(la - lo.lmax_adj) < 1e-8 * lo.lmax_adj, (l, la, lo.lmax_adj)
            assert used == la


@pytest.mark.parametrize("name", ["c1_p2", "c2_p2_128"])
def test_library_numbering_without_reordering(nnmg, name):
    """The same V-cycle and solve with the internal reordering switched off (operators in the
    library's numbering, 32-bit indices) and with it on."""
    meshes, Ho, degree, layers = case(name)
    lam = [lv.lmax for lv in Ho.levels[:-1]]
    n = Ho.levels[0].n
    b, x0 = rng_vec(n, 160), rng_vec(n, 161)
    ref = x0 + mg.vcycle(Ho, b - Ho.levels[0].A @ x0)
    xr, itr, _, _ = mg.pcg(Ho, b, 1e-10)
    for reorder in (0, 1, 2):
        with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, lambda_override=lam,
                                        reorder=reorder) as H:
            x = dev(x0)
            H.vcycle(dev(b), x)
            assert rel_err(host(x), ref) < TOL64, reorder
            xs = torch.zeros(n, dtype=torch.float64, device="cuda")
            info = H.solve(dev(b), xs, rtol=1e-10)
            assert info["iterations"] == itr
            assert np.linalg.norm(host(xs) - xr) <= solution_gap_bound(Ho.levels[0].A, b, host(xs), xr), reorder


def test_time_vcycle_per_level(nnmg):
    """The graph-timed V-cycle from each level: positive, and entering lower adds work."""
    H = lib_geo(nnmg, "c2_p2_128")
    t = [H.time_vcycle(l, reps=5) for l in range(H.num_levels)]
    assert all(x > 0 for x in t)
    assert t[0] > t[-1]
    with pytest.raises(nnmg.NnmgError):
        H.time_vcycle(H.num_levels, reps=1)


@pytest.mark.parametrize("name", ["c1_p2", "c2_p2_128", "cube_p2"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tma_staged_spmv(nnmg, name, precision, monkeypatch):
    """Every level operator on the TMA-staged kernel (bulk copies of slice chunks into shared
    memory; the test hook forces it wherever it fits): the same V-cycle and solve as the oracle
    in FP64, and a converged mixed-precision solve."""
    monkeypatch.setenv("NNMG_FORCE_LAYOUT", "tma")
    meshes, Ho, degree, layers = case(name)
    lam = [lv.lmax for lv in Ho.levels[:-1]]
    n = Ho.levels[0].n
    b, x0 = rng_vec(n, 170), rng_vec(n, 171)
    with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, lambda_override=lam,
                                    precision=precision) as H:
        n1 = Ho.levels[1].n  # level 0's apply goes through the FP64 CG operator; level 1's does not
        v = rng_vec(n1, 172)
        y = torch.zeros(n1, dtype=torch.float64, device="cuda")
        H.apply_A(1, dev(v), y)
        if precision == "fp64":
            assert rel_err(host(y), Ho.levels[1].A @ v) < TOL64
        else:
            tape, var = Fp32Schedule(Ho, fp32=fp32_flags(H)).apply(1, v)
            check32(tape, var, host(y), "apply")
        xs = torch.zeros(n, dtype=torch.float64, device="cuda")
        if precision == "fp64":
            x = dev(x0)
            H.vcycle(dev(b), x)
            assert rel_err(host(x), x0 + mg.vcycle(Ho, b - Ho.levels[0].A @ x0)) < TOL64
            xr, itr, _, _ = mg.pcg(Ho, b, 1e-10)
            info = H.solve(dev(b), xs, rtol=1e-10)
            assert info["iterations"] == itr
            assert np.linalg.norm(host(xs) - xr) <= solution_gap_bound(Ho.levels[0].A, b, host(xs), xr)
        else:
            _, itr, _, _ = mg.pcg(Ho, b, 1e-8)
            info = H.solve(dev(b), xs, rtol=1e-8)
            assert info["converged"] and info["iterations"] <= itr + 1 and info["true_rel_residual"] < 1.5e-8
            x = dev(x0)
            H.vcycle(dev(b), x)
            tape, var = Fp32Schedule(Ho, fp32=fp32_flags(H)).vcycle(b, x0)
            check32(tape, var, host(x), "tma vcycle")


@pytest.mark.parametrize("order,nu,k", [("global_then_local", 1, 2), ("global", 1, 2), ("sandwich", 2, 3),
                                        ("sandwich", 1, 1), ("global_then_local", 2, 1)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vcycle_orders_nu_degree(nnmg, order, nu, k, precision):
    """The whole V-cycle (with its folded launches: the S_c from zero fused with the first
    Chebyshev step, the post-smoothing S_c residual fused with the prolongation) for every
    smoother order, nu = 1, 2 and odd/even Chebyshev degrees, against the oracle cycle with
    the same options."""
    from oracle import hierarchy
    meshes, _, degree, layers = case("c2_p2_128")
    Ho = hierarchy.build(meshes, degree, layers=layers, order=order, nu=nu, cheb_degree=k)
    lam = [lv.lmax for lv in Ho.levels[:-1]]
    n = Ho.levels[0].n
    b, x0 = rng_vec(n, 180), rng_vec(n, 181)
    ref = x0 + mg.vcycle(Ho, b - Ho.levels[0].A @ x0)
    with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, lambda_override=lam, smoother=order,
                                    nu=nu, cheb_degree=k, precision=precision) as H:
        x = dev(x0)
        H.vcycle(dev(b), x)
        if precision == "fp64":
            assert rel_err(host(x), ref) < TOL64
        else:   # the FP32 cycle within its rounding-error bound
            tape, var = Fp32Schedule(Ho, fp32=fp32_flags(H)).vcycle(b, x0)
            check32(tape, var, host(x), (order, nu, k))
        # the solve as well where the local correction is on (without it CG needs a few hundred
        # iterations on these low-quality cells, and rounding moves the count by a few)
        if precision == "fp64" and order != "global":
            xr, itr, _, _ = mg.pcg(Ho, b, 1e-10)
            xs = torch.zeros(n, dtype=torch.float64, device="cuda")
            info = H.solve(dev(b), xs, rtol=1e-10)
            assert info["iterations"] == itr
            assert np.linalg.norm(host(xs) - xr) <= solution_gap_bound(Ho.levels[0].A, b, host(xs), xr)


def test_large_patch_limit_survives_a_later_smaller_hierarchy(nnmg):
    """The shared-memory limit of the patch-solve kernels is per function and process-wide:
    a hierarchy set up later with smaller (but above 48 KB) patches must not lower it under
    an earlier hierarchy with larger ones. Patches of 7000 and 6200 DoFs (56 and 49.6 KB of
    staged residual) on the 128^2 P2 case's fine level, then a V-cycle with the first."""
    from oracle import hierarchy
    _, Ho, _, _ = case("c2_p2_128")
    As, Ps, patches, lam = csr_arrays(Ho)
    big = [[np.arange(7000)]] + [list(p) for p in patches[1:]]
    small = [[np.arange(10000, 16200)]] + [list(p) for p in patches[1:]]
    H1 = nnmg.Hierarchy.from_csr(As, Ps, big, lam)
    H2 = nnmg.Hierarchy.from_csr(As, Ps, small, lam)
    try:
        Hb = hierarchy.from_matrices(As, Ps, big, lam)
        n = Ho.levels[0].n
        b, x0 = rng_vec(n, 190), rng_vec(n, 191)
        x = dev(x0)
        H1.vcycle(dev(b), x)
        assert rel_err(host(x), x0 + mg.vcycle(Hb, b - Hb.levels[0].A @ x0)) < TOL64
        x = dev(x0)
        H2.vcycle(dev(b), x)     # and the later hierarchy still runs
        assert np.all(np.isfinite(host(x)))
    finally:
        H1.close()
        H2.close()


@pytest.mark.parametrize("name", ["c1_p2", "c2_p2_128", "cube_p2"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_small_levels(nnmg, name, precision):
    """The cycle from the first level with at most small_level_dofs DoFs down runs in one
    persistent launch (phases and grid barriers instead of one launch per step): for every
    split point (0 = off, so each level in turn, up to the whole cycle) the V-cycle matches the
    oracle and the solve takes the oracle's iteration count."""
    meshes, Ho, degree, layers = case(name)
    lam = [lv.lmax for lv in Ho.levels[:-1]]
    n = Ho.levels[0].n
    b, x0 = rng_vec(n, 195), rng_vec(n, 196)
    ref = x0 + mg.vcycle(Ho, b - Ho.levels[0].A @ x0)
    rtol = 1e-10 if precision == "fp64" else 1e-8
    xr, itr, _, _ = mg.pcg(Ho, b, rtol)
    sizes = [lv.n for lv in Ho.levels]
    for thr in [0] + sizes[::-1]:
        with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, lambda_override=lam,
                                        precision=precision, small_level_dofs=thr) as H:
            x = dev(x0)
            H.vcycle(dev(b), x)
            if precision == "fp64":
                assert rel_err(host(x), ref) < TOL64, thr
            else:
                tape, var = Fp32Schedule(Ho, fp32=fp32_flags(H)).vcycle(b, x0)
                check32(tape, var, host(x), thr)
            xs = torch.zeros(n, dtype=torch.float64, device="cuda")
            info = H.solve(dev(b), xs, rtol=rtol)
            ok = info["iterations"] == itr if precision == "fp64" else info["iterations"] <= itr + 1
            assert info["converged"] and ok, (thr, info, itr)
            xh = host(xs)
            assert np.linalg.norm(xh - xr) <= solution_gap_bound(Ho.levels[0].A, b, xh, xr)


def test_persistent_batch_matches_alone_and_oracle(nnmg):
    """mg_solve_batch with hierarchies whose whole solve runs persistently (small_level_dofs
    >= n_0): one cooperative launch per precision iterates every problem's MG-PCG (phases of
    all problems merged, a stopped problem idle) and the others run their graphs meanwhile.
    Each result is bitwise the one of the same hierarchy solved alone, whatever else is in
    the batch, and matches the oracle (FP64: the oracle's iteration count)."""
    names = ["c1_p1", "c1_p2", "cube_p1", "cube_p2", "c2_p2_128"]
    hs, bs, refs = [], [], []
    big = 1 << 30
    for k, nm in enumerate(names):
        meshes, Ho, degree, layers = case(nm)
        lam = [lv.lmax for lv in Ho.levels[:-1]]
        prec = "fp64" if k % 2 == 0 else "mixed"
        hs.append(nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, lambda_override=lam,
                                             precision=prec, small_level_dofs=big))
        b = rng_vec(Ho.levels[0].n, 500 + k)
        bs.append(dev(b))
        refs.append((Ho, b, prec))
    hs.append(lib_geo(nnmg, "c1_p1"))   # a graph-path hierarchy in the same call
    bs.append(dev(rng_vec(case("c1_p1")[1].levels[0].n, 510)))
    try:
        alone = []
        for h, b in zip(hs, bs):
            x = torch.zeros_like(b)
            h.solve(b, x, rtol=1e-9)
            alone.append(x)
        for order in (list(range(len(hs))), list(range(len(hs)))[::-1], [0, 2]):
            xs = [torch.zeros_like(bs[i]) for i in order]
            infos = nnmg.solve_batch([hs[i] for i in order], [bs[i] for i in order], xs, rtol=1e-9)
            for i, x, inf in zip(order, xs, infos):
                assert inf["converged"]
                assert torch.equal(alone[i], x), (i, order)
        for (Ho, b, prec), x in zip(refs, alone):
            xr, itr, _, _ = mg.pcg(Ho, b, 1e-9)
            xh = host(x)
            assert np.linalg.norm(xh - xr) <= solution_gap_bound(Ho.levels[0].A, b, xh, xr)
    finally:
        for h in hs[:-1]:
            h.close()
