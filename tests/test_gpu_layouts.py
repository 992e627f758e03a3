"""Every SpMV layout the autotuner can choose, forced on every operator, against the oracle.

The autotuner keeps, per operator, the fastest of several SELL / CSR-vector layouts (row
loops with steps of four or eight, 1, 2 or 4 lanes per row, sorting windows, L2 prefetch
distances) with 16- or 32-bit column indices, so a timing-picked layout alone would leave most
kernel instantiations untested. NNMG_FORCE_LAYOUT=<name> gives every operator of a hierarchy
that layout; each one must reproduce Alg. 1's V-cycle and the MG-PCG solve of Sec. 6.2. The
case is the 2D P2 family of the benchmark at 192^2 (146,689 fine DoFs, 4 levels): its fine
operator's slices span more than 2^16 columns, so there the kernels run on 32-bit column
indices, as on the 1024^2 benchmark, and on the coarser levels on 16-bit offsets.

Bars: FP64 at 1e-10 (steps, V-cycle), FP32 within the first-order rounding-error bound of the
FP32 schedule (tests/_fp32_bound.py), solutions within the gap that the two residuals allow
(_util.solution_gap_bound), FP64 iteration counts equal to the oracle's, mixed ones at most
one more.
"""
import numpy as np
import pytest

from _fp32_bound import Fp32Schedule, check as check32
from _util import TOL64, case, fp32_flags, rel_err, solution_gap_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mg  # noqa: E402

NAME = "c2_p2_192"
LAYOUTS = ["s1", "s1p", "s1q", "s256", "s256p", "s256q", "s2048q", "s1x2p", "s1x4p", "s256x2p", "s256x4p",
           "v4", "v8", "v16", "v32", "s1qf4864", "s1f9728", "s256qf19456", "s1pf2432", "tma"]


@pytest.fixture(scope="module")
def nnmg():
    from paper_2402_12947_gb300 import build
    build.build()
    from paper_2402_12947_gb300 import nnmg as mod
    return mod


_ref = {}


def reference():
    """Oracle hierarchy, inputs, exact V-cycle and the oracle's PCG solutions (cached)."""
    if not _ref:
        meshes, Ho, degree, layers = case(NAME)
        n = Ho.levels[0].n
        b = np.random.default_rng(200).uniform(-1, 1, n)
        x0 = np.random.default_rng(201).uniform(-1, 1, n)
        _ref.update(meshes=meshes, Ho=Ho, degree=degree, layers=layers, b=b, x0=x0,
                    vc=x0 + mg.vcycle(Ho, b - Ho.levels[0].A @ x0),
                    pcg10=mg.pcg(Ho, b, 1e-10), pcg8=mg.pcg(Ho, b, 1e-8))
    return _ref


_sched = {}


def schedule(H):
    """The FP32 schedule with the library's per-patch precision (identical in every forced
    layout: it depends on the patch blocks only)."""
    flags = fp32_flags(H)
    key = tuple(tuple(f.tolist()) for f in flags)
    if key not in _sched:
        _sched[key] = Fp32Schedule(reference()["Ho"], fp32=flags)
    return _sched[key]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_case_has_32_bit_fine_level():
    Ho = reference()["Ho"]
    A = Ho.levels[0].A
    wide = 0
    for s in range(0, A.shape[0], 32):
        a, e = A.indptr[s], A.indptr[min(A.shape[0], s + 32)]
        if e > a and A.indices[a:e].max() - A.indices[a:e].min() > 65535:
            wide += e - a
    assert A.shape[0] > 65536 and wide > A.nnz // 2     # the 32-bit index layout on the fine level
    assert all(lv.n < 65536 for lv in Ho.levels[1:])    # 16-bit offsets below


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forced_layout(nnmg, layout, precision, monkeypatch):
    monkeypatch.setenv("NNMG_FORCE_LAYOUT", layout)
    R = reference()
    Ho, b, x0 = R["Ho"], R["b"], R["x0"]
    n = Ho.levels[0].n
    lam = [lv.lmax for lv in Ho.levels[:-1]]
    with nnmg.Hierarchy.from_meshes(R["meshes"], R["degree"], 0.1, patch_layers=R["layers"], lambda_override=lam,
                                    precision=precision) as H:
        # y = A x on every level (level 0 is the FP64 operator of the CG recurrence in both forms)
        for l, lo in enumerate(Ho.levels):
            v = np.random.default_rng(210 + l).uniform(-1, 1, lo.n)
            y = torch.zeros(lo.n, dtype=torch.float64, device="cuda")
            H.apply_A(l, dev(v), y)
            if precision == "fp64" or l == 0:
                assert rel_err(host(y), lo.A @ v) < TOL64, (layout, l)
            else:
                tape, var = schedule(H).apply(l, v)
                check32(tape, var, host(y), (layout, l))
        # one V-cycle from x0 (every smoothing, transfer and correction kernel of the layout)
        x = dev(x0)
        H.vcycle(dev(b), x)
        if precision == "fp64":
            assert rel_err(host(x), R["vc"]) < TOL64, layout
        else:
            tape, var = schedule(H).vcycle(b, x0)
            check32(tape, var, host(x), layout)
        # the solve (the CG product q = A p and its reduction run on the forced layout too)
        rtol = 1e-10 if precision == "fp64" else 1e-8
        xr, itr, _, _ = R["pcg10"] if precision == "fp64" else R["pcg8"]
        xs = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = H.solve(dev(b), xs, rtol=rtol, maxit=200)
        if precision == "fp64":
            assert info["converged"] and info["iterations"] == itr, (layout, info, itr)
        else:
            assert info["converged"] and info["iterations"] <= itr + 1, (layout, info, itr)
        xh = host(xs)
        A = Ho.levels[0].A
        assert np.linalg.norm(b - A @ xh) <= 1.5 * rtol * np.linalg.norm(b)
        assert np.linalg.norm(xh - xr) <= solution_gap_bound(A, b, xh, xr), layout


def test_unknown_forced_layout_is_rejected(nnmg, monkeypatch):
    monkeypatch.setenv("NNMG_FORCE_LAYOUT", "s1z")
    meshes, Ho, degree, layers = case("c1_p1")
    lam = [lv.lmax for lv in Ho.levels[:-1]]
    with pytest.raises(nnmg.NnmgError):
        nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, lambda_override=lam)
