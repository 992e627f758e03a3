"""GPU parity of the linear elasticity path (Sec. 6.3): vector P1/P2 on the clamped lattice
with sliver clusters, Chebyshev and multicolour SGS global smoothers (two applications per
side, as in the paper's elasticity runs), against the oracle."""
import numpy as np
import pytest

from _util import TOL64, rel_err, solution_gap_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import elasticity, hierarchy, mg  # noqa: E402
from paper_2402_12947_gb300 import inputs  # noqa: E402

CASES = {"p1": ("lattice", (4, 2, 1), 1), "p2": ("lattice", (2, 1), 2), "dumbbell_p1": ("dumbbell", (4, 2), 1)}
_cache = {}


@pytest.fixture(scope="module")
def nnmg():
    from paper_2402_12947_gb300 import build
    build.build()
    from paper_2402_12947_gb300 import nnmg as mod
    assert torch.cuda.is_available()
    return mod


def lattice(name, kind):
    key = (name, kind)
    if key not in _cache:
        geo, ns, degree = CASES[name]
        make = inputs.config_lattice if geo == "lattice" else inputs.config_dumbbell
        ms, masks = make(ns=ns, n_clusters=3)
        Ho = hierarchy.build(ms, degree, pde="elasticity", dirichlet_masks=masks, smoother_kind=kind, nu=2)
        _cache[key] = (ms, masks, degree, Ho)
    return _cache[key]


def parity_tol(Ho):
    """FP64 parity bar for a V-cycle: the oracle solves each patch block and the coarsest
    matrix by Cholesky, the library applies explicit inverses. Both are backward stable,
    so each solve's forward error is bounded by a small multiple of kappa * u (u = 2^-53)
    and the two may differ by that much: bar = max(1e-10, 8 kappa_max u) over the blocks."""
    u = 2.0 ** -53
    kap = [np.linalg.cond(Ho.levels[-1].A.toarray())]
    for lv in Ho.levels:
        kap += [np.linalg.cond(lv.A[p][:, p].toarray()) for p in lv.patches]
    return max(TOL64, 8.0 * max(kap) * u)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def traction(ms, Ho):
    """Sec. 6.3 loads: traction (1e3, 0, 0) on x = 6 plus the body force (0, 0, -1e3)."""
    from oracle import fem
    lo = Ho.levels[0]
    b = elasticity.traction_load_full(ms[0].coords, ms[0].cells, lo.dm, [1e3, 0, 0], 0, 6.0)
    b = b + np.stack([fem.load_vector_full(ms[0].coords, ms[0].cells, lo.dm, fc) for fc in (0.0, 0.0, -1e3)],
                     axis=1).ravel()
    return b[elasticity.free_vector_dofs(lo.dm)]


def make(nnmg, ms, masks, degree, Ho, kind, **kw):
    opts = dict(pde="elasticity", dirichlet_masks=masks, global_smoother=kind, nu=2, **kw)
    if kind == "chebyshev":
        opts["lambda_override"] = [lv.lmax for lv in Ho.levels[:-1]]
    return nnmg.Hierarchy.from_meshes(ms, degree, 0.1, **opts)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("kind", ["chebyshev", "sgs"])
def test_vcycle_and_pcg(nnmg, name, kind):
    ms, masks, degree, Ho = lattice(name, kind)
    n = Ho.levels[0].n
    rng = np.random.default_rng(7)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    with make(nnmg, ms, masks, degree, Ho, kind) as H:
        x = dev(x0)
        H.vcycle(dev(b), x)
        assert rel_err(host(x), mg.vcycle(Ho, b, x0)) < parity_tol(Ho)
        bt = traction(ms, Ho)
        assert rel_err(H.load_traction(0, 6.0, [1e3, 0, 0]) + H.load_body([0.0, 0.0, -1e3]), bt) < 1e-13
        xr, itr, _, _ = mg.pcg(Ho, bt, 1e-10)
        xs = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = H.solve(dev(bt), xs, rtol=1e-10, maxit=300)
        assert info["converged"] and info["iterations"] == itr, (info, itr)
        xh = host(xs)
        assert np.linalg.norm(xh - xr) <= solution_gap_bound(Ho.levels[0].A, bt, xh, xr)


@pytest.mark.parametrize("kind", ["chebyshev", "sgs"])
def test_mixed_precision(nnmg, kind):
    ms, masks, degree, Ho = lattice("p1", kind)
    bt = traction(ms, Ho)
    _, itr, _, _ = mg.pcg(Ho, bt, 1e-8)
    with make(nnmg, ms, masks, degree, Ho, kind, precision="mixed") as H:
        x = torch.zeros(bt.size, dtype=torch.float64, device="cuda")
        info = H.solve(dev(bt), x, rtol=1e-8, maxit=300)
        assert info["converged"] and info["iterations"] <= itr + 1, (info, itr)
        xh = host(x)
        assert np.linalg.norm(bt - Ho.levels[0].A @ xh) < 1.5e-8 * np.linalg.norm(bt)
