"""GPU parity of the multicolour symmetric Gauss-Seidel global smoother (the paper's SGS,
Sec. 3.1 and Sec. 6, in its parallel multicolour form) against the oracle: one sweep on
every smoothed level, the V-cycle with S_c around SGS, MG-PCG iteration counts, and the
mixed-precision solve."""
import numpy as np
import pytest

from _util import solution_gap_bound, CASES, TOL64, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import hierarchy, mg, smoother  # noqa: E402

NAMES = ["c1_p1", "c1_p2", "c2_p2_128", "cube_p1", "cube_p2"]
_cache = {}


@pytest.fixture(scope="module")
def nnmg():
    from paper_2402_12947_gb300 import build
    build.build()
    from paper_2402_12947_gb300 import nnmg as mod
    assert torch.cuda.is_available()
    return mod


def sgs_case(name):
    if name not in _cache:
        make, degree, layers = CASES[name]
        meshes = make()
        Ho = hierarchy.build(meshes, degree, layers=layers, smoother_kind="sgs")
        _cache[name] = (meshes, Ho, degree, layers)
    return _cache[name]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rng(n, seed):
    return np.random.default_rng(seed).uniform(-1, 1, n)


@pytest.mark.parametrize("name", NAMES)
def test_sweep_and_vcycle(nnmg, name):
    meshes, Ho, degree, layers = sgs_case(name)
    with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, global_smoother="sgs") as H:
        for l, lo in enumerate(Ho.levels[:-1]):
            assert np.array_equal(H.export_colouring(l), lo.colour), l
            b, x0 = rng(lo.n, 10 + l), rng(lo.n, 20 + l)
            x = dev(x0)
            H.sgs(l, dev(b), x)
            ref = smoother.multicolour_sgs(lo.A, lo.dinv, b, x0, lo.colour)
            assert rel_err(host(x), ref) < TOL64, l
            x = dev(x0)
            H.smooth(l, dev(b), x)
            ref = smoother.smooth(lo.A, lo.dinv, b, x0, 0, 0, 0, lo.local, "sandwich", False, kind="sgs",
                                  colour=lo.colour)
            assert rel_err(host(x), ref) < TOL64, l
        n = Ho.levels[0].n
        b, x0 = rng(n, 30), rng(n, 31)
        x = dev(x0)
        H.vcycle(dev(b), x)
        assert rel_err(host(x), mg.vcycle(Ho, b, x0)) < TOL64


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("graph", [1, 0])
def test_pcg(nnmg, name, graph):
    meshes, Ho, degree, layers = sgs_case(name)
    n = Ho.levels[0].n
    b = rng(n, 40)
    xr, itr, hist, _ = mg.pcg(Ho, b, 1e-10)
    with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, global_smoother="sgs",
                                    use_graph=graph) as H:
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = H.solve(dev(b), x, rtol=1e-10, maxit=200)
        assert info["converged"] and info["iterations"] == itr, (info, itr)
        assert info["true_rel_residual"] < 2e-10
        xh = host(x)
        assert np.linalg.norm(xh - xr) <= solution_gap_bound(Ho.levels[0].A, b, xh, xr)


@pytest.mark.parametrize("name", ["c1_p2", "c2_p2_128", "cube_p1"])
def test_mixed(nnmg, name):
    meshes, Ho, degree, layers = sgs_case(name)
    n = Ho.levels[0].n
    b = rng(n, 50)
    _, itr, _, _ = mg.pcg(Ho, b, 1e-8)
    with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, global_smoother="sgs",
                                    precision="mixed") as H:
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        info = H.solve(dev(b), x, rtol=1e-8, maxit=200)
        assert info["converged"] and info["iterations"] <= itr + 1, (info, itr)
        xh = host(x)
        assert np.linalg.norm(b - Ho.levels[0].A @ xh) < 1.5e-8 * np.linalg.norm(b)


def test_wrong_smoother_calls_rejected(nnmg):
    meshes, Ho, degree, layers = sgs_case("c1_p1")
    n = Ho.levels[0].n
    with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, patch_layers=layers, global_smoother="sgs") as H:
        with pytest.raises(nnmg.NnmgError):
            H.chebyshev(0, dev(rng(n, 1)), dev(rng(n, 2)))
