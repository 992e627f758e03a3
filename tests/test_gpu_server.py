"""The solve server: continuous batching under an HBM budget, results identical alone and
in the mix, budget and slot limits respected (GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2402_12947_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def nnmg():
    from paper_2402_12947_gb300 import build
    build.build()
    from paper_2402_12947_gb300 import nnmg as mod
    return mod


def requests():
    """A small mixed stream: 2D P1/P2 and 3D P1 hierarchies with clusters, random RHS."""
    out = []
    spec = [(2, 32, 1, 3), (2, 64, 2, 3), (3, 8, 1, 2), (2, 64, 1, 3), (2, 32, 2, 3), (3, 12, 1, 3), (2, 128, 1, 4)]
    for k, (dim, n, degree, levels) in enumerate(spec):
        kw = dict(cluster_levels=tuple(range(levels - 1)), n_clusters=2, moves_per_cluster=(1, 2))
        meshes = inputs.hierarchy_meshes(dim, n, levels, 0.2 if dim == 2 else 0.15, 100 + k, **kw)
        nfree = (n - 1) ** dim if degree == 1 else (2 * n - 1) ** dim
        b = inputs.uniform_rhs(nfree, 200 + k)
        out.append((meshes, degree, b))
    return out


OPTS = dict(sell_sigma=1)   # fixed layouts: no timing-dependent choice


# Server requests lay out every operator by the deterministic rule (tune = 0); the same
# hierarchy solved alone gets the rule everywhere from tune_min_nnz = 2^31 - 1.
RULE = dict(tune_min_nnz=2 ** 31 - 1)


@pytest.mark.parametrize("opts,alone_opts", [(OPTS, OPTS), ({}, RULE)], ids=["fixed-sell", "rule"])
def test_results_identical_alone_and_in_the_mix(nnmg, opts, alone_opts):
    reqs = requests()
    alone = []
    for meshes, degree, b in reqs:
        with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, **alone_opts) as H:
            x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
            info = H.solve(torch.from_numpy(b).cuda(), x, rtol=1e-8)
            assert info["converged"]
            alone.append(x.cpu().numpy())
    with nnmg.Server(hbm_budget_bytes=8 << 30, max_active=4, setup_threads=4) as srv:
        ids = [srv.submit(m, d, b=b, rtol=1e-8, **opts) for m, d, b in reqs]
        res = [srv.wait(i) for i in ids]
        xs = [srv.fetch(i, r["n"]) for i, r in zip(ids, res)]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["peak_active"] >= 2
    for r, x, xa in zip(res, xs, alone):
        assert r["status"] == 0 and 0.0 < r["true_rel_residual"] < 1.5e-8
        assert np.array_equal(x, xa)


def test_budget_and_slots(nnmg):
    reqs = requests()[:4]
    with nnmg.Server(hbm_budget_bytes=8 << 30, max_active=1, setup_threads=2) as srv:
        ids = [srv.submit(m, d, b=b, **OPTS) for m, d, b in reqs]
        res = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert all(r["status"] == 0 for r in res)
    assert st["peak_active"] == 1 and st["bytes_in_use"] == 0
    # a budget below one request's estimate: refused with OOM, the server keeps going
    with nnmg.Server(hbm_budget_bytes=1 << 20, max_active=2, setup_threads=1) as srv:
        rid = srv.submit(*reqs[0][:2], b=reqs[0][2], **OPTS)
        r = srv.wait(rid)
        assert r["status"] == nnmg.ERR_OOM
    # a malformed request fails cleanly
    with nnmg.Server(hbm_budget_bytes=8 << 30, max_active=2, setup_threads=1) as srv:
        meshes, degree, b = reqs[0]
        rid = srv.submit(meshes, degree, b=b[:-1])
        assert srv.wait(rid)["status"] == nnmg.ERR_INVALID_ARG
