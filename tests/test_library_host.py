"""The C-ABI library on the host (no GPU): it loads, exports every declared symbol, and
its C++ set-up (assembly, quality, patches, transfer, Galerkin, eigenvalues) matches the
oracle; error codes for invalid input."""
import ctypes
import os
import re

import numpy as np
import pytest

from _util import case, csr_arrays, rel_err, to_csr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nnmg():
    from paper_2402_12947_gb300 import build
    build.build()
    from paper_2402_12947_gb300 import nnmg as mod
    return mod


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nnmg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(nnmg):
    names = declared_functions()
    assert len(names) >= 25
    lib = ctypes.CDLL(nnmg.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
        assert n in nnmg.EXPORTED, f"binding misses {n}"


@pytest.mark.parametrize("name", ["c1_p1", "c1_p2", "c2_p2_128", "cube_p1", "cube_p2"])
def test_host_setup_matches_oracle(nnmg, name):
    meshes, Ho, degree, layers = case(name)
    H = nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, host_only=1, patch_layers=layers)
    try:
        assert H.num_levels == Ho.L
        for l, lo in enumerate(Ho.levels):
            n = lo.n
            assert H.num_dofs(l) == n
            A = to_csr(*H.export_level(l), (n, n))
            assert abs(A - lo.A).max() <= 1e-12 * abs(lo.A).max(), l
            pt = H.export_patches(l)
            assert len(pt) == len(lo.patches)
            for a, b in zip(pt, lo.patches):
                assert np.array_equal(a, b)
            g = H.cell_quality(l, meshes[l].nc)
            assert np.max(np.abs(g - lo.gamma)) < 1e-12
            pts = H.dof_coords(l, meshes[l].dim)
            assert np.array_equal(pts, lo.dm.points[lo.dm.free])
            if l < Ho.L - 1:
                nc = Ho.levels[l + 1].n
                P = to_csr(*H.export_transfer(l), (n, nc))
                assert np.array_equal(P.indptr, lo.P.indptr) and np.array_equal(P.indices, lo.P.indices)
                assert np.max(np.abs(P.data - lo.P.data)) < 1e-13
                lu, la, used = H.eigs(l)
                assert abs(lu - lo.lmax_unadj) < 1e-8 * lo.lmax_unadj
                assert abs(la - lo.lmax_adj) < 1e-8 * lo.lmax_adj
                assert used == la
        from oracle import fem
        dm = Ho.levels[0].dm
        b = fem.load_vector_full(meshes[0].coords, meshes[0].cells, dm, 2.5)[dm.free]
        assert rel_err(H.load_constant(2.5), b) < 1e-13
    finally:
        H.close()


def test_csr_setup_roundtrip(nnmg):
    _, Ho, _, _ = case("c1_p1")
    As, Ps, patches, lam = csr_arrays(Ho)
    H = nnmg.Hierarchy.from_csr(As, Ps, patches, lam, host_only=1)
    try:
        for l in range(Ho.L):
            n = Ho.levels[l].n
            assert (to_csr(*H.export_level(l), (n, n)) != As[l]).nnz == 0
            assert [np.array_equal(a, b) for a, b in zip(H.export_patches(l), patches[l])] == [True] * len(patches[l])
        assert H.eigs(0)[2] == lam[0]
    finally:
        H.close()


def test_setup_errors(nnmg):
    from paper_2402_12947_gb300 import inputs
    meshes = inputs.config_c1()
    with pytest.raises(nnmg.NnmgError) as e:
        nnmg.Hierarchy.from_meshes(meshes, 3, 0.1, host_only=1)
    assert e.value.code == nnmg.ERR_INVALID_ARG
    with pytest.raises(nnmg.NnmgError) as e:
        nnmg.Hierarchy.from_meshes(meshes[:1], 1, 0.1, host_only=1)
    assert e.value.code == nnmg.ERR_INVALID_ARG
    # a degenerate (zero-area) cell
    bad = inputs.Mesh(coords=meshes[1].coords.copy(), cells=meshes[1].cells.copy(), n=meshes[1].n)
    c = bad.cells[100]
    bad.coords[c[2]] = bad.coords[c[0]]
    with pytest.raises(nnmg.NnmgError) as e:
        nnmg.Hierarchy.from_meshes([meshes[0], bad], 1, 0.1, host_only=1)
    assert e.value.code == nnmg.ERR_DEGENERATE_CELL
    # a coarse mesh that does not cover the fine one: point location fails
    small = inputs.Mesh(coords=meshes[1].coords * 0.5, cells=meshes[1].cells, n=meshes[1].n)
    with pytest.raises(nnmg.NnmgError) as e:
        nnmg.Hierarchy.from_meshes([meshes[0], small], 1, 0.1, host_only=1)
    assert e.value.code == nnmg.ERR_POINT_LOCATION
    # out-of-range vertex index
    broken = inputs.Mesh(coords=meshes[1].coords, cells=meshes[1].cells.copy(), n=meshes[1].n)
    broken.cells[0, 0] = 10 ** 7
    with pytest.raises(nnmg.NnmgError) as e:
        nnmg.Hierarchy.from_meshes([meshes[0], broken], 1, 0.1, host_only=1)
    assert e.value.code == nnmg.ERR_INVALID_ARG
    # algebraic set-up needs the eigenvalues
    _, Ho, _, _ = case("c1_p1")
    As, Ps, patches, lam = csr_arrays(Ho)
    with pytest.raises(nnmg.NnmgError) as e:
        nnmg.Hierarchy.from_csr(As, Ps[:1] + [Ps[0]], patches, lam, host_only=1)
    assert e.value.code == nnmg.ERR_INVALID_ARG
    # compute on a host-only hierarchy
    H = nnmg.Hierarchy.from_meshes(meshes, 1, 0.1, host_only=1)
    try:
        code = nnmg.lib.mg_vcycle(H._h, None, None, None)
        assert code in (nnmg.ERR_NO_DEVICE, nnmg.ERR_INVALID_ARG)
    finally:
        H.close()


def test_options_validation(nnmg):
    from paper_2402_12947_gb300 import inputs
    meshes = inputs.config_c1()
    for kw in (dict(cheb_degree=0), dict(nu=0), dict(smoother=7), dict(precision=5), dict(lmin_ratio=1.5),
               dict(tune_min_nnz=-1)):
        with pytest.raises(nnmg.NnmgError) as e:
            nnmg.Hierarchy.from_meshes(meshes, 1, 0.1, host_only=1, **kw)
        assert e.value.code == nnmg.ERR_INVALID_ARG


def test_unreached_coarse_dofs_get_unit_diagonal(nnmg):
    """On a coarse level with needles shorter than the fine mesh size, some coarse P2 DoFs
    are seen by no fine interpolation point: their Galerkin row is the unit row, on both
    the library and the oracle side."""
    _, Ho, _, _ = case("c2_p2_128")
    P = Ho.levels[0].P.tocsc()
    unreached = np.flatnonzero(np.diff(P.indptr) == 0)
    A1 = Ho.levels[1].A
    for j in unreached:
        row = A1.getrow(j)
        assert row.nnz == 1 and row.indices[0] == j and row.data[0] == 1.0


@pytest.mark.parametrize("name", ["c1_p1", "c1_p2", "c2_p2_128", "cube_p1", "cube_p2"])
def test_host_colouring_matches_oracle(nnmg, name):
    """The multicolour SGS colouring of every smoothed level, bit for bit (index work)."""
    from oracle import smoother
    meshes, Ho, degree, layers = case(name)
    with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, host_only=1, patch_layers=layers,
                                    global_smoother="sgs") as H:
        for l, lo in enumerate(Ho.levels[:-1]):
            c = H.export_colouring(l)
            assert np.array_equal(c, smoother.greedy_colouring(lo.A)), l
        with pytest.raises(nnmg.NnmgError):
            H.export_colouring(Ho.L - 1)
    with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, host_only=1, patch_layers=layers) as H:
        with pytest.raises(nnmg.NnmgError):
            H.export_colouring(0)


_LATTICE = {}


def lattice_case(ns, degree, **kw):
    key = (ns, degree, tuple(sorted(kw.items())))
    if key not in _LATTICE:
        from oracle import hierarchy
        from paper_2402_12947_gb300 import inputs
        ms, masks = inputs.config_lattice(ns=ns, n_clusters=3)
        Ho = hierarchy.build(ms, degree, pde="elasticity", dirichlet_masks=masks, **kw)
        _LATTICE[key] = (ms, masks, Ho)
    return _LATTICE[key]


@pytest.mark.parametrize("ns,degree", [((4, 2, 1), 1), ((2, 1), 2)])
def test_host_elasticity_setup_matches_oracle(nnmg, ns, degree):
    """Sec. 6.3: vector operator, componentwise transfer, vector patches, lambda_max and
    the traction load of the clamped lattice, against the oracle."""
    from oracle import elasticity, fem
    ms, masks, Ho = lattice_case(ns, degree)
    with nnmg.Hierarchy.from_meshes(ms, degree, 0.1, host_only=1, pde="elasticity", dirichlet_masks=masks) as H:
        for l, lo in enumerate(Ho.levels):
            n = lo.n
            assert H.num_dofs(l) == n
            A = to_csr(*H.export_level(l), (n, n))
            assert abs(A - lo.A).max() <= 1e-12 * abs(lo.A).max(), l
            pt = H.export_patches(l)
            assert len(pt) == len(lo.patches) and all(np.array_equal(a, b) for a, b in zip(pt, lo.patches))
            if l < Ho.L - 1:
                P = to_csr(*H.export_transfer(l), (n, Ho.levels[l + 1].n))
                assert np.array_equal(P.indptr, lo.P.indptr) and np.array_equal(P.indices, lo.P.indices)
                assert np.max(np.abs(P.data - lo.P.data)) < 1e-13
                lu, la, _ = H.eigs(l)
                assert abs(lu - lo.lmax_unadj) < 1e-8 * lo.lmax_unadj
                assert abs(la - lo.lmax_adj) < 1e-8 * lo.lmax_adj
        m0, dm = ms[0], Ho.levels[0].dm
        t = [1e3, -20.0, 5.0]
        b = H.load_traction(0, 6.0, t)
        bo = elasticity.traction_load_full(m0.coords, m0.cells, dm, t, 0, 6.0)[elasticity.free_vector_dofs(dm)]
        assert rel_err(b, bo) < 1e-13
        with pytest.raises(nnmg.NnmgError):
            H.load_constant(1.0)
        f = [0.0, 2.0, -1e3]
        bb = H.load_body(f)
        bo = np.stack([fem.load_vector_full(m0.coords, m0.cells, dm, fc) for fc in f], axis=1).ravel()
        assert rel_err(bb, bo[elasticity.free_vector_dofs(dm)]) < 1e-13


def test_elasticity_options_validated(nnmg):
    ms, masks, _ = lattice_case((4, 2, 1), 1)
    for bad in (dict(poisson_ratio=0.5), dict(young=-1.0), dict(pde=7)):
        with pytest.raises(nnmg.NnmgError):
            nnmg.Hierarchy.from_meshes(ms, 1, 0.1, host_only=1, pde=bad.pop("pde", "elasticity"),
                                       dirichlet_masks=masks, **bad)
    meshes, _, degree, layers = case("c1_p1")
    with nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, host_only=1) as H:
        with pytest.raises(nnmg.NnmgError):
            H.load_traction(0, 1.0, [1.0, 0.0])


def test_binding_structs_match_the_header(nnmg, tmp_path):
    """The ctypes mirrors of the ABI structs have the C header's size and field offsets
    (compiled with the host C compiler against include/nnmg.h)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"mg_options_t": nnmg.MgOptions, "mg_request_t": nnmg.MgRequest,
               "mg_request_result_t": nnmg.MgRequestResult, "mg_solve_info_t": nnmg.MgSolveInfo,
               "mg_mesh_t": nnmg.MgMesh, "mg_csr_t": nnmg.MgCsr, "mg_server_stats_t": nnmg.MgServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nnmg.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
