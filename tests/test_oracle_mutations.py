"""The oracle's pins catch plausible mistakes: each case plants one mistake in the oracle
(on the CPU, through monkeypatch) and checks that the pin meant to catch it fails."""
import numpy as np
import pytest

import test_oracle_elasticity as t_el
import test_oracle_fem as t_fem
import test_oracle_mg as t_mg
import test_oracle_quality as t_q
import test_oracle_smoother as t_sm
import test_oracle_transfer as t_tr
from oracle import eig, elasticity, fem, mg, patches, smoother, transfer


def _cheb_first_step_by_lmax(orig):
    def f(lmax, lmin, k):
        out = orig(lmax, lmin, k)
        out[0] = (0.0, 1.0 / lmax)                 # first step scaled by 1/lmax, not 1/theta
        return out
    return f


def _cheb_sign(orig):
    def f(lmax, lmin, k):
        return [(-cd, cr) for cd, cr in orig(lmax, lmin, k)]   # three-term recurrence sign
    return f


def _local_without_residual(self, A, b, x):
    x = x.copy()
    for p, fac in zip(self.patches, self.factors):
        x[p] += fac.solve(b[p])                   # b instead of b - A x
    return x


def _vcycle_no_post(H, b, x=None, l=0):
    lev = H.levels[l]
    if l == H.L - 1:
        return H.coarse.solve(b)
    x = np.zeros_like(b) if x is None else x.copy()
    for _ in range(H.nu):
        x = smoother.smooth(lev.A, lev.dinv, b, x, lev.lmax, lev.lmin, H.cheb_degree, lev.local, H.order,
                            post=False, kind=H.smoother_kind, colour=lev.colour)
    x = x + lev.P @ _vcycle_no_post(H, lev.R @ (b - lev.A @ x), None, l + 1)
    return x                                      # post-smoothing dropped


def _sgs_forward_only(A, dinv, b, x, colour):
    x = x.copy()
    for c in range(int(colour.max()) + 1):        # backward sweep dropped
        rows = np.flatnonzero(colour == c)
        x[rows] += dinv[rows] * (b[rows] - A[rows] @ x)
    return x


CASES = [
    # (name, module, attribute, mutation(original) -> replacement, pin)
    ("chebyshev first step", smoother, "chebyshev_coefficients", _cheb_first_step_by_lmax,
     lambda r: t_sm.test_chebyshev_error_polynomial(2)),
    ("chebyshev recurrence sign", smoother, "chebyshev_coefficients", _cheb_sign,
     lambda r: t_sm.test_chebyshev_error_polynomial(3)),
    ("local correction without residual", smoother.LocalSolver, "apply", lambda o: _local_without_residual,
     lambda r: t_sm.test_combined_smoother_closed_form_and_symmetry("sandwich")),
    ("multicolour SGS forward only", smoother, "multicolour_sgs", lambda o: _sgs_forward_only,
     lambda r: t_sm.test_multicolour_sgs_is_sequential_sgs_in_colour_order()),
    ("adjusted lambda not adjusted", eig, "adjusted_lambda_max", lambda o: (lambda A, patches: eig.lambda_max(A)),
     lambda r: t_sm.test_adjusted_lambda_recovers_high_quality_value()),
    ("stiffness scaled", fem, "element_stiffness", lambda o: (lambda c, cl, d: 2.0 * o(c, cl, d)),
     lambda r: t_fem.test_p1_five_point_stencil()),
    # the quality pins call the function they imported, so the mistake is planted there
    ("radius ratio without the dimension", t_q, "radius_ratio",
     lambda o: (lambda c, cl: o(c, cl) / c.shape[1]), lambda r: t_q.test_regular_simplices_are_one()),
    ("prolongation scaled", transfer, "prolongation", lambda o: (lambda *a, **k: 1.01 * o(*a, **k)),
     lambda r: t_tr.test_polynomial_reproduction_and_partition_of_unity(2, 2)),
    ("galerkin scaled", transfer, "galerkin", lambda o: (lambda A, P: 2.0 * o(A, P)),
     lambda r: t_tr.test_galerkin_spd_and_dense_triple_product(2, 1)),
    ("v-cycle without post-smoothing", mg, "vcycle", lambda o: _vcycle_no_post,
     lambda r: t_mg.test_vcycle_linear_and_symmetric(r.getfixturevalue("c1_meshes"))),
    ("patch components all merged", patches, "connected_components",
     lambda o: (lambda g, directed=False: (1, np.zeros(g.shape[0], dtype=np.int32))),
     lambda r: t_sm.test_patch_components_are_vertex_connected_components(1)),
    ("elasticity lambda term dropped", elasticity, "element_elasticity",
     lambda o: (lambda c, cl, d, mu, lam: o(c, cl, d, mu, 0.0)), lambda r: t_el.test_affine_energies(2, 1)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(case, monkeypatch, request):
    name, module, attr, mutate, pin = case
    monkeypatch.setattr(module, attr, mutate(getattr(module, attr)))
    with pytest.raises(AssertionError):
        pin(request)
