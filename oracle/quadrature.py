"""Exact quadrature on the reference simplex (oracle; test infrastructure only).

The reference simplex is {xi_i >= 0, sum xi_i <= 1} with volume 1/d!. Rules are built by
the collapsed-coordinate (Duffy) map from the unit cube with Gauss-Legendre points in
each direction, so a rule of requested polynomial degree q integrates every polynomial
of total degree <= q exactly.

Pinned by: tests/test_oracle_fem.py (monomial integrals against the closed form
int xi^a = d! prod a_i! / (d + |a|)! times the volume 1/d!).
"""
from __future__ import annotations

import functools

import numpy as np


@functools.lru_cache(maxsize=None)
def simplex_rule(dim: int, degree: int):
    """Points [nq, dim] and weights [nq] (sum = 1/dim!) exact for total degree <= ``degree``."""
    # In collapsed coordinates the integrand gains Jacobian factors (1-u)^(dim-1) ...,
    # so each 1D direction needs degree + dim - 1 exactness: m points give 2m - 1.
    m = (degree + dim) // 2 + 1
    g, w = np.polynomial.legendre.leggauss(m)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    if dim == 1:
        return g[:, None].copy(), w.copy()
    if dim == 2:
        u, v = np.meshgrid(g, g, indexing="ij")
        wu, wv = np.meshgrid(w, w, indexing="ij")
        x1 = u
        x2 = v * (1.0 - u)
        wt = wu * wv * (1.0 - u)
        pts = np.stack([x1.ravel(), x2.ravel()], axis=1)
        return pts, wt.ravel()
    if dim == 3:
        u, v, s = np.meshgrid(g, g, g, indexing="ij")
        wu, wv, ws = np.meshgrid(w, w, w, indexing="ij")
        x1 = u
        x2 = v * (1.0 - u)
        x3 = s * (1.0 - u) * (1.0 - v)
        wt = wu * wv * ws * (1.0 - u) ** 2 * (1.0 - v)
        pts = np.stack([x1.ravel(), x2.ravel(), x3.ravel()], axis=1)
        return pts, wt.ravel()
    raise ValueError("dim must be 1, 2 or 3")


def barycentric_of_reference(pts: np.ndarray) -> np.ndarray:
    """[nq, dim] reference points -> [nq, dim+1] barycentric coordinates (lambda_0 = 1 - sum)."""
    return np.concatenate([1.0 - pts.sum(axis=1, keepdims=True), pts], axis=1)
