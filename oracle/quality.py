"""Normalised radius ratio gamma (oracle; test infrastructure only).

Sec. 3, Eq. (radius_ratio): gamma = R_I / (gamma* R_C) with R_I the inscribed and R_C the
circumscribed radius. The printed normalisation is garbled (gamma* "equal to the
dimension" would cap gamma at 1/d^2 instead of the stated range (0, 1]); the reading
used here is gamma = d R_I / R_C, which is 1 for the regular simplex and lies in (0, 1].

2D: R_I = 2|K| / perimeter, R_C = a b c / (4|K|).
3D: R_I = 3|K| / (sum of face areas), R_C = |c - v0| with the circumcentre c solving
    2 (v_i - v0) . (c - v0) = |v_i - v0|^2, i = 1..3.

Pinned by tests/test_oracle_quality.py: regular simplex = 1, right isosceles triangle
= 2(sqrt 2 - 1), Kuhn tetrahedron = 0.71744..., scale/rotation invariance, and the
asymptotics of a flattened triangle.
"""
from __future__ import annotations

import numpy as np


def radius_ratio(coords: np.ndarray, cells: np.ndarray) -> np.ndarray:
    dim = coords.shape[1]
    cells = cells.astype(np.int64)
    X = coords[cells]                                   # [nc, d+1, dim]
    if dim == 2:
        a = np.linalg.norm(X[:, 1] - X[:, 2], axis=1)
        b = np.linalg.norm(X[:, 0] - X[:, 2], axis=1)
        c = np.linalg.norm(X[:, 0] - X[:, 1], axis=1)
        e1 = X[:, 1] - X[:, 0]
        e2 = X[:, 2] - X[:, 0]
        area = 0.5 * np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
        r_in = 2.0 * area / (a + b + c)
        r_circ = a * b * c / (4.0 * area)
        return 2.0 * r_in / r_circ
    if dim == 3:
        E = X[:, 1:] - X[:, :1]                         # [nc, 3, 3] rows v_i - v0
        vol = np.abs(np.linalg.det(E)) / 6.0
        faces = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]
        area = np.zeros(len(cells))
        for i, j, k in faces:
            area += 0.5 * np.linalg.norm(np.cross(X[:, j] - X[:, i], X[:, k] - X[:, i]), axis=1)
        r_in = 3.0 * vol / area
        rhs = 0.5 * np.sum(E * E, axis=2)                # [nc, 3]
        cc = np.linalg.solve(E, rhs[..., None])[..., 0]  # circumcentre relative to v0
        r_circ = np.linalg.norm(cc, axis=1)
        return 3.0 * r_in / r_circ
    raise ValueError("dim must be 2 or 3")
