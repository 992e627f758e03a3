"""Pins for the normalised radius ratio (Sec. 3, Eq. radius_ratio) (no GPU)."""
import math

import numpy as np

from oracle.quality import radius_ratio


def test_regular_simplices_are_one():
    tri = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, math.sqrt(3) / 2]])
    assert abs(radius_ratio(tri, np.array([[0, 1, 2]]))[0] - 1.0) < 1e-14
    tet = np.array([[1.0, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]])
    assert abs(radius_ratio(tet, np.array([[0, 1, 2, 3]]))[0] - 1.0) < 1e-14


def test_right_isosceles_and_kuhn():
    tri = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    assert abs(radius_ratio(tri, np.array([[0, 1, 2]]))[0] - 2 * (math.sqrt(2) - 1)) < 1e-14
    # Kuhn tet: circumsphere = the cube's (R_C = sqrt(3)/2), faces 1/2, 1/2, sqrt2/2, sqrt2/2
    kuhn = np.array([[0.0, 0, 0], [1, 0, 0], [1, 1, 0], [1, 1, 1]])
    assert abs(radius_ratio(kuhn, np.array([[0, 1, 2, 3]]))[0] - math.sqrt(3) / (1 + math.sqrt(2))) < 1e-14


def test_flattened_triangle_asymptotics():
    # apex at height e over the midpoint of a unit base: gamma = 2 R_I / R_C, closed form
    for e in (1e-2, 1e-3, 1e-5):
        tri = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, e]])
        s = math.sqrt(0.25 + e * e)
        area = e / 2
        r_in = 2 * area / (1 + 2 * s)
        r_c = 1 * s * s / (4 * area)
        g = radius_ratio(tri, np.array([[0, 1, 2]]))[0]
        assert abs(g - 2 * r_in / r_c) < 1e-12 * max(g, 1e-300) + 1e-18
        assert abs(g / (8 * e * e) - 1) < 10 * e


def test_invariances():
    rng = np.random.default_rng(5)
    for dim in (2, 3):
        X = rng.normal(size=(50, dim + 1, dim))
        cells = np.arange(50 * (dim + 1)).reshape(50, dim + 1)
        g = radius_ratio(X.reshape(-1, dim), cells)
        assert np.all((g > 0) & (g <= 1 + 1e-12))
        Q, _ = np.linalg.qr(rng.normal(size=(dim, dim)))
        Y = 3.7 * X @ Q.T + 0.3
        assert np.allclose(radius_ratio(Y.reshape(-1, dim), cells), g, rtol=1e-10)
        perm = rng.permutation(dim + 1)
        assert np.allclose(radius_ratio(X[:, perm].reshape(-1, dim), cells), g, rtol=1e-10)
