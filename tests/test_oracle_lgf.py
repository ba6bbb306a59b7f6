"""Pins of the oracle LGF (oracle/lgf.py) against facts fixed by the paper and
the mathematics, not against the oracle itself."""
import math

import numpy as np
import pytest

from oracle import lgf as L


def test_watson_closed_form():
    # G(0) is minus one sixth of Watson's simple-cubic integral; Glasser-Zucker
    # closed form in Gamma functions.  Printed value (six digits) -0.252731.
    g0 = float(L.lgf([[0, 0, 0]])[0])
    assert abs(g0 - L.watson_g0()) <= 2e-15 * abs(g0)
    assert round(g0, 6) == -0.252731


def test_first_neighbour_from_stencil_identity():
    # L G = delta at the origin with the 6-fold symmetry: 6 G(e1) - 6 G(0) = 1.
    g = L.lgf([[0, 0, 0], [1, 0, 0]])
    assert abs((g[1] - g[0]) - 1.0 / 6.0) < 1e-15


def test_stencil_identity_on_box():
    # L G = delta at every point of a box (7-point Laplacian of Eq. dpoisson).
    V = 24
    tab = L.lgf_abs_table(1, V + 1)
    r1 = np.abs(np.arange(-V - 1, V + 2))
    G = tab[np.ix_(r1, r1, r1)]                  # signed box [-V-1, V+1]^3
    c = G[1:-1, 1:-1, 1:-1]
    lap = (G[2:, 1:-1, 1:-1] + G[:-2, 1:-1, 1:-1] + G[1:-1, 2:, 1:-1] + G[1:-1, :-2, 1:-1]
           + G[1:-1, 1:-1, 2:] + G[1:-1, 1:-1, :-2] - 6.0 * c)
    delta = np.zeros_like(lap)
    delta[V, V, V] = 1.0
    assert np.abs(lap - delta).max() < 1e-15


def test_far_field_two_term_expansion():
    # G - A^2 = O(|n|^-5) (Eq. lgf2 with q = 2): along rays |G - A^2| |n|^5 stays
    # bounded, and -4 pi |n| G -> 1.
    for ray in ([1, 0, 0], [1, 1, 0], [1, 1, 1], [3, 2, 1]):
        ray = np.array(ray)
        ks = np.array([8, 16, 32, 64])
        pts = ks[:, None] * ray[None, :]
        g = L.lgf(pts)
        a2 = L.asymptotic_a2(pts.astype(float))
        rn = np.linalg.norm(pts, axis=1)
        scaled = np.abs(g - a2) * rn ** 5
        assert scaled.max() < 0.1
        assert np.all(np.abs(-4 * math.pi * rn * g - 1) < 1.0 / rn ** 2)
    # the paper's remark: A^2 alone is far from FP64 accuracy at |n| ~ 10
    g10 = L.lgf([[10, 0, 0]])[0]
    assert 1e-6 < abs((L.asymptotic_a2(np.array([10.0, 0, 0])) - g10) / g10) < 1e-3


def test_adaptive_gauss_kronrod_cross_check():
    # App. A's scheme (adaptive Gauss-Kronrod, QUADPACK) agrees with the panel rule.
    pts = [[0, 0, 0], [1, 2, 3], [0, 0, 17], [5, 9, 40], [100, 3, 7], [64, 64, 64]]
    fast = L.lgf(pts)
    for p, v in zip(pts, fast):
        ref = L.lgf_quad(p)
        assert abs(v - ref) <= 2e-14 * abs(ref), (p, v, ref)


def test_quadrature_converged():
    pts = [[0, 0, 0], [0, 0, 512], [512, 512, 512], [3, 5, 300], [31, 0, 2]]
    a = L.lgf(pts)
    b = L.lgf(pts, q=40)
    assert np.all(np.abs(a - b) <= 1e-14 * np.abs(b))


def test_symmetry_48():
    # reflections about the axes and index permutations (Sec. 2.1)
    base = np.array([2, 5, 11])
    vals = []
    for perm in ([0, 1, 2], [1, 2, 0], [2, 0, 1], [0, 2, 1], [2, 1, 0], [1, 0, 2]):
        for s in ([1, 1, 1], [-1, 1, 1], [1, -1, -1], [-1, -1, -1]):
            vals.append(L.lgf([base[perm] * np.array(s)])[0])
    assert max(vals) == min(vals)
