"""Lattice Green's function of the 7-point discrete Laplacian, FP64.

TEST INFRASTRUCTURE ONLY (see the package header): the CUDA library has its own,
independently written generator.

What it computes (App. A, Eq. lgf3):

    G(n) = - int_0^inf  e^{-6t} I_{n1}(2t) I_{n2}(2t) I_{n3}(2t) dt
         = - int_0^inf  Ie_{n1}(2t) Ie_{n2}(2t) Ie_{n3}(2t) dt,

with Ie_k(x) = e^{-x} I_k(x) the exponentially scaled modified Bessel function
(scipy.special.ive).  As App. A describes, the half line is split at alpha:
[0, alpha] is integrated numerically and [alpha, inf) analytically from the
large-argument expansion of I_k (Abramowitz & Stegun 9.7.1), integrating the
product of the three series term by term.  alpha is a power of two at least
max(2^10, 50 * max|n_i|^2), which makes the series terms beyond the tenth
smaller than 1e-17 of the first.  [0, alpha] is cut into [0, 2^-6] and dyadic
panels [2^e, 2^(e+1)], each with a Gauss-Legendre rule (numpy.leggauss); the
integrand is smooth on each dyadic panel in log t, and the tests check the rule
against a twice-refined one and against scipy's adaptive Gauss-Kronrod
(``lgf_quad``), the scheme App. A names.

Symmetry (Sec. 2.1): G is invariant under reflections about the axes and
permutations of the indices, so only sorted |n| triples are evaluated.

Pins (tests/test_oracle_lgf.py): Watson's closed form for G(0); G(1,0,0) = G(0)
+ 1/6 from L G = delta at the origin; the stencil identity L G = delta on a
whole tabulated box; the far field against the printed two-term expansion A^2
(Eq. lgf2); 48-fold symmetry; the adaptive quadrature cross-check.
"""
from __future__ import annotations

import functools
import math

import numpy as np
from scipy import integrate, special

PANEL_NODES = 24      # Gauss-Legendre nodes per panel
T0_EXP = -6           # first panel is [0, 2^T0_EXP]
ALPHA_MIN_EXP = 10    # alpha >= 2^10
TAIL_FACTOR = 50.0    # alpha >= TAIL_FACTOR * max|n_i|^2
TAIL_TERMS = 10       # terms kept in the product of the three expansions


def _alpha_exp(cmax: np.ndarray) -> np.ndarray:
    need = np.maximum(2.0 ** ALPHA_MIN_EXP, TAIL_FACTOR * cmax.astype(np.float64) ** 2)
    return np.ceil(np.log2(need)).astype(np.int64)


def _expansion_coeffs(k: int, nterms: int) -> np.ndarray:
    """b_j with Ie_k(2t) ~ (4 pi t)^(-1/2) sum_j b_j t^(-j)  (A&S 9.7.1, z = 2t)."""
    mu = 4.0 * k * k
    b = np.zeros(nterms + 1)
    a = 1.0
    b[0] = 1.0
    for j in range(1, nterms + 1):
        a *= (mu - (2 * j - 1) ** 2) / (8.0 * j)
        b[j] = (-1) ** j * a / 2.0 ** j
    return b


def _tail(triple, alpha: float) -> float:
    """int_alpha^inf prod_i Ie_{n_i}(2t) dt from the term-by-term integral."""
    return float(_tail_many(np.asarray([triple]), np.asarray([alpha]))[0])


def _tail_many(trip: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """_tail for many triples at once: the product of the three expansions is
    truncated after TAIL_TERMS and integrated term by term."""
    J = TAIL_TERMS
    b = [np.stack([_expansion_coeffs(int(k), J) for k in range(int(trip.max()) + 1)])[trip[:, i]]
         for i in range(3)]                                   # (m, J+1) each
    c = np.zeros((len(trip), J + 1))
    for i in range(J + 1):
        for j in range(J + 1 - i):
            c[:, i + j:] += (b[0][:, i] * b[1][:, j])[:, None] * b[2][:, : J + 1 - i - j]
    jj = np.arange(J + 1)
    return (4.0 * math.pi) ** -1.5 * np.sum(c * alpha[:, None] ** (-0.5 - jj) / (jj + 0.5), axis=1)


def _panels(max_exp: int, q: int):
    """Nodes and weights on [0, 2^T0] and [2^e, 2^(e+1)], e = T0 .. max_exp-1."""
    xi, wi = np.polynomial.legendre.leggauss(q)
    edges = [0.0] + [2.0 ** e for e in range(T0_EXP, max_exp + 1)]
    ts, ws = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        ts.append(0.5 * (b - a) * xi + 0.5 * (a + b))
        ws.append(0.5 * (b - a) * wi)
    return np.concatenate(ts), np.concatenate(ws)


def _lgf_sorted(trip: np.ndarray, q: int = PANEL_NODES) -> np.ndarray:
    """G for sorted non-negative triples (a <= b <= c), shape (m, 3)."""
    if len(trip) == 0:
        return np.zeros(0)
    aexp = _alpha_exp(trip[:, 2])
    t, w = _panels(int(aexp.max()), q)
    kmax = int(trip.max())
    # Ie_k(2 t_q) for every order and node: rows k, columns q.
    bes = special.ive(np.arange(kmax + 1)[:, None], 2.0 * t[None, :])
    out = np.empty(len(trip))
    for ae in np.unique(aexp):
        nq = q * (1 + ae - T0_EXP)              # nodes with t < 2^ae
        sel = np.nonzero(aexp == ae)[0]
        wq = w[:nq]
        for s in range(0, len(sel), 4096):
            idx = sel[s: s + 4096]
            tr = trip[idx]
            prod = bes[tr[:, 0], :nq] * bes[tr[:, 1], :nq] * bes[tr[:, 2], :nq]
            out[idx] = prod @ wq
        out[sel] += _tail_many(trip[sel], np.full(len(sel), 2.0 ** ae))
    return -out


def lgf(n, q: int = PANEL_NODES) -> np.ndarray:
    """G(n) for integer triples n (any shape (..., 3), any signs), FP64."""
    n = np.asarray(n, dtype=np.int64)
    shp = n.shape[:-1]
    s = np.sort(np.abs(n.reshape(-1, 3)), axis=1)
    uniq, inv = np.unique(s, axis=0, return_inverse=True)
    return _lgf_sorted(uniq, q)[inv.ravel()].reshape(shp)


@functools.lru_cache(maxsize=16)
def lgf_abs_table(h: int, vmax: int) -> np.ndarray:
    """Dense table T[a, b, c] = G(h*(a, b, c)) for 0 <= a, b, c <= vmax (read-only).

    By the reflection symmetry, G(h*v) = T[|v_x|, |v_y|, |v_z|] for any v."""
    r = np.arange(vmax + 1)
    a, b, c = np.meshgrid(r, r, r, indexing="ij")
    tab = lgf(h * np.stack([a, b, c], axis=-1))
    tab.setflags(write=False)
    return tab


def lgf_quad(n) -> float:
    """Independent slow check: scipy's adaptive Gauss-Kronrod (QUADPACK) on
    [0, alpha] plus the same analytic tail, for one triple."""
    k = sorted(abs(int(v)) for v in n)
    alpha = 2.0 ** int(_alpha_exp(np.array([k[2]]))[0])
    f = lambda tt: float(special.ive(k[0], 2 * tt) * special.ive(k[1], 2 * tt)
                         * special.ive(k[2], 2 * tt))
    # break points on a dyadic grid so the adaptive rule sees each scale
    pts = [2.0 ** e for e in range(-4, int(math.log2(alpha)))]
    total = 0.0
    edges = [0.0] + pts + [alpha]
    for a, b in zip(edges[:-1], edges[1:]):
        val, _ = integrate.quad(f, a, b, epsabs=0.0, epsrel=2e-14, limit=200)
        total += val
    return -(total + _tail(k, alpha))


def asymptotic_a2(x) -> np.ndarray:
    """Two-term far-field expansion A^2_G(x) of Eq. lgf2."""
    x = np.asarray(x, dtype=np.float64)
    x1, x2, x3 = x[..., 0], x[..., 1], x[..., 2]
    r = np.sqrt(x1 * x1 + x2 * x2 + x3 * x3)
    num = x1 ** 4 + x2 ** 4 + x3 ** 4 - 3 * (x1 * x1 * x2 * x2 + x1 * x1 * x3 * x3 + x2 * x2 * x3 * x3)
    return -1.0 / (4 * math.pi * r) - num / (16 * math.pi * r ** 7)


def watson_g0() -> float:
    """G(0) from Watson's integral in the Glasser-Zucker Gamma-function form:
    -(sqrt 6 / (192 pi^3)) Gamma(1/24) Gamma(5/24) Gamma(7/24) Gamma(11/24)."""
    g = math.gamma
    return -(math.sqrt(6.0) / (192.0 * math.pi ** 3)) * g(1 / 24) * g(5 / 24) * g(7 / 24) * g(11 / 24)
