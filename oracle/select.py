"""Choice of the interpolation stencil size and interval size for a target
error: the two-step procedure of Sec. 2.5, written out plainly in NumPy FP64.

TEST INFRASTRUCTURE ONLY (see the package header).

Step 1 (Sec. 2.5, Eq. leb): interpolating nodal values that carry relative
perturbations eps_p perturbs the interpolant by at most Lambda^d eps_p in d
dimensions on tensor-product nodes, Lambda the Lebesgue constant of the 1D
node set.  n_max is the largest n with Lambda_n^3 eps_p < eps, Lambda_n the
Lebesgue constant of n equally spaced nodes (the maximum over their interval
of sum_i |l_i(x)|), eps_p the unit roundoff (2^-53 FP64, 2^-24 FP32).

Step 2: more nodes per interval (n_I = n_b + 1; only the nearest n_max used)
until the interpolation error of the function at hand is below eps.  The
reading adopted here: the function is the field of the nearest sources a
parent interval's interaction list can hold, G(x - y) with y on the face of
the interval one interval width away (x = 4 n_b; y, z at the face's corners,
edge midpoints and centre), known at the parent's nodes (spacing 2) and
interpolated with the Sec. 2.5 stencil to the nodes of its two children
(spacing 1); the error is relative to max |G| over those nodes.  The block
sizes tried are 4, 6, ..., 32 (the supported range) with n_b + 1 >= n_max.

Pins (tests/test_oracle_select.py): the classical Lebesgue constants of 2..5
equispaced nodes; the paper's example (FP64, eps = 1.25e-12 allows n_max = 10);
the step-2 error of a stencil that interpolates the sampled function exactly
(n_max equal to the node count along a line and a polynomial field).
"""
from __future__ import annotations

import numpy as np

from . import fmm
from . import lgf as _lgf


def lebesgue_equispaced(n: int, samples: int = 200001) -> float:
    """max over [0, n-1] of sum_i |l_i(x)| for the nodes 0..n-1, by dense sampling."""
    if n <= 1:
        return 1.0
    x = np.linspace(0.0, n - 1.0, samples)
    total = np.zeros_like(x)
    nodes = np.arange(n, dtype=np.float64)
    for i in range(n):
        li = np.ones_like(x)
        for j in range(n):
            if j != i:
                li *= (x - nodes[j]) / (nodes[i] - nodes[j])
        total += np.abs(li)
    return float(total.max())


def unit_roundoff(precision: str) -> float:
    return 2.0 ** -53 if precision == "fp64" else 2.0 ** -24


def step1_n_max(eps: float, precision: str, n_limit: int = 17) -> tuple[int, float]:
    """Largest n <= n_limit with Lambda_n^3 * eps_p < eps, and its Lambda_n."""
    ep = unit_roundoff(precision)
    best, lam = 1, 1.0
    for n in range(2, n_limit + 1):
        l = lebesgue_equispaced(n)
        if l ** 3 * ep >= eps:
            break
        best, lam = n, l
    return best, lam


def far_field_interp_error(n_b: int, n_max: int) -> float:
    """Step-2 error for one block size: max over the source positions of
    max|Interp(G(. - y)) - G(. - y)| / max|G(. - y)| on the children's nodes."""
    n_I = n_b + 1
    W = fmm.interp_weights(n_b, n_max)          # W[c, i, p]
    tab = _lgf.lgf_abs_table(1, 4 * n_b)
    child = np.arange(2 * n_b + 1)              # child node coordinates (spacing 1)
    parent = 2 * np.arange(n_I)                 # parent node coordinates (spacing 2)
    worst = 0.0
    for a in (0, n_b, 2 * n_b):
        for b in (0, n_b, 2 * n_b):
            y = (4 * n_b, a, b)
            # field at the parent's nodes, [z, y, x]
            F = tab[np.abs(parent[None, None, :] - y[0]), np.abs(parent[None, :, None] - y[1]),
                    np.abs(parent[:, None, None] - y[2])]
            exact = tab[np.abs(child[None, None, :] - y[0]), np.abs(child[None, :, None] - y[1]),
                        np.abs(child[:, None, None] - y[2])]
            # each child (cz, cy, cx) interpolated with the oracle's own Interp
            got = np.zeros_like(exact)
            for cz in (0, 1):
                for cy in (0, 1):
                    for cx in (0, 1):
                        v = fmm.interp(W, (cx, cy, cz), F)
                        got[cz * n_b:cz * n_b + n_I, cy * n_b:cy * n_b + n_I, cx * n_b:cx * n_b + n_I] = v
            worst = max(worst, float(np.abs(got - exact).max() / np.abs(exact).max()))
    return worst


def select(eps: float, precision: str) -> dict:
    """Both steps: {"n_max", "lebesgue", "n_b", "interp_err", "reached"}."""
    n_max, lam = step1_n_max(eps, precision)
    err, chosen = 0.0, 0
    for n_b in range(4, 33, 2):
        if n_b + 1 < n_max:
            continue
        err = far_field_interp_error(n_b, n_max)
        chosen = n_b
        if err < eps:
            break
    return {"n_max": n_max, "lebesgue": lam, "n_b": chosen, "interp_err": err,
            "reached": chosen > 0 and err < eps}
