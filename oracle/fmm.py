"""The Fast Lattice Green's Function method, step by step, FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see the package header).  Also the timed CPU baseline.

It follows Sec. 3.1: Step 0 pre-computes the kernel spectra (Eq. precomp), Step 1
regularizes and forward-transforms upward (Eqs. alg_reg, alg_upfft), Step 2 sums
spectral products over each influence list (Eq. alg_mult), Step 3 truncates the
inverse transforms and interpolates downward (Eqs. alg_dwfft, alg_interp).  The
FFT convolution is the Pad / FFT / Prod / FFT^-1 / Trunc sequence of Sec. 2.2 in
three dimensions; numpy.fft is the library primitive for each FFT.

Readings of the paper this oracle adopts (the paper is silent or garbled there):
  * Tree: leaves are one level-1 interval per active block with the same integer
    index; the level-l index of a block b is b >> (l-1) (floor), and a level-l
    interval exists iff some block below it is active (Sec. 3.1).  Interval I at
    level l >= 1 has n_I = n_b + 1 nodes per axis with spacing h_l = 2^(l-1) from
    origin I*n_b*h_l, so neighbours share one node plane (Sec. 4, footnote).
  * Lists: near(P) = same-level Q with max|Q-P| <= 1 (27 incl. P).  Level 0 uses
    near; 1 <= l < L uses the interaction list {Q: parent(Q) near parent(P), Q not
    near P} (<= 189); at the top level L, where no parent exists, every Q not
    near P, which counts each pair of blocks exactly once.
  * Interpolation "order p" is the polynomial degree: n_max = p + 1 nodes (Sec.
    2.5 calls n_max = 10 one order above the interpolation order).  Child c in
    {0,1} node i sits at parent coordinate x = c*n_b/2 + i/2; integer x copies
    that node; otherwise the n_max nodes nearest x are used, the odd extra node
    taken on the side of the interval centre n_b/2 (lower side at the centre),
    the window shifted inside [0, n_I - 1]; weights are the Lagrange products.
    Reg is the exact adjoint (transpose) of Interp (Sec. 2.4).
  * Kernel vectors: target node i of P and source node j of Q interact through
    G(h(-d*n_b + i - j)), d = idx(Q) - idx(P); the vector k(m) = G(h(m - d*n_b)),
    |m_a| <= n-1, is stored at index m mod S with S = 2n (Sec. 3.2), and the block
    result is the first n samples of the circular convolution (the Pad/Trunc
    index formulas of Sec. 2.2 are garbled; this is the linear convolution they
    describe).  Level 0 uses n = n_b, level l >= 1 uses n = n_I.
  * Level 1 carries the block's sources on nodes [0, n_b)^3 and zero on the
    shared last node plane (it belongs to the neighbouring block); overlapping
    nodes of neighbouring intervals are never merged.  The output of a block is
    the level-0 near field plus the level-1 field on its first n_b^3 nodes.
  * The kernel is G itself at every offset (the printed two-term far-field
    expansion is far too coarse for a 1e-12 answer; see oracle/lgf.py).

Pins (tests/test_oracle_fmm.py): with no interpolation in play (two levels, or
a single block) the result equals the exact direct sum to ~1e-13; the random
manufactured solution of Sec. 4.1 is reproduced to the method's truncation
error; 1D/3D FFT convolution against a dense sum; interpolation reproduces
polynomials of degree <= n_max-1 and Reg is its transpose; list sizes 27/189/316;
linearity, translation and mirror invariance.
"""
from __future__ import annotations

import numpy as np

from . import lgf as _lgf

# --------------------------------------------------------------------------
# Tree and lists (Sec. 3.1)


def _key(v):
    return (int(v[0]), int(v[1]), int(v[2]))


def _near(p, q) -> bool:
    return max(abs(p[0] - q[0]), abs(p[1] - q[1]), abs(p[2] - q[2])) <= 1


def _parent(p):
    return (p[0] >> 1, p[1] >> 1, p[2] >> 1)


def _child_pos(p):
    return (p[0] & 1, p[1] & 1, p[2] & 1)


def build_levels(blocks, n_levels: int):
    """levels[l] = sorted list of interval indices at level l (level 0 = blocks)."""
    b = [_key(v) for v in np.asarray(blocks)]
    levels = {0: sorted(b)}
    for l in range(1, n_levels + 1):
        s = l - 1
        levels[l] = sorted({(x >> s, y >> s, z >> s) for (x, y, z) in b})
    return levels


def influence_list(levels, l: int, P, n_levels: int, members=None):
    """InflList(P) at level l: near neighbours at l = 0, interaction list above.

    ``members`` (a set of levels[l]) only speeds up the membership test: the
    candidates enumerated are exactly the intervals the definition can admit."""
    mem = set(levels[l]) if members is None else members
    if l == 0:
        cand = [(P[0] + a, P[1] + b, P[2] + c)
                for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)]
        return [Q for Q in cand if Q in mem]
    if l < n_levels:
        pp = _parent(P)
        cand = [(2 * (pp[0] + ex) + cx, 2 * (pp[1] + ey) + cy, 2 * (pp[2] + ez) + cz)
                for ez in (-1, 0, 1) for ey in (-1, 0, 1) for ex in (-1, 0, 1)
                for cz in (0, 1) for cy in (0, 1) for cx in (0, 1)]
        return sorted(Q for Q in cand if Q in mem and not _near(P, Q))
    return [Q for Q in levels[l] if not _near(P, Q)]


# --------------------------------------------------------------------------
# Interpolation between levels (Sec. 2.4-2.5)


def interp_weights(n_b: int, n_max: int) -> np.ndarray:
    """W[c][i, p]: weight of parent node p for node i of child c (c = 0, 1)."""
    n_I = n_b + 1
    if not (1 <= n_max <= n_I):
        raise ValueError("need 1 <= n_max <= n_I")
    W = np.zeros((2, n_I, n_I))
    centre = n_b / 2.0
    for c in (0, 1):
        for i in range(n_I):
            x = c * n_b / 2.0 + i / 2.0
            if float(x).is_integer():
                W[c, i, int(x)] = 1.0
                continue
            k = int(np.floor(x))
            if n_max % 2 == 0:
                start = k - n_max // 2 + 1
            else:
                m = (n_max - 1) // 2
                start = k - m + 1 if x < centre else k - m
            start = min(max(start, 0), n_I - n_max)
            nodes = np.arange(start, start + n_max, dtype=np.float64)
            for a, xa in enumerate(nodes):
                w = 1.0
                for bnode in nodes:
                    if bnode != xa:
                        w *= (x - bnode) / (xa - bnode)
                W[c, i, start + a] = w
    return W


def interp(W, c, U):
    """Interp: child field from parent field U[z, y, x]; the tensor product
    (W_cz x W_cy x W_cx) applied one axis at a time."""
    t = np.einsum("kr,pqr->pqk", W[c[0]], U)
    t = np.einsum("jq,pqk->pjk", W[c[1]], t)
    return np.einsum("ip,pjk->ijk", W[c[2]], t)


def reg(W, c, F):
    """Reg: the adjoint of interp, parent sources from child sources F[z, y, x];
    the transposed tensor product applied one axis at a time."""
    t = np.einsum("kr,ijk->ijr", W[c[0]], F)
    t = np.einsum("jq,ijr->iqr", W[c[1]], t)
    return np.einsum("ip,iqr->pqr", W[c[2]], t)


# --------------------------------------------------------------------------
# Kernel vectors and their spectra (Step 0, Eq. precomp)


def kernel_vector(h: int, d, n: int, n_b: int, S: int) -> np.ndarray:
    """k(m) = G(h (m - d n_b)) for |m_a| <= n-1 at circular index m mod S; [z, y, x]."""
    m = np.arange(-(n - 1), n)
    vmax = (n - 1) + n_b * max(3, abs(int(d[0])), abs(int(d[1])), abs(int(d[2])))
    tab = _lgf.lgf_abs_table(int(h), int(vmax))
    vx = np.abs(m - d[0] * n_b)
    vy = np.abs(m - d[1] * n_b)
    vz = np.abs(m - d[2] * n_b)
    vals = tab[vx[None, None, :], vy[None, :, None], vz[:, None, None]]
    k = np.zeros((S, S, S))
    idx = m % S
    k[np.ix_(idx, idx, idx)] = vals
    return k


class Spectra:
    """Cache of kernel spectra k_hat per (level, offset)."""

    def __init__(self, n_b: int):
        self.n_b = n_b
        self.cache = {}

    def get(self, l: int, d):
        key = (l, d)
        if key not in self.cache:
            n_b = self.n_b
            if l == 0:
                n, h = n_b, 1
            else:
                n, h = n_b + 1, 2 ** (l - 1)
            S = 2 * n
            self.cache[key] = np.fft.rfftn(kernel_vector(h, d, n, n_b, S))
        return self.cache[key]


# --------------------------------------------------------------------------
# The solve (Steps 1-3)


def fmm_solve(blocks, f, n_b: int, n_levels: int, order: int, spectra: Spectra | None = None,
              level_orders: dict | None = None):
    """u on every active block, shaped like f (n_blocks, n_b, n_b, n_b) [z, y, x].

    level_orders optionally maps a parent level l >= 2 to the interpolation
    order of the stencil between levels l and l - 1 (Interp from l, Reg into
    l); other levels use ``order`` (Sec. 4 allows the interval sizes and
    stencils to differ per level)."""
    blocks = np.asarray(blocks)
    f = np.asarray(f, dtype=np.float64)
    L = int(n_levels)
    n_I = n_b + 1
    S0, S = 2 * n_b, 2 * n_I
    lo = dict(level_orders or {})
    Wl = {l: interp_weights(n_b, lo.get(l, order) + 1) for l in range(2, L + 1)}
    levels = build_levels(blocks, L)
    sp = Spectra(n_b) if spectra is None else spectra
    bidx = {_key(v): i for i, v in enumerate(blocks)}

    # Step 1, upward pass: sources at nodes, then padded forward FFTs.
    ft = {}                                    # f~ per level: dict interval -> n_I^3
    fh = {0: {P: np.fft.rfftn(f[bidx[P]], s=(S0, S0, S0), axes=(0, 1, 2)) for P in levels[0]}}
    for l in range(1, L + 1):
        ft[l] = {}
        for P in levels[l]:
            if l == 1:
                x = np.zeros((n_I, n_I, n_I))
                x[:n_b, :n_b, :n_b] = f[bidx[P]]
            else:
                x = np.zeros((n_I, n_I, n_I))
                for c in np.ndindex(2, 2, 2):
                    Q = (2 * P[0] + c[2], 2 * P[1] + c[1], 2 * P[2] + c[0])
                    if Q in ft[l - 1]:
                        x += reg(Wl[l], _child_pos(Q), ft[l - 1][Q])
            ft[l][P] = x
        fh[l] = {P: np.fft.rfftn(ft[l][P], s=(S, S, S), axes=(0, 1, 2)) for P in levels[l]}

    # Step 2, level interactions: sum of spectral products over InflList.
    uh = {}
    for l in range(0, L + 1):
        uh[l] = {}
        mem = set(levels[l])
        for P in levels[l]:
            acc = None
            for Q in influence_list(levels, l, P, L, mem):
                d = (Q[0] - P[0], Q[1] - P[1], Q[2] - P[2])
                term = fh[l][Q] * sp.get(l, d)
                acc = term if acc is None else acc + term
            uh[l][P] = acc

    # Step 3, downward pass: truncated inverse FFTs plus interpolation.
    ut = {}
    for l in range(L, 0, -1):
        ut[l] = {}
        for P in levels[l]:
            v = (np.zeros((n_I, n_I, n_I)) if uh[l][P] is None
                 else np.fft.irfftn(uh[l][P], s=(S, S, S), axes=(0, 1, 2))[:n_I, :n_I, :n_I])
            if l < L:
                v = v + interp(Wl[l + 1], _child_pos(P), ut[l + 1][_parent(P)])
            ut[l][P] = v
    u = np.empty_like(f)
    for P in levels[0]:
        v = np.fft.irfftn(uh[0][P], s=(S0, S0, S0), axes=(0, 1, 2))[:n_b, :n_b, :n_b]
        u[bidx[P]] = v + ut[1][P][:n_b, :n_b, :n_b]
    return u


def rel_linf(u, ref) -> float:
    """max|u - ref| / max|ref| over the active points."""
    u = np.asarray(u, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.abs(u - ref).max() / np.abs(ref).max())
