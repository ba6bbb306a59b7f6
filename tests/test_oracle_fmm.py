"""Pins of the CPU FMM oracle (oracle/fmm.py).

Each check rests on something other than the oracle itself: the exact direct
sum where the method involves no interpolation (Sec. 4.1 notes those cases sit
at machine precision), the exact random manufactured solution of Sec. 4.1,
dense sums, polynomial exactness, adjointness, the list sizes of Sec. 3.2, and
invariances of the discrete problem.
"""
import numpy as np
import pytest

import workloads as W
from oracle import direct, fmm, lgf


def test_two_level_gaussian_equals_direct_sum():
    # 32^3 grid, 4^3 blocks, 2 levels: level-1 nodes are grid points and the
    # top level has no interaction list, so the FMM is exact up to rounding.
    p = W.config(0)
    u = fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order)
    ud = direct.direct_sum(p.blocks, p.n_b, p.f)
    assert fmm.rel_linf(u, ud) < 1e-13


def test_single_block_is_fft_convolution():
    rng = np.random.default_rng(3)
    blocks = np.array([[2, -1, 5]], dtype=np.int32)
    f = rng.standard_normal((1, 8, 8, 8))
    u = fmm.fmm_solve(blocks, f, 8, 1, 6)
    assert fmm.rel_linf(u, direct.direct_sum(blocks, 8, f)) < 1e-13


def test_irregular_two_level_equals_direct_sum():
    # scattered blocks, general top-level rule (L = 1 and L = 2)
    rng = np.random.default_rng(11)
    blocks = np.array([[0, 0, 0], [1, 0, 0], [3, 1, 0], [0, 3, 2], [2, 2, 3], [3, 3, 3]],
                      dtype=np.int32)
    f = rng.uniform(-1, 1, size=(len(blocks), 4, 4, 4))
    ud = direct.direct_sum(blocks, 4, f)
    for L in (1, 2):
        assert fmm.rel_linf(fmm.fmm_solve(blocks, f, 4, L, 3), ud) < 1e-13


def test_block_fft_convolution_matches_dense_sum():
    # Sec. 2.2 Pad/FFT/Prod/FFT^-1/Trunc with k(m) = G(h(m - d n_b)) at m mod S:
    # the block-pair field equals the dense sum over the source block.
    n_b, h = 4, 2
    d = (1, 0, -2)
    rng = np.random.default_rng(7)
    fq = rng.standard_normal((n_b, n_b, n_b))              # [z, y, x]
    S = 2 * n_b
    k = fmm.kernel_vector(h, d, n_b, n_b, S)
    u = np.fft.irfftn(np.fft.rfftn(fq, s=(S, S, S), axes=(0, 1, 2)) * np.fft.rfftn(k), s=(S, S, S), axes=(0, 1, 2))[:n_b, :n_b, :n_b]
    ref = np.zeros_like(u)
    for iz, iy, ix in np.ndindex(n_b, n_b, n_b):
        s = 0.0
        for jz, jy, jx in np.ndindex(n_b, n_b, n_b):
            # target node of P minus source node of Q, in grid units
            v = h * np.array([ix - jx - d[0] * n_b, iy - jy - d[1] * n_b, iz - jz - d[2] * n_b])
            s += lgf.lgf([v])[0] * fq[jz, jy, jx]
        ref[iz, iy, ix] = s
    assert np.abs(u - ref).max() < 1e-15 * 100


@pytest.mark.parametrize("n_b,n_max", [(8, 7), (8, 9), (16, 9), (16, 10), (6, 4)])
def test_interpolation_weights(n_b, n_max):
    Wt = fmm.interp_weights(n_b, n_max)
    n_I = n_b + 1
    # reproduces polynomials of degree <= n_max - 1 exactly (Sec. 2.5)
    p = np.arange(n_I, dtype=float)
    for c in (0, 1):
        x = c * n_b / 2 + np.arange(n_I) / 2
        for deg in range(n_max):
            assert np.allclose(Wt[c] @ (p / n_b) ** deg, (x / n_b) ** deg, atol=1e-12)
        # at most n_max non-zeros per row, inside the interval
        assert np.all((np.abs(Wt[c]) > 0).sum(axis=1) <= n_max)
    # mirror symmetry of the centre-ward tie rule (even n_b)
    if n_b % 2 == 0:
        assert np.abs(Wt[1][::-1, ::-1] - Wt[0]).max() < 1e-14


def test_reg_is_adjoint_of_interp():
    Wt = fmm.interp_weights(8, 7)
    rng = np.random.default_rng(0)
    U = rng.standard_normal((9, 9, 9))
    F = rng.standard_normal((9, 9, 9))
    for c in np.ndindex(2, 2, 2):
        lhs = np.sum(fmm.interp(Wt, c, U) * F)
        rhs = np.sum(U * fmm.reg(Wt, c, F))
        assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)
    # and interp on one axis equals an explicit loop with the 1D weights
    c = (1, 0, 1)
    ref = np.einsum("ip,jq,kr,pqr->ijk", Wt[c[2]], Wt[c[1]], Wt[c[0]], U)
    assert np.allclose(fmm.interp(Wt, c, U), ref, atol=1e-13)


def test_list_sizes():
    # Sec. 3.2: 27 near neighbours, 189 interaction-list members, and
    # 7^3 - 3^3 = 316 distinct offsets (the paper prints 317).
    blocks = W.full_box_blocks(8)
    L = 3
    levels = fmm.build_levels(blocks, L)
    mem = set(levels[1])
    P = (3, 4, 3)
    assert len(fmm.influence_list(levels, 0, P, L)) == 27
    assert len(fmm.influence_list(levels, 1, P, L, mem)) == 189
    offs = set()
    for Q in levels[1]:
        for R in fmm.influence_list(levels, 1, Q, L, mem):
            offs.add((R[0] - Q[0], R[1] - Q[1], R[2] - Q[2]))
    assert len(offs) == 316
    # each pair of blocks is counted exactly once over the levels
    count = {}
    for l in range(0, L + 1):
        ml = set(levels[l])
        for Pl in levels[l]:
            for Ql in fmm.influence_list(levels, l, Pl, L, ml):
                count[(l, Pl, Ql)] = 1
    per_pair = np.zeros((len(blocks), len(blocks)), dtype=int)
    bl = [tuple(b) for b in blocks]
    for i, a in enumerate(bl):
        for j, b in enumerate(bl):
            for l in range(0, L + 1):
                s = max(l - 1, 0)
                key = (l, (a[0] >> s, a[1] >> s, a[2] >> s), (b[0] >> s, b[1] >> s, b[2] >> s))
                per_pair[i, j] += key in count
    assert np.all(per_pair == 1)


def test_manufactured_solution_two_levels_exact():
    m = W.manufactured(W.full_box_blocks(4), 8, 2, 6, seed=4)
    u = fmm.fmm_solve(m.blocks, m.f, m.n_b, m.n_levels, m.order)
    assert fmm.rel_linf(u, m.u_exact) < 1e-13


def test_manufactured_solution_truncation_trend():
    # Sec. 4.1: with interpolation the error is the method's truncation error,
    # falling steeply with n_I at fixed n_max (n_I^-10 for n_max = 10).
    e = []
    for n_b in (8, 16):
        m = W.manufactured(W.full_box_blocks(8), n_b, 3, 8, seed=0)
        u = fmm.fmm_solve(m.blocks, m.f, m.n_b, m.n_levels, m.order)
        e.append(fmm.rel_linf(u, m.u_exact))
    assert 1e-9 < e[0] < 1e-5
    assert e[1] < e[0] / 50


def test_linearity_translation_permutation():
    rng = np.random.default_rng(2)
    blocks = W.full_box_blocks(4)
    n_b, L, order = 4, 2, 3
    f1 = rng.standard_normal((len(blocks), n_b, n_b, n_b))
    f2 = rng.standard_normal((len(blocks), n_b, n_b, n_b))
    u1 = fmm.fmm_solve(blocks, f1, n_b, L, order)
    u2 = fmm.fmm_solve(blocks, f2, n_b, L, order)
    u12 = fmm.fmm_solve(blocks, 2 * f1 - 3 * f2, n_b, L, order)
    assert fmm.rel_linf(u12, 2 * u1 - 3 * u2) < 1e-13
    # shift by whole top-level intervals: identical arithmetic, identical bits
    shift = np.array([2, -4, 6], dtype=np.int32)
    assert np.array_equal(fmm.fmm_solve(blocks + shift, f1, n_b, L, order), u1)
    # permuted block list: same field per block
    perm = rng.permutation(len(blocks))
    up = fmm.fmm_solve(blocks[perm], f1[perm], n_b, L, order)
    assert np.array_equal(up, u1[perm])


def test_mirror_symmetry():
    # Reflecting the source about a mid-plane reflects u exactly when no
    # interpolation takes part (one level: all far pairs at level 1).  With interpolation the one-node
    # interval overlap always sits on the +axis side, so the mirrored domain sees
    # shifted nodes and the two results agree only to the truncation error.
    rng = np.random.default_rng(9)
    blocks = W.full_box_blocks(8)
    n_b = 4
    f = rng.standard_normal((len(blocks), n_b, n_b, n_b))
    mb = blocks.copy()
    mb[:, 0] = 7 - mb[:, 0]
    fm = f[:, :, :, ::-1]
    u2 = fmm.fmm_solve(blocks, f, n_b, 1, 4)
    um2 = fmm.fmm_solve(mb, fm, n_b, 1, 4)
    assert fmm.rel_linf(um2[:, :, :, ::-1], u2) < 1e-13
    u3 = fmm.fmm_solve(blocks, f, n_b, 3, 4)
    um3 = fmm.fmm_solve(mb, fm, n_b, 3, 4)
    e_mirror = fmm.rel_linf(um3[:, :, :, ::-1], u3)
    e_trunc = fmm.rel_linf(u3, u2)          # u2 is exact (no interpolation)
    assert e_mirror <= 2.5 * e_trunc
