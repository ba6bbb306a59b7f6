"""Degenerate cases of the method on the GPU, each checked against something
other than the oracle FMM:
  * a zero source gives exactly zero (every step is linear);
  * a unit point source gives the lattice Green's function itself, u(n) =
    G(n - n0) (Eq. dpoissonsoln with f = delta), exact where no
    interpolation is involved (level 0 and level 1), compared with the
    oracle's own Bessel-integral G;
  * an empty block list is rejected;
  * translating the domain by whole top-level intervals leaves the tree,
    lists and arithmetic unchanged: identical bits."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
import workloads as W
from oracle import direct, lgf
from paper_1402_6081_gb300 import build as lgf_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    lgfm.library()


def solve(blocks, n_b, L, order, prec, f):
    dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
    s = lgfm.Solver(blocks, n_b, L, order, prec)
    u = s(torch.from_numpy(np.ascontiguousarray(f)).to(dt).cuda())
    torch.cuda.synchronize()
    out = u.double().cpu().numpy()
    s.close()
    return out


@pytest.mark.parametrize("n_b,L", [(8, 3), (16, 3), (20, 3)])
def test_zero_source_gives_zero(n_b, L):
    blocks = W.full_box_blocks(6)
    f = np.zeros((len(blocks), n_b, n_b, n_b))
    for prec in (lgfm.LGF_FP32, lgfm.LGF_FP64):
        assert not np.any(solve(blocks, n_b, L, 8, prec, f)), prec


@pytest.mark.parametrize("n_b", [8, 16, 20])
def test_point_source_gives_the_green_function(n_b):
    # 3^3 blocks, two levels: every block pair is near at level 0 or in a
    # level-1 interaction list computed on the grid points themselves (no
    # interpolation), so u is exactly G(n - n0) up to rounding
    blocks = W.full_box_blocks(3)
    f = np.zeros((len(blocks), n_b, n_b, n_b))
    b0, (i0, j0, k0) = 13, (n_b // 3, n_b // 2, n_b - 2)     # block (1, 1, 1), an off-centre point
    f[b0, k0, j0, i0] = 1.0
    n0 = blocks[b0] * n_b + np.array([i0, j0, k0])
    pts = direct.point_coords(blocks, n_b).reshape(len(blocks), n_b, n_b, n_b, 3)
    g = lgf.lgf(pts - n0)
    for prec, tol in ((lgfm.LGF_FP64, 1e-13), (lgfm.LGF_FP32, 1e-6)):
        u = solve(blocks, n_b, 2, 8, prec, f)
        err = np.abs(u - g).max() / np.abs(g).max()
        assert err <= tol, (prec, err)


def test_empty_block_list_rejected():
    with pytest.raises(lgfm.LgfError) as e:
        lgfm.lgf_plan_create(np.zeros((0, 3), dtype=np.int32), 8, 1, 4, lgfm.LGF_FP32)
    assert e.value.status == 1


@pytest.mark.parametrize("n_b", [8, 20])
def test_translation_by_top_level_intervals_is_bit_exact(n_b):
    # a 3-level irregular domain moved by (4, -8, 12) blocks (multiples of the
    # level-3 interval, 4 blocks): same bits, FP32 and FP64
    base = W.block_subset(W.torus_box(seed=4, nb=8, n_b=n_b, radius=0.3 * 8 * n_b, sigma=0.08 * 8 * n_b,
                                      order=8, n_levels=3), 0.5, seed=9)
    moved = base.blocks + np.array([4, -8, 12], dtype=np.int32)
    for prec in (lgfm.LGF_FP32, lgfm.LGF_FP64):
        a = solve(base.blocks, n_b, 3, 8, prec, base.f)
        b = solve(moved, n_b, 3, 8, prec, base.f)
        assert np.array_equal(a, b), prec
