"""Reduced-precision interpolation modes (Reg and Interp as tensor-core GEMMs,
tcgen05.mma kind::f16, FP32 accumulation) against the FP64 oracle.

Bounds.  Only the interpolated far field (levels >= 2) sees the rounding.
Each axis pass of Reg and of Interp rounds its inputs (field values and
weights) to the mode's type, unit roundoff u = 2^-8 (BF16), 2^-11 (FP16),
about 2^-24 for BF16x3 (three-part split, six products).  A field passes
through up to 12 such roundings (3 Reg + 3 Interp passes at each of two
levels in these 4-level trees), each amplified by the Lebesgue constant of the
order-8 stencil (about 3), so |error| <= 36 u of the far field, which is below
max|u|; the bound is 48 u: 0.19 (BF16) and 2.3e-2 (FP16).  Measured: 31 u
(BF16) and 27 u (FP16).  The bound is a model of trees of up to 4 levels:
each further level adds six rounded passes whose error the levels below
amplify again (the 5-level 512^3 domain measures 0.40 BF16, 5.6e-2 FP16), so
the header states the depth it holds to and these tests stay at 3-4 levels.
BF16x3 must meet the FP32 contract (1e-5), and so
must the compensated FP32 mode (CUDA cores, Dot2 sums), which is no less
accurate than the native one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
import workloads as W
from oracle import fmm
from paper_1402_6081_gb300 import build as lgf_build
from conftest import record_error

pytestmark = pytest.mark.gpu

BOUND = {lgfm.LGF_INTERP_BF16: 48 * 2.0 ** -8, lgfm.LGF_INTERP_FP16: 48 * 2.0 ** -11,
         lgfm.LGF_INTERP_BF16X3: 1e-5, lgfm.LGF_INTERP_COMPENSATED: 1e-5}


@pytest.fixture(scope="session", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    lgfm.library()


_ref = {}


def _problem(n_b):
    if n_b == 16:
        return W.torus_box(seed=2, nb=6, n_b=16, radius=30.0, sigma=5.0, n_levels=3)
    return W.torus_box(seed=3, nb=8, n_b=n_b, radius=0.3 * 8 * n_b, sigma=0.06 * 8 * n_b, n_levels=4)


def _oracle(p):
    key = (p.name, p.n_b, p.n_levels)
    if key not in _ref:
        _ref[key] = fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order)
    return _ref[key]


def _solve(p, mode, **opts):
    s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP32, interp_mode=mode, **opts)
    u = s(torch.from_numpy(p.f).float().cuda())
    lgfm.lgf_plan_sync(s.plan)
    out = u.double().cpu().numpy()
    s.close()
    return out


@pytest.mark.parametrize("n_b", [8, 16])
@pytest.mark.parametrize("mode", [lgfm.LGF_INTERP_BF16, lgfm.LGF_INTERP_FP16, lgfm.LGF_INTERP_BF16X3,
                                  lgfm.LGF_INTERP_COMPENSATED])
def test_mode_against_oracle(n_b, mode):
    p = _problem(n_b)
    ref = _oracle(p)
    err = fmm.rel_linf(_solve(p, mode), ref)
    native = fmm.rel_linf(_solve(p, lgfm.LGF_INTERP_NATIVE), ref)
    record_error(f"{p.name}_nb{n_b}_interp{mode}", fp32_vs_oracle=err, native_fp32_vs_oracle=native)
    print(f"n_b {n_b} mode {mode}: {err:.3e} (native {native:.3e})")
    assert err <= BOUND[mode], (mode, err)
    # (the compensated mode's total error need not be below the native one's
    # here: the FP32 transforms and products dominate in these shallow trees,
    # and their rounding pattern decides the maximum; the 5-level 512^3 test
    # shows the gain where the interpolation sums matter)
    assert err >= 0.5 * native or mode in (lgfm.LGF_INTERP_BF16X3, lgfm.LGF_INTERP_COMPENSATED)


def test_bf16x3_close_to_native_and_split_schedule():
    # both schedules (split with the persistent products, and one-CTA-per-chunk
    # products beside the level-0 pass) and the native mode agree to FP32
    # accuracy (each is within 1e-5 of the oracle)
    p = _problem(16)
    a = _solve(p, lgfm.LGF_INTERP_BF16X3)
    b = _solve(p, lgfm.LGF_INTERP_BF16X3, interval_kernel=1)
    c = _solve(p, lgfm.LGF_INTERP_NATIVE)
    scale = np.abs(c).max()
    assert np.abs(a - c).max() / scale <= 1e-5
    assert np.abs(a - b).max() / scale <= 1e-5


def test_mode_n_b4():
    blocks = W.full_box_blocks(8)
    rng = np.random.default_rng(4)
    f = rng.uniform(0.0, 1.0, size=(len(blocks), 4, 4, 4))
    p = W.Problem(blocks, f, 4, 3, 3, "nb4_box")
    ref = _oracle(p)
    err = fmm.rel_linf(_solve(p, lgfm.LGF_INTERP_BF16X3), ref)
    record_error("nb4_box_interp3", fp32_vs_oracle=err)
    assert err <= 1e-5, err


def test_mode_errors():
    b = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.int32)
    with pytest.raises(lgfm.LgfError, match="FP32"):
        lgfm.lgf_plan_create(b, 8, 1, 4, lgfm.LGF_FP64, lgfm.LGF_INTERP_BF16)
    with pytest.raises(lgfm.LgfError):
        lgfm.lgf_plan_create(b, 8, 1, 4, lgfm.LGF_FP32, 7)
