"""Block sizes 6, 10, 12 and 14 (level-0 transforms of 12, 20, 24, 28 points,
intervals of n_I = 7, 11, 13, 15 nodes) and per-level interpolation orders,
through the C ABI, against the oracle.

Tolerances as in test_gpu_parity.py: relative L-infinity 1e-12 (FP64) and
1e-5 (FP32) against the oracle FMM; the non-negative sources here have kappa
= 1, so the bounds are plain.  A single block is the exact FFT convolution,
checked against the direct sum."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
import workloads as W
from oracle import direct, fmm
from paper_1402_6081_gb300 import build as lgf_build
from conftest import record_error

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5
NEW_SIZES = [6, 10, 12, 14]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    lgfm.library()


def solve(p, prec, f=None, **opts):
    dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
    s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, prec, **opts)
    u = s(torch.from_numpy(np.ascontiguousarray(p.f if f is None else f)).to(dt).cuda())
    lgfm.lgf_plan_sync(s.plan)
    out = u.double().cpu().numpy()
    s.close()
    return out


@pytest.mark.parametrize("n_b", NEW_SIZES)
def test_single_block_is_fft_convolution(n_b):
    rng = np.random.default_rng(30 + n_b)
    blocks = np.array([[2, -1, 5]], dtype=np.int32)
    f = rng.standard_normal((1, n_b, n_b, n_b))
    p = W.Problem(blocks, f, n_b, 1, min(n_b, 8), f"single{n_b}")
    ud = direct.direct_sum(blocks, n_b, f)
    assert fmm.rel_linf(solve(p, lgfm.LGF_FP64), ud) <= TOL64
    assert fmm.rel_linf(solve(p, lgfm.LGF_FP32), ud) <= TOL32


_cache = {}


def torus(n_b):
    # about 80^3 points: 3 levels for n_b >= 10, 4 for n_b = 6 (level 2 and up interpolated)
    if n_b not in _cache:
        nb = -(-80 // n_b)
        p = W.torus_box(seed=40 + n_b, nb=nb, n_b=n_b, radius=0.3 * nb * n_b, sigma=0.06 * nb * n_b,
                        order=min(8, n_b))
        _cache[n_b] = (p, fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order))
    return _cache[n_b]


@pytest.mark.parametrize("n_b", NEW_SIZES)
def test_torus_against_oracle(n_b):
    p, ref = torus(n_b)
    e64 = fmm.rel_linf(solve(p, lgfm.LGF_FP64), ref)
    e32 = fmm.rel_linf(solve(p, lgfm.LGF_FP32), ref)
    record_error(f"torus_nb{n_b}_L{p.n_levels}", fp64_vs_oracle=e64, fp32_vs_oracle=e32)
    assert p.n_levels >= 3
    assert e64 <= TOL64 and e32 <= TOL32, (e64, e32)


@pytest.mark.parametrize("n_b", [6, 12])
@pytest.mark.parametrize("opts", [{"separate_level1": 1}, {"interval_kernel": 1}, {"interval_kernel": 5},
                                  {"single_stream": 1, "free_sms": 24}, {"free_sms": -1}])
def test_schedules_and_forms(n_b, opts):
    # the same sums whatever the kernel forms and schedule
    p, ref = torus(n_b)
    for prec, tol in ((lgfm.LGF_FP64, TOL64), (lgfm.LGF_FP32, TOL32)):
        assert fmm.rel_linf(solve(p, prec, **opts), ref) <= tol, (prec, opts)


def test_manufactured_deep_tree_nb10():
    # 4 levels with n_b = 10: exact answer known (Sec. 4.1); the GPU error
    # against it equals the oracle's to within the FP64 rounding
    m = W.manufactured(W.full_box_blocks(10), 10, 4, 9, seed=5)
    ref = fmm.fmm_solve(m.blocks, m.f, 10, 4, 9)
    u64 = solve(m, lgfm.LGF_FP64)
    e_orc = fmm.rel_linf(ref, m.u_exact)
    e_gpu = fmm.rel_linf(u64, m.u_exact)
    record_error("manufactured_nb10_L4", fp64_vs_oracle=fmm.rel_linf(u64, ref), oracle_vs_exact=e_orc,
                 fp64_vs_exact=e_gpu)
    assert abs(e_gpu - e_orc) <= 1e-3 * e_orc and e_orc < 1e-6


def test_level_orders_against_oracle():
    # per-level stencils: order 9 between levels 2 and 1, order 5 between 3
    # and 2, 3 between 4 and 3 (Sec. 4: n_I and the stencils may differ per level)
    p = W.torus_box(seed=8, nb=16, n_b=8, radius=40.0, sigma=7.0, n_levels=4)
    lo = {2: 8, 3: 4, 4: 2}
    ref = fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order, level_orders=lo)
    uni = fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order)
    assert fmm.rel_linf(uni, ref) > 1e-9          # the orders change the result
    e64 = fmm.rel_linf(solve(p, lgfm.LGF_FP64, level_orders=lo), ref)
    e32 = fmm.rel_linf(solve(p, lgfm.LGF_FP32, level_orders=lo), ref)
    record_error("torus_128_nb8_level_orders", fp64_vs_oracle=e64, fp32_vs_oracle=e32)
    assert e64 <= TOL64 and e32 <= TOL32, (e64, e32)


def test_block_size_errors():
    b = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.int32)
    for n_b, status in ((7, 1), (2, 1), (34, 1), (19, 1), (0, 1)):
        with pytest.raises(lgfm.LgfError) as e:
            lgfm.lgf_plan_create(b, n_b, 1, 3, lgfm.LGF_FP32)
        assert e.value.status == status, n_b
    for n_b in (10, 20):
        with pytest.raises(lgfm.LgfError) as e:
            lgfm.lgf_plan_create(b, n_b, 1, 3, lgfm.LGF_FP32, lgfm.LGF_INTERP_BF16)
        assert e.value.status == 2
    with pytest.raises(lgfm.LgfError) as e:
        lgfm.Solver(b, 20, 1, 3, lgfm.LGF_FP32, fft_kernel=2)
    assert e.value.status == 1
    with pytest.raises(lgfm.LgfError) as e:
        lgfm.Solver(b, 8, 1, 3, lgfm.LGF_FP32, level_orders={2: 9})
    assert e.value.status == 1
