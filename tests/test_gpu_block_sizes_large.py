"""Block sizes 18 to 32 (the run-time-size kernels: level-0 transforms of
2 n_b points, intervals of n_I = n_b + 1 nodes on 2 n_b + 2 points) through
the C ABI, against the oracle.

Tolerances as in test_gpu_parity.py: relative L-infinity 1e-12 (FP64) and
1e-5 (FP32) against the oracle FMM (non-negative sources, kappa = 1).  A
single block is the exact FFT convolution, checked against the direct sum.
The multi-level cases are irregular subsets of a torus box with three levels,
so that Reg and Interp run between levels 1 and 2."""
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


@pytest.mark.parametrize("n_b", [18, 20, 24, 32])
def test_single_block_is_fft_convolution(n_b):
    rng = np.random.default_rng(60 + n_b)
    blocks = np.array([[-3, 2, 1]], dtype=np.int32)
    f = rng.standard_normal((1, n_b, n_b, n_b))
    p = W.Problem(blocks, f, n_b, 1, 8, f"single{n_b}")
    ud = direct.direct_sum(blocks, n_b, f)
    e64, e32 = fmm.rel_linf(solve(p, lgfm.LGF_FP64), ud), fmm.rel_linf(solve(p, lgfm.LGF_FP32), ud)
    record_error(f"single_block_nb{n_b}", fp64_vs_direct=e64, fp32_vs_direct=e32)
    assert e64 <= TOL64 and e32 <= TOL32, (e64, e32)


_cache = {}
# (n_b, blocks per axis, kept fraction): 1.1e6, 1.3e6 and 2.4e6 points
CASES = {18: (8, 0.35), 24: (6, 0.4), 32: (6, 0.3)}


def subset_torus(n_b):
    if n_b not in _cache:
        nb, frac = CASES[n_b]
        box = W.torus_box(seed=50 + n_b, nb=nb, n_b=n_b, radius=0.3 * nb * n_b, sigma=0.08 * nb * n_b, order=8,
                          n_levels=3)
        p = W.block_subset(box, frac, seed=n_b)
        _cache[n_b] = (p, fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order))
    return _cache[n_b]


@pytest.mark.parametrize("n_b", sorted(CASES))
def test_subset_torus_against_oracle(n_b):
    p, ref = subset_torus(n_b)
    e64 = fmm.rel_linf(solve(p, lgfm.LGF_FP64), ref)
    e32 = fmm.rel_linf(solve(p, lgfm.LGF_FP32), ref)
    record_error(f"subset_torus_nb{n_b}_L3", fp64_vs_oracle=e64, fp32_vs_oracle=e32)
    assert e64 <= TOL64 and e32 <= TOL32, (e64, e32)


@pytest.mark.parametrize("n_b", [18, 24])
def test_four_levels_against_oracle(n_b):
    # four levels: Reg from level-2 intervals into level 3 and Interp into the
    # level-2 field (not only from and into blocks) on these kernels
    box = W.torus_box(seed=77, nb=12, n_b=n_b, radius=0.3 * 12 * n_b, sigma=0.08 * 12 * n_b, order=8,
                      n_levels=4)
    p = W.block_subset(box, 0.2, seed=5)
    ref = fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order)
    s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP32)
    st = s.stats()
    s.close()
    assert st["top_product_level"] >= 3
    e64 = fmm.rel_linf(solve(p, lgfm.LGF_FP64), ref)
    e32 = fmm.rel_linf(solve(p, lgfm.LGF_FP32), ref)
    record_error(f"subset_torus_nb{n_b}_L4", fp64_vs_oracle=e64, fp32_vs_oracle=e32)
    assert e64 <= TOL64 and e32 <= TOL32, (e64, e32)


@pytest.mark.parametrize("opts", [{"separate_level1": 1}, {"interval_kernel": 1}, {"interval_kernel": 4},
                                  {"single_stream": 1, "free_sms": 24}, {"free_sms": -1},
                                  {"interp_mode": lgfm.LGF_INTERP_COMPENSATED}])
def test_schedules_and_forms_nb18(opts):
    # the same sums whatever the schedule; n_b = 18 FP32 level-0 products run
    # the persistent kernel of 36-point transforms unless interval_kernel = 1
    p, ref = subset_torus(18)
    opts = dict(opts)
    mode = opts.pop("interp_mode", lgfm.LGF_INTERP_NATIVE)
    precs = ((lgfm.LGF_FP64, TOL64), (lgfm.LGF_FP32, TOL32))
    if mode != lgfm.LGF_INTERP_NATIVE:
        precs = precs[1:]          # the other modes are FP32 options
    for prec, tol in precs:
        s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, prec, interp_mode=mode, **opts)
        dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
        u = s(torch.from_numpy(p.f).to(dt).cuda())
        lgfm.lgf_plan_sync(s.plan)
        e = fmm.rel_linf(u.double().cpu().numpy(), ref)
        s.close()
        assert e <= tol, (prec, opts, mode, e)


@pytest.mark.parametrize("n_b", [24, 32])
@pytest.mark.parametrize("ik", [4, 5])
def test_persistent_products_large_lengths(n_b, ik):
    # the persistent products kernel at every level (interval_kernel 4: one
    # FMA per real product, 5: packed), transform lengths 48 / 50 (n_b = 24)
    # and 64 / 66 (n_b = 32); FP32 only
    p, ref = subset_torus(n_b)
    e = fmm.rel_linf(solve(p, lgfm.LGF_FP32, interval_kernel=ik), ref)
    record_error(f"subset_torus_nb{n_b}_persist{ik}", fp32_vs_oracle=e)
    assert e <= TOL32, e


def test_manufactured_nb20():
    # exact answer known (Sec. 4.1).  The random source (the Laplacian of
    # noise) is badly conditioned, so the FP64 difference from the oracle is
    # bounded relative to max|G * |f||, the size of the terms summed (kappa =
    # max|G * |f|| / max|u|, from the FP64 solve of |f|), and the error
    # against the exact answer equals the oracle's to within that
    m = W.manufactured(W.full_box_blocks(6), 20, 3, 9, seed=7)
    ref = fmm.fmm_solve(m.blocks, m.f, 20, 3, 9)
    u64 = solve(m, lgfm.LGF_FP64)
    kappa = float(np.abs(solve(m, lgfm.LGF_FP64, f=np.abs(m.f))).max() / np.abs(u64).max())
    e_ref = fmm.rel_linf(u64, ref)
    e_orc = fmm.rel_linf(ref, m.u_exact)
    e_gpu = fmm.rel_linf(u64, m.u_exact)
    record_error("manufactured_nb20_L3", fp64_vs_oracle=e_ref, oracle_vs_exact=e_orc, fp64_vs_exact=e_gpu,
                 kappa=kappa)
    assert e_ref <= TOL64 * kappa, (e_ref, kappa)
    assert abs(e_gpu - e_orc) <= TOL64 * kappa and e_orc < 1e-6


def test_repeat_solves_identical():
    # the transform scratch never holds state from one solve to the next
    p, _ = subset_torus(18)
    s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP32)
    f = torch.from_numpy(p.f).float().cuda()
    a = s(f).clone()
    s(torch.flip(f, dims=[0]))
    b = s(f)
    lgfm.lgf_plan_sync(s.plan)
    s.close()
    assert torch.equal(a, b)
