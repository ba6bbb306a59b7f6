"""Truncation error of the method against exact manufactured solutions
(Sec. 4.1) on cube, sphere and spherical-shell active grids of the same
physical size, for interval sizes n_I = 5, 9, 17 at a fixed interpolation
order: the paper's error experiment (Sec. 4, error against n_I at fixed n_max).
The FP64 path is used, so the error is the method's own; at fixed n_max it
falls as n_I grows (finer intervals relative to the kernel's smoothness).
Every GPU result is also compared with the oracle FMM on the same domain,
element by element: the GPU computes the same truncated method, so FP64 agrees
with it to 1e-12 and FP32 to 1e-5, both times the source's conditioning kappa =
max|G * |f|| / max|G * f| (about 2e3 for these random manufactured sources;
the oracle's solve of |f|).  Rates (points/s, FP32 and FP64) are recorded with
the errors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
import workloads as W
from oracle import fmm
from paper_1402_6081_gb300 import build as lgf_build
from conftest import record_error

pytestmark = pytest.mark.gpu

DIAMETER = 96
ORDER = 4           # n_max = 5 <= n_I for every block size


@pytest.fixture(scope="session", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    lgfm.library()


def _solve(m, prec, reps=3):
    dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
    s = lgfm.Solver(m.blocks, m.n_b, m.n_levels, m.order, prec)
    f = torch.from_numpy(m.f).to(dt).cuda()
    u = torch.empty_like(f)
    s(f, u)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        s(f, u)
    b.record()
    b.synchronize()
    rate = m.n_points * reps / (a.elapsed_time(b) * 1e-3)
    out = u.double().cpu().numpy()
    s.close()
    return out, rate


@pytest.mark.parametrize("shape", ["box", "sphere", "shell"])
def test_error_falls_with_interval_size(shape):
    errs = []
    for n_b in (4, 8, 16):
        blocks = W.shape_blocks(shape, DIAMETER, n_b)
        L = W.levels_for(int(np.ceil(DIAMETER / n_b)))
        m = W.manufactured(blocks, n_b, L, ORDER, seed=11)
        u64, r64 = _solve(m, lgfm.LGF_FP64)
        u32, r32 = _solve(m, lgfm.LGF_FP32)
        e64 = fmm.rel_linf(u64, m.u_exact)
        e32 = fmm.rel_linf(u32, m.u_exact)
        ref = fmm.fmm_solve(m.blocks, m.f, n_b, L, ORDER)
        kappa = max(1.0, float(np.abs(fmm.fmm_solve(m.blocks, np.abs(m.f), n_b, L, ORDER)).max()
                               / np.abs(ref).max()))
        p64, p32 = fmm.rel_linf(u64, ref), fmm.rel_linf(u32, ref)
        record_error(f"sweep_{shape}_nI{n_b + 1}", fp64_vs_exact=e64, fp32_vs_exact=e32, points=m.n_points,
                     fp64_points_per_s=r64, fp32_points_per_s=r32, fp64_vs_oracle=p64, fp32_vs_oracle=p32,
                     oracle_vs_exact=fmm.rel_linf(ref, m.u_exact), kappa=kappa)
        print(f"{shape} n_I {n_b + 1}: fp64 err {e64:.3e} fp32 err {e32:.3e} vs oracle {p64:.2e}/{p32:.2e} "
              f"kappa {kappa:.0f} rate fp32 {r32:.3e} fp64 {r64:.3e} points {m.n_points}")
        assert p64 <= 1e-12 * kappa, (n_b, p64, kappa)
        assert p32 <= 1e-5 * kappa, (n_b, p32, kappa)
        errs.append(e64)
    assert errs[0] > errs[1] > errs[2], errs


@pytest.mark.parametrize("shape", ["box", "sphere", "shell"])
def test_error_trend_at_n_max_10(shape):
    # The paper's setting (Sec. 4.1): n_max = 10 nodes per point, n_I = n_b + 1
    # > n_max, where the error should fall like n_I^-10 (measured there:
    # n_I^-10.7 for n_I = 11..28).  Block sizes 10..16 give n_I = 11..17.
    errs, n_is = [], []
    for n_b in (10, 12, 14, 16):
        blocks = W.shape_blocks(shape, DIAMETER, n_b)
        L = W.levels_for(int(np.ceil(DIAMETER / n_b)))
        m = W.manufactured(blocks, n_b, L, 9, seed=11)
        u64, r64 = _solve(m, lgfm.LGF_FP64)
        u32, r32 = _solve(m, lgfm.LGF_FP32)
        ref = fmm.fmm_solve(m.blocks, m.f, n_b, L, 9)
        kappa = max(1.0, float(np.abs(fmm.fmm_solve(m.blocks, np.abs(m.f), n_b, L, 9)).max()
                               / np.abs(ref).max()))
        e64, e_orc = fmm.rel_linf(u64, m.u_exact), fmm.rel_linf(ref, m.u_exact)
        p64, p32 = fmm.rel_linf(u64, ref), fmm.rel_linf(u32, ref)
        record_error(f"sweep10_{shape}_nI{n_b + 1}", fp64_vs_exact=e64, oracle_vs_exact=e_orc, fp64_vs_oracle=p64,
                     fp32_vs_oracle=p32, kappa=kappa, points=m.n_points, fp64_points_per_s=r64,
                     fp32_points_per_s=r32)
        print(f"n_max 10 {shape} n_I {n_b + 1}: fp64 err {e64:.3e} (oracle {e_orc:.3e}) vs oracle {p64:.2e}/"
              f"{p32:.2e} kappa {kappa:.0f}")
        assert p64 <= 1e-12 * kappa and p32 <= 1e-5 * kappa, (n_b, p64, p32, kappa)
        errs.append(e64)
        n_is.append(n_b + 1)
    slope = float(np.polyfit(np.log(n_is), np.log(errs), 1)[0])
    record_error(f"sweep10_{shape}_slope", slope=slope)
    print(f"n_max 10 {shape}: error ~ n_I^{slope:.2f}")
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert -13.0 < slope < -9.0, slope


def test_error_trend_to_n_I_27_box():
    # The paper's range n_I = 11..28 (Sec. 4.1) with the even block sizes:
    # n_I = 11..27 at n_max = 10 on a 128^3 box, against the exact answer.
    # The error falls like n_I^-10 until it meets the FP64 rounding floor of
    # this random source (kappa ~ 2e3; a few 1e-11), so the slope is fitted
    # below n_I = 25 and the largest sizes are only required to stay at the
    # floor.  n_b >= 18 runs the run-time-size kernels.
    errs, n_is = [], []
    for n_b in (10, 14, 18, 22, 26):
        blocks = W.shape_blocks("box", 128, n_b)
        L = W.levels_for(int(np.ceil(128 / n_b)))
        m = W.manufactured(blocks, n_b, L, 9, seed=11)
        u64, r64 = _solve(m, lgfm.LGF_FP64)
        e64 = fmm.rel_linf(u64, m.u_exact)
        record_error(f"sweep10_box128_nI{n_b + 1}", fp64_vs_exact=e64, points=m.n_points, fp64_points_per_s=r64,
                     levels=L)
        print(f"n_max 10 box 128 n_I {n_b + 1} (L {L}): fp64 err {e64:.3e}")
        errs.append(e64)
        n_is.append(n_b + 1)
    slope = float(np.polyfit(np.log(n_is[:4]), np.log(errs[:4]), 1)[0])
    record_error("sweep10_box128_slope_nI_11_23", slope=slope)
    print(f"n_max 10 box 128: error ~ n_I^{slope:.2f} (n_I 11..23)")
    assert all(a > b for a, b in zip(errs[:4], errs[1:4])), errs
    assert -13.0 < slope < -9.0, slope
    assert errs[-1] < 1e-10, errs
