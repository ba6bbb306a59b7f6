"""Host-buffer solves and the measured arithmetic peak, through the C ABI.

lgf_solve_host_pipelined overlaps each step's copies with the neighbouring
steps' solves inside the library; every step must return the bits of a plain
device solve of the same input (same kernels, same arithmetic).
lgf_measure_fma_peak must report rates inside what the hardware can do: at
most 152 SMs x 128 FP32 lanes x 2 flop x the maximum SM clock for FP32, and
FP64 well below FP32 on this part."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
import workloads as W
from paper_1402_6081_gb300 import build as lgf_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    lgfm.library()


@pytest.mark.parametrize("prec", [lgfm.LGF_FP32, lgfm.LGF_FP64])
def test_pipelined_host_solves_equal_device_solves(prec):
    p = W.torus_box(seed=4, nb=4, n_b=8, radius=10.0, sigma=3.0, n_levels=3)
    dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
    s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, prec)
    rng = np.random.default_rng(9)
    n = 5
    fs = [torch.from_numpy(p.f * (1.0 + 0.1 * k) + 0.01 * rng.standard_normal(p.f.shape)).to(dt).pin_memory()
          for k in range(n)]
    us = [torch.full_like(x, float("nan")).pin_memory() for x in fs]
    stream = torch.cuda.Stream()
    lgfm.lgf_solve_host_pipelined(s.plan, fs, us, stream)
    for k in range(n):
        ref = s(fs[k].cuda())
        torch.cuda.synchronize()
        assert torch.equal(us[k], ref.cpu()), k
    # repeated output buffers are written in step order: the last step wins
    u1 = torch.empty_like(fs[0]).pin_memory()
    lgfm.lgf_solve_host_pipelined(s.plan, fs[:3], [u1] * 3, stream)
    assert torch.equal(u1, s(fs[2].cuda()).cpu())
    lgfm.lgf_solve_host_pipelined(s.plan, [], [], stream)
    s.close()


def test_measured_fma_peaks_are_physical():
    props = torch.cuda.get_device_properties(0)
    n_sm = props.multi_processor_count
    r32, ms32 = lgfm.lgf_measure_fma_peak(1, 2)
    r2, ms2 = lgfm.lgf_measure_fma_peak(2, 2)
    r64, ms64 = lgfm.lgf_measure_fma_peak(0, 2)
    bound = n_sm * 128 * 2 * 2.2e9            # lanes x 2 flop x a clock above the 2.07 GHz maximum
    for r, ms in ((r32, ms32), (r2, ms2), (r64, ms64)):
        assert ms > 1.0 and 0 < r <= bound, (r, ms)
    assert max(r32, r2) > 0.3 * bound          # the FP32 pipes really run
    assert r64 < 0.5 * max(r32, r2)
    with pytest.raises(lgfm.LgfError):
        lgfm.lgf_measure_fma_peak(3, 1)
