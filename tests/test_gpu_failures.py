"""Failure paths, made on the host or by a wait that nothing completes; none
faults, traps or hangs the GPU:
  * the bounded device wait (mbarrier phase, %globaltimer limit) returns an
    error status and the context stays usable;
  * a workspace allocation that fails (fault injected by LGF_FAULT_ALLOC_AT)
    fails plan creation cleanly, at any point of the build, and later plans
    work."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
import workloads as W
from paper_1402_6081_gb300 import build as lgf_build

pytestmark = pytest.mark.gpu

LGF_ERR_OOM, LGF_ERR_TIMEOUT = 3, 5


@pytest.fixture(scope="session", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    lgfm.library()


def _solve(p):
    s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP32)
    u = s(torch.from_numpy(p.f).float().cuda())
    lgfm.lgf_plan_sync(s.plan)
    out = u.cpu().numpy()
    s.close()
    return out


def test_bounded_wait_completes_and_times_out():
    p = W.torus_box(seed=5, nb=4, n_b=8, radius=10.0, sigma=3.0)
    before = _solve(p)
    lgfm.lgf_selftest_bounded_wait(1, 1000)
    with pytest.raises(lgfm.LgfError) as ei:
        lgfm.lgf_selftest_bounded_wait(0, 2000)
    assert ei.value.status == LGF_ERR_TIMEOUT
    # the context is intact: the same solve gives the same bits
    assert np.array_equal(_solve(p), before)


def test_injected_allocation_failure_at_every_point():
    # fail the 1st, 2nd, ... allocation of a 3-level plan until the build no
    # longer reaches the failing one: every failure point fails cleanly
    p = W.torus_box(seed=6, nb=4, n_b=16, radius=20.0, sigma=4.0, n_levels=3)
    ref = _solve(p)
    failures = 0
    for k in range(1, 80):
        os.environ["LGF_FAULT_ALLOC_AT"] = str(k)
        try:
            s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP32)
        except lgfm.LgfError as exc:
            assert exc.status == LGF_ERR_OOM and "injected" in str(exc)
            failures += 1
            continue
        finally:
            del os.environ["LGF_FAULT_ALLOC_AT"]
        s.close()
        break
    assert failures >= 5
    assert np.array_equal(_solve(p), ref)
