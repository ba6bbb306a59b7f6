"""The no-allocation entry point against the planned solve.

lgf_solve_blocks_noalloc serves callers that cannot allocate device memory while
they run; it keeps its working memory in a fixed device array inside the
library.  Each block it solves is an isolated one-block problem, which is what
lgf_solve computes for a one-block plan, so every block of its output is
compared with that, element by element, within the tolerances of the parity
tests (relative L-infinity 1e-12 in FP64, 1e-5 in FP32).  Two calls run back to
back with different data and block counts, since calls share the array, and the
second call must leave the device's free memory and torch's allocation count
unchanged: it allocates nothing.  This file sorts last so that a run stopping at
its first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
from paper_1402_6081_gb300 import build as lgf_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    lgfm.library()


def planned_one_block(f_block, n_b, prec):
    dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
    s = lgfm.Solver(np.array([[0, 0, 0]], dtype=np.int32), n_b, 1, min(n_b, 6), prec)
    u = s(f_block.to(dt).contiguous())
    torch.cuda.synchronize()
    out = u.double().cpu().numpy()
    s.close()
    return out


@pytest.mark.parametrize("prec,tol", [(lgfm.LGF_FP32, 1e-5), (lgfm.LGF_FP64, 1e-12)])
@pytest.mark.parametrize("n_b", [4, 8, 16])
def test_noalloc_matches_planned_solve(prec, tol, n_b):
    dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
    rng = np.random.default_rng(100 + n_b)
    for call, n in enumerate((5, 3)):      # two calls in a row, different sizes
        f = torch.from_numpy(rng.uniform(-1.0, 1.0, size=(n, n_b, n_b, n_b))).to(dt).cuda()
        u = torch.full_like(f, float("nan"))
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        lgfm.lgf_solve_blocks_noalloc(f, u, n, n_b, prec)
        torch.cuda.synchronize()
        if call == 1:
            # after the first call on the device nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
        got = u.double().cpu().numpy()
        for b in range(n):
            ref = planned_one_block(f[b:b + 1], n_b, prec)[0]
            err = np.abs(got[b] - ref).max() / np.abs(ref).max()
            assert err <= tol, (n, b, err)


def test_noalloc_rejects_too_many_blocks():
    mx = lgfm.lgf_noalloc_max_blocks(16, lgfm.LGF_FP32)
    assert mx == 232
    f = torch.zeros((1, 16, 16, 16), device="cuda")
    u = torch.zeros_like(f)
    with pytest.raises(lgfm.LgfError) as e:
        lgfm.lgf_solve_blocks_noalloc(f, u, mx + 1, 16, lgfm.LGF_FP32)
    assert e.value.status == 1          # LGF_ERR_INVALID_ARG
    assert "exceed the limit" in str(e.value)


def test_noalloc_rejects_overlapping_buffers():
    # u starting inside f (one block later) would overwrite sources still to be read
    f = torch.zeros((4, 8, 8, 8), device="cuda")
    with pytest.raises(lgfm.LgfError) as e:
        lgfm.lgf_solve_blocks_noalloc(f[:3], f[1:], 3, 8, lgfm.LGF_FP32)
    assert e.value.status == 1 and "overlap" in str(e.value)
