"""The two forms of the level-0 transforms (one CTA per block, the default;
persistent CTAs moving whole cubes by bulk copies, each line transform split
into output classes) compute the same DFTs with different FP32 rounding:
solves agree to a few FP32 ulps of the largest value, each form matches the
oracle, and each form alone is deterministic (a block's arithmetic does not
depend on which CTA takes it)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
import workloads as W
from oracle import fmm
from paper_1402_6081_gb300 import build as lgf_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    lgfm.library()


# two FP32 roundings of the same transforms: ~log2(32) ulps per pass, three
# passes each way, carried linearly through the products
FORM_TOL = 5e-6


def _close(a, b):
    return float((a - b).abs().max()) <= FORM_TOL * float(a.abs().max())


def _solve(p, f, **kw):
    s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP32, **kw)
    u = s(f).clone()
    u2 = s(f).clone()   # again: the block counters start from zero each launch
    u3 = s(f).clone()
    torch.cuda.synchronize()
    stats = s.stats()
    s.close()
    assert torch.equal(u, u2) and torch.equal(u, u3)
    return u, stats


@pytest.mark.parametrize("free", [0, -1, 24])
def test_forms_identical_torus_128(free):
    p = W.config(1)
    f = torch.from_numpy(p.f).float().cuda()
    a, sa = _solve(p, f, free_sms=free, fft_kernel=1)
    b, sb = _solve(p, f, free_sms=free, fft_kernel=2)
    assert sa["fft_kernel"] == 1 and sb["fft_kernel"] == 2
    assert _close(a, b)
    c, sc = _solve(p, f, free_sms=free)
    assert sc["fft_kernel"] == 1 and torch.equal(a, c)


@pytest.mark.parametrize("n_b,nb", [(8, 4), (8, 6), (16, 3)])
def test_forms_identical_small(n_b, nb):
    p = W.torus_box(seed=9, nb=nb, n_b=n_b, radius=0.3 * nb * n_b, sigma=2.0)
    f = torch.from_numpy(p.f).float().cuda()
    a, _ = _solve(p, f, fft_kernel=1)
    b, _ = _solve(p, f, fft_kernel=2)
    assert _close(a, b)
    ref = fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order)
    assert fmm.rel_linf(b.double().cpu().numpy(), ref) <= 1e-5


def test_single_block_and_misaligned_buffers():
    # one block (fewer blocks than CTAs); then f and u 4 bytes off a 16-byte
    # boundary: the forward transform falls back to the per-block form, the
    # inverse one writes with scalar stores
    p = W.torus_box(seed=4, nb=1, n_b=16, radius=5.0, sigma=2.0, n_levels=1)
    f = torch.from_numpy(p.f).float().cuda()
    a, _ = _solve(p, f, fft_kernel=1)
    b, _ = _solve(p, f, fft_kernel=2)
    assert _close(a, b)
    q = W.config(1)
    fq = torch.from_numpy(q.f).float().cuda()
    ref, _ = _solve(q, fq, fft_kernel=2)   # aligned: both persistent transforms
    n = fq.numel()
    fbuf = torch.zeros(n + 1, device="cuda")
    fbuf[1:] = fq.reshape(-1)
    fv = fbuf[1:].view(fq.shape)
    ubuf = torch.zeros(n + 1, device="cuda")
    uv = ubuf[1:].view(fq.shape)
    s = lgfm.Solver(q.blocks, q.n_b, q.n_levels, q.order, lgfm.LGF_FP32, fft_kernel=2)
    s(fv, uv)
    torch.cuda.synchronize()
    s.close()
    assert _close(uv, ref)


def test_form_options():
    p = W.config(1)
    s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP64)
    assert s.stats()["fft_kernel"] == 1
    s.close()
    with pytest.raises(lgfm.LgfError) as e:
        lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP64, fft_kernel=2)
    assert e.value.status == 1 and "fft_kernel" in str(e.value)
    with pytest.raises(lgfm.LgfError):
        lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP32, fft_kernel=3)


def test_batch_graph_replays():
    # the persistent transforms inside a captured graph: the kernels reset
    # their counters themselves, so every replay gives the same bits, close to
    # the per-block form's
    probs = [W.torus_box(seed=s, nb=nb, n_b=16, radius=0.3 * nb * 16, sigma=3.0)
             for s, nb in ((1, 4), (2, 6), (3, 5))]
    specs = [(p.blocks, p.n_b, p.n_levels, p.order) for p in probs]
    outs = {}
    for form in (1, 2):
        bs = lgfm.BatchSolver(specs, precision=lgfm.LGF_FP32, use_graph=1, options={16: {"fft_kernel": form}})
        bs.set_sources([torch.from_numpy(p.f).float() for p in probs])
        runs = []
        for _ in range(3):
            bs()
            torch.cuda.synchronize()
            runs.append([bs.u_view(i).clone() for i in range(len(probs))])
        bs.close()
        for r in runs[1:]:
            assert all(torch.equal(x, y) for x, y in zip(r, runs[0]))
        outs[form] = runs[0]
    assert all(_close(x, y) for x, y in zip(outs[1], outs[2]))
