"""The solve server on the GPU: requests of several shapes arrive faster than
they are served, overlap on the device, and each result is the one the same
request gives when solved alone (bit for bit: same plan shape, same kernels)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
import workloads as W
from paper_1402_6081_gb300 import build as lgf_build
from paper_1402_6081_gb300.serve import GpuServer, Request, summarize

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    lgfm.library()


@pytest.mark.parametrize("prec", [lgfm.LGF_FP32, lgfm.LGF_FP64])
def test_each_result_same_alone_and_in_the_mix(prec):
    shapes = [(8, 2), (8, 4), (16, 2), (16, 3)]
    problems = {k: W.request_problem(k[0], k[1], seed=i) for i, k in enumerate(shapes)}
    rng = np.random.default_rng(5)
    n = 48
    t = np.cumsum(rng.exponential(1.0 / 5000.0, size=n))
    reqs = [Request(i, float(t[i]), shapes[int(rng.integers(len(shapes)))], 0) for i in range(n)]
    dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
    # every request its own seeded source on its shape's blocks
    src = {r.rid: torch.from_numpy(np.random.default_rng(100 + r.rid).uniform(
        0.0, 1.0, size=problems[r.key].f.shape)).to(dt).pin_memory() for r in reqs}
    srv = GpuServer(prec, problems, budget_bytes=8e9, n_streams=8, source=lambda r: src[r.rid],
                    keep_results=True)
    srv.warm(shapes)
    done, rejected = srv.run(reqs)
    srv.close()
    assert not rejected and len(done) == n
    starts = sorted((d.start, d.finish) for d in done)
    overlapped = sum(1 for a, b in zip(starts, starts[1:]) if b[0] < a[1])
    assert overlapped > 0                                  # requests ran concurrently
    summarize(done, lambda rid: 1)
    for r in reqs:
        p = problems[r.key]
        s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, prec)
        u = s(src[r.rid].cuda())
        torch.cuda.synchronize()
        alone = u.cpu().numpy()
        s.close()
        assert np.array_equal(srv.results[r.rid], alone), r.rid


@pytest.mark.parametrize("prec", [lgfm.LGF_FP32, lgfm.LGF_FP64])
def test_folded_requests_same_as_alone(prec):
    # requests of two small shapes all pending at once: the server folds up to
    # eight of a shape into one multi-problem plan; each result keeps the bits
    # of the same request solved alone
    shapes = [(8, 2), (8, 3)]
    problems = {k: W.request_problem(k[0], k[1], seed=i) for i, k in enumerate(shapes)}
    reqs = [Request(i, 0.0, shapes[i % 2], 0) for i in range(32)]
    dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
    src = {r.rid: torch.from_numpy(np.random.default_rng(300 + r.rid).uniform(
        -1.0, 1.0, size=problems[r.key].f.shape)).to(dt).pin_memory() for r in reqs}
    srv = GpuServer(prec, problems, budget_bytes=8e9, n_streams=4, source=lambda r: src[r.rid % 100],
                    keep_results=True)
    srv.warm(shapes)
    assert srv.fold(shapes[0]) == 8
    done, rejected = srv.run(reqs)
    # a second round finds the folded plans made during the first
    done2, _ = srv.run([Request(100 + r.rid, 0.0, r.key, 0) for r in reqs])
    srv.close()
    assert not rejected and len(done) == 32 and len(done2) == 32
    assert srv.folded >= 16
    for r in reqs:
        p = problems[r.key]
        s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, prec)
        alone = s(src[r.rid].cuda()).cpu().numpy()
        torch.cuda.synchronize()
        s.close()
        assert np.array_equal(srv.results[r.rid], alone), r.rid
        assert np.array_equal(srv.results[100 + r.rid], alone), r.rid


def test_budget_too_small_rejects():
    problems = {(16, 4): W.request_problem(16, 4, seed=0)}
    srv = GpuServer(lgfm.LGF_FP32, problems, budget_bytes=1e6, n_streams=2)
    done, rejected = srv.run([Request(0, 0.0, (16, 4), 0)])
    srv.close()
    assert rejected == [0] and not done


def test_served_request_against_oracle():
    # one small request of the stream's kind, through the server, against the
    # oracle FMM (FP32 within 1e-5: non-negative source, kappa = 1)
    from oracle import fmm
    key = (8, 4)
    problems = {key: W.request_problem(8, 4, seed=9)}
    srv = GpuServer(lgfm.LGF_FP32, problems, budget_bytes=4e9, n_streams=2, keep_results=True)
    done, rejected = srv.run([Request(0, 0.0, key, problems[key].n_points)])
    srv.close()
    assert not rejected and len(done) == 1
    p = problems[key]
    ref = fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order)
    assert fmm.rel_linf(srv.results[0].astype(np.float64), ref) <= 1e-5
