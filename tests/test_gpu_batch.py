"""Batched solves: a multi-problem plan and a batch (stream pool, CUDA graph)
give every problem the result its own plan gives alone.

No list links two problems of a multi-problem plan, and every kernel computes
an item (a block, an interval, a sibling group) from that item's data in a fixed
order.  With the same kernel forms and schedule on both sides the results are
compared bit for bit with the single-problem solves (which the parity tests
tie to the oracle).  With default options the library may pick different
forms for the larger plan (the persistent products need enough sibling
groups; the schedule follows the plan's work split), which changes only the
FP32 rounding (summation order over up to 216 sources per point): those
results agree within the FP32 tolerance, 1e-5 of max|u| (measured 1.7e-6).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
import workloads as W
from paper_1402_6081_gb300 import build as lgf_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    lgfm.library()


def _dtype(prec):
    return torch.float64 if prec == lgfm.LGF_FP64 else torch.float32


# the same forms on both sides: persistent packed products at every level,
# the split schedule
SAME = {"interval_kernel": 5, "free_sms": -1}


def solo(p, prec, **opts):
    s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, prec, **opts)
    u = s(torch.from_numpy(np.ascontiguousarray(p.f)).to(_dtype(prec)).cuda())
    torch.cuda.synchronize()
    out = u.cpu().numpy()
    s.close()
    return out


def _hand_problems(n_b, order=8):
    """Small problems that exercise the per-problem level logic: one block
    (one level, no interval products), two distant blocks (products only at
    level 2), a sparse set with negative indices, a fully occupied box."""
    rng = np.random.default_rng(11)
    out = []
    specs = [
        (np.array([[0, 0, 0]]), 1),
        (np.array([[0, 0, 0], [5, 0, 0]]), 3),
        (np.array([[-3, -1, 0], [-2, -1, 0], [0, 2, 1], [1, 1, -2], [2, -3, 1], [-1, 0, 0]]), 4),
        (W.full_box_blocks(4), 2),
    ]
    for blocks, L in specs:
        f = rng.uniform(-1.0, 1.0, size=(len(blocks), n_b, n_b, n_b))
        out.append(W.Problem(blocks, f, n_b, L, order, f"hand_{len(blocks)}_{L}"))
    return out


def _mix(n_b):
    bp = [p for p in W.batch_problems(24, seed=3) if p.n_b == n_b][:4]
    return _hand_problems(n_b) + bp


@pytest.mark.parametrize("prec", [lgfm.LGF_FP32, lgfm.LGF_FP64])
@pytest.mark.parametrize("n_b", [8, 16, 20])     # 20: the run-time-size kernels
@pytest.mark.parametrize("separate", [0, 1])
@pytest.mark.parametrize("same", [True, False])
def test_multi_plan_matches_each_problem_alone(prec, n_b, separate, same):
    probs = _mix(n_b)
    opts = dict(SAME) if same and prec == lgfm.LGF_FP32 else {}
    plan = lgfm.lgf_plan_create_multi([p.blocks for p in probs], n_b, [p.n_levels for p in probs], 8, prec,
                                      separate_level1=separate, **opts)
    st = lgfm.lgf_plan_get_stats(plan)
    assert st["n_problems"] == len(probs)
    assert st["n_blocks"] == sum(len(p.blocks) for p in probs)
    f = torch.from_numpy(np.concatenate([p.f.reshape(-1) for p in probs])).to(_dtype(prec)).cuda()
    u = torch.empty_like(f)
    lgfm.lgf_solve(plan, f, u)
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    lgfm.lgf_destroy(plan)
    at = 0
    for p in probs:
        ref = solo(p, prec, separate_level1=separate, **opts)
        n = ref.size
        mine = got[at:at + n].reshape(ref.shape)
        if same or prec == lgfm.LGF_FP64:
            assert np.array_equal(mine, ref), p.name
        else:
            assert np.abs(mine - ref).max() <= 1e-5 * np.abs(ref).max(), p.name
        at += n


def test_multi_plan_stats_are_sums():
    probs = _mix(8)
    plan = lgfm.lgf_plan_create_multi([p.blocks for p in probs], 8, [p.n_levels for p in probs], 8)
    st = lgfm.lgf_plan_get_stats(plan)
    lgfm.lgf_destroy(plan)
    pairs = np.zeros(len(st["pairs"]), dtype=np.int64)
    for p in probs:
        pl = lgfm.lgf_plan_create(p.blocks, 8, p.n_levels, 8)
        s1 = lgfm.lgf_plan_get_stats(pl)
        lgfm.lgf_destroy(pl)
        pairs[: len(s1["pairs"])] += np.array(s1["pairs"], dtype=np.int64)
    assert list(pairs) == st["pairs"]
    assert st["n_levels"] == max(p.n_levels for p in probs)


def test_multi_plan_errors():
    b = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.int32)
    # the same block indices in two problems are two separate domains
    plan = lgfm.lgf_plan_create_multi([b, b], 8, [1, 1], 8)
    lgfm.lgf_destroy(plan)
    with pytest.raises(lgfm.LgfError, match="problem 1"):
        lgfm.lgf_plan_create_multi([b, np.array([[0, 0, 0], [9, 0, 0]])], 8, [1, 1], 8)
    with pytest.raises(lgfm.LgfError, match="problem 0"):
        lgfm.lgf_plan_create_multi([np.array([[0, 0, 0], [0, 0, 0]]), b], 8, [1, 1], 8)
    with pytest.raises(ValueError):
        lgfm.lgf_plan_create_multi([b, b], 8, [1], 8)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_solver_matches_each_problem_alone(use_graph):
    probs = W.batch_problems(12, seed=3) + _hand_problems(8)
    bs = lgfm.BatchSolver([(p.blocks, p.n_b, p.n_levels, p.order) for p in probs], lgfm.LGF_FP32,
                          use_graph=use_graph, options={8: SAME, 16: SAME})
    bs.set_sources([torch.from_numpy(p.f).float() for p in probs])
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        bs(st)
        bs(st)     # a relaunch recomputes the same values
    st.synchronize()
    outs = [bs.u_view(i).cpu().numpy() for i in range(len(probs))]
    bs.close()
    for p, got in zip(probs, outs):
        assert np.array_equal(got, solo(p, lgfm.LGF_FP32, **SAME)), p.name


def test_batch_of_separate_plans():
    probs = _hand_problems(8)[:3] + [p for p in W.batch_problems(6, seed=3) if p.n_b == 16][:2]
    plans = [lgfm.lgf_plan_create(p.blocks, p.n_b, p.n_levels, p.order) for p in probs]
    fs = [torch.from_numpy(p.f).float().cuda() for p in probs]
    us = [torch.empty_like(f) for f in fs]
    for g in (0, 1):
        b = lgfm.lgf_batch_create(plans, fs, us, g)
        lgfm.lgf_batch_launch(b)
        torch.cuda.synchronize()
        for p, u in zip(probs, us):
            assert np.array_equal(u.cpu().numpy(), solo(p, lgfm.LGF_FP32)), (g, p.name)
            u.fill_(float("nan"))
        lgfm.lgf_batch_destroy(b)
    with pytest.raises(lgfm.LgfError):
        lgfm.lgf_batch_create([plans[0], plans[0]], fs[:2], us[:2], 0)
    lgfm.lgf_plan_set_timing(plans[0], 16)
    with pytest.raises(lgfm.LgfError, match="timing"):
        lgfm.lgf_batch_create(plans[:1], fs[:1], us[:1], 1)
    for pl in plans:
        lgfm.lgf_destroy(pl)


def _kappa(p, ref):
    from oracle import fmm
    if np.all(p.f >= 0):
        return 1.0
    ua = fmm.fmm_solve(p.blocks, np.abs(p.f), p.n_b, p.n_levels, p.order)
    return max(1.0, float(np.abs(ua).max() / np.abs(ref).max()))


@pytest.mark.parametrize("n_b", [8, 16])
def test_batch_problems_against_oracle(n_b):
    # the smallest batch problems of each block size, solved in one batch,
    # against the oracle FMM (FP32 within 1e-5, FP64 within 1e-12)
    from oracle import fmm
    probs = sorted([p for p in W.batch_problems(64, seed=3) if p.n_b == n_b], key=lambda p: p.n_points)[:2]
    for prec, tol in ((lgfm.LGF_FP32, 1e-5), (lgfm.LGF_FP64, 1e-12)):
        bs = lgfm.BatchSolver([(p.blocks, p.n_b, p.n_levels, p.order) for p in probs], prec, use_graph=1)
        bs.set_sources([torch.from_numpy(p.f).to(_dtype(prec)) for p in probs])
        bs()
        torch.cuda.synchronize()
        for i, p in enumerate(probs):
            ref = fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order)
            err = fmm.rel_linf(bs.u_view(i).double().cpu().numpy(), ref)
            assert err <= tol * _kappa(p, ref), (p.name, prec, err)
        bs.close()
