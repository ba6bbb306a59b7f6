"""The autotuner (paper_1402_6081_gb300/autotune.py): a coordinate search over
the scheduling options on the GPU.  The options it returns build a plan whose
result is the method's (against the oracle, within the FP32 tolerance), its
cache is written and read back, and its search space is the documented one."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1402_6081_gb300 as lgfm
import workloads as W
from oracle import fmm
from paper_1402_6081_gb300 import autotune
from paper_1402_6081_gb300 import build as lgf_build


@pytest.mark.gpu
def test_tuned_options_solve_the_same_problem(tmp_path, monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lgf_build.build()
    monkeypatch.setenv("LGF_TUNE_CACHE", str(tmp_path / "tune.json"))
    p = W.torus_box(seed=3, nb=6, n_b=8, radius=14.0, sigma=3.0, n_levels=3)
    opts = autotune.tune(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP32, reps=2)
    cache = json.loads((tmp_path / "tune.json").read_text())
    (entry,) = cache.values()
    assert entry["options"] == opts and len(entry["all"]) >= 8
    assert entry["ms"] <= min(t["ms"] for t in entry["all"]) / 0.98   # kept unless beaten by 2%
    assert autotune.tune(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP32) == opts   # from the cache
    s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP32, **opts)
    u = s(torch.from_numpy(p.f).float().cuda())
    lgfm.lgf_plan_sync(s.plan)
    ref = fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order)
    assert fmm.rel_linf(u.double().cpu().numpy(), ref) <= 1e-5
    s.close()
