"""Autotuner for the solver's scheduling options.

For one problem shape it times candidate option sets on the current GPU (CUDA
events, a few warm solves each) and keeps the fastest.  The choices only
change scheduling, never the method: the interval FFT length S_I (any S_I >=
2 n_I - 1 is exact), the interaction-kernel form, the SMs left to the levels
>= 2 chain, the level-0 FFT form (the FFT tile: one block per CTA, or a
persistent CTA per SM streaming blocks), the kernel tables (half tables or
reflection-reduced ones) and the interaction-list chunk (sibling groups per
CTA of the one-CTA-per-chunk products).  The search is coordinate-wise: from
the library's defaults, each dimension in turn is set to each of its values
with the others held at the best so far.  Results are cached per (GPU name,
n_b, precision, levels, block-count bucket) in a JSON file ($LGF_TUNE_CACHE,
default ~/.cache/paper_1402_6081_gb300/autotune.json).
"""
from __future__ import annotations

import json
import math
import os
import pathlib
import threading

import numpy as np

from . import LGF_FP32

_LOCK = threading.Lock()

# Values per dimension (0 = the library's choice).  interval_kernel: 1 = one
# CTA per frequency chunk, 3 = paired groups; free_sms: SMs left to levels >= 2
# beside the persistent products (-1: none); fft_kernel 2: persistent level-0
# transforms (FP32, n_b 8 or 16); mac_groups_per_cta: the interaction-list chunk
DIMENSIONS = {
    "fft_size_interval": {4: [0], 8: [0, 17], 16: [0, 34, 36]},
    "interval_kernel": [0, 1, 3],
    "free_sms": [0, -1, 8, 16, 32],
    "fft_kernel": [0, 2],
    "symmetric_spectra": [0, 1],
    "mac_groups_per_cta": [0, 8, 32, 128],
}


def candidates(n_b: int, precision: int):
    """The dimensions searched for this block size and precision, in order."""
    dims = []
    for name, vals in DIMENSIONS.items():
        v = vals.get(n_b, [0]) if isinstance(vals, dict) else list(vals)
        if precision != LGF_FP32 and name in ("fft_kernel", "free_sms"):
            v = [0]
        if precision != LGF_FP32 and name == "interval_kernel":
            v = [0, 1]
        if name == "fft_kernel" and n_b not in (8, 16):
            v = [0]
        # block sizes of the run-time-size kernels: the reduced tables and the
        # chunk size of the one-CTA-per-chunk products do not apply, and the
        # product-kernel choice is persistent (0) or not (1)
        if n_b > 16 and name in ("symmetric_spectra", "mac_groups_per_cta"):
            v = [0]
        if n_b > 16 and name == "interval_kernel":
            v = [0, 1]
        if len(v) > 1:
            dims.append((name, v))
    return dims


def cache_path() -> pathlib.Path:
    p = os.environ.get("LGF_TUNE_CACHE")
    if p:
        return pathlib.Path(p)
    return pathlib.Path.home() / ".cache" / "paper_1402_6081_gb300" / "autotune.json"


def _key(n_b, precision, n_levels, n_blocks) -> str:
    import torch
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    bucket = 1 << max(0, int(math.ceil(math.log2(max(1, n_blocks)))))
    return f"{dev}|nb{n_b}|p{precision}|L{n_levels}|B{bucket}"


def _load() -> dict:
    try:
        return json.loads(cache_path().read_text())
    except Exception:
        return {}


def _store(d: dict) -> None:
    p = cache_path()
    try:
        p.parent.mkdir(parents=True, exist_ok=True)
        tmp = p.with_suffix(f".{os.getpid()}.tmp")
        tmp.write_text(json.dumps(d, indent=1, sort_keys=True))
        os.replace(tmp, p)
    except OSError:
        pass


def _time_plan(plan, n_points, dtype, reps, warmup) -> float:
    import torch

    from . import lgf_solve
    rng = np.random.default_rng(0)
    f = torch.from_numpy(rng.uniform(0.0, 1.0, size=n_points)).to(dtype).cuda()
    u = torch.empty_like(f)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            lgf_solve(plan, f, u, stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            lgf_solve(plan, f, u, stream)
        b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def time_options(blocks_list, n_b, levels_list, order, precision, opts, reps=5, warmup=2) -> float:
    """Mean milliseconds per solve of a (multi-problem) plan with these options."""
    import torch

    from . import LGF_FP64, lgf_destroy, lgf_plan_create_multi
    plan = lgf_plan_create_multi(blocks_list, n_b, levels_list, order, precision, **opts)
    try:
        npts = sum(int(np.asarray(b).reshape(-1, 3).shape[0]) for b in blocks_list) * n_b ** 3
        dt = torch.float64 if precision == LGF_FP64 else torch.float32
        return _time_plan(plan, npts, dt, reps, warmup)
    finally:
        lgf_destroy(plan)


def tune_multi(blocks_list, n_b: int, levels_list, order: int, precision: int = LGF_FP32,
               use_cache: bool = True, reps: int = 10) -> dict:
    """Fastest option set for a set of problems solved as one plan (the cache
    key is the block size, precision, deepest level count and total blocks,
    rounded up to a power of two)."""
    n_blocks = sum(int(np.asarray(b).reshape(-1, 3).shape[0]) for b in blocks_list)
    key = _key(n_b, precision, max(levels_list), n_blocks) + f"|P{len(blocks_list)}"
    if use_cache:
        with _LOCK:
            hit = _load().get(key)
        if hit is not None:
            return dict(hit["options"])
    timings = []

    def measure(opts):
        try:
            ms = time_options(blocks_list, n_b, levels_list, order, precision, opts, reps=reps)
        except Exception:
            return None
        timings.append((ms, dict(opts)))
        return ms

    best = {}
    best_ms = measure(best)
    if best_ms is None:
        return {}
    for name, values in candidates(n_b, precision):
        for v in values:
            if v == best.get(name, 0):
                continue
            trial = dict(best)
            if v == 0:
                trial.pop(name, None)
            else:
                trial[name] = v
            ms = measure(trial)
            # a change must win by more than the timing noise (2%)
            if ms is not None and ms < 0.98 * best_ms:
                best_ms, best = ms, trial
    if use_cache:
        with _LOCK:
            d = _load()
            d[key] = {"options": best, "ms": best_ms,
                      "all": [{"options": c, "ms": t} for t, c in timings]}
            _store(d)
    return dict(best)


def tune(blocks, n_b: int, n_levels: int, order: int, precision: int = LGF_FP32,
         use_cache: bool = True, reps: int = 10) -> dict:
    """Fastest option set for one problem (from the cache when present)."""
    return tune_multi([np.asarray(blocks).reshape(-1, 3)], n_b, [n_levels], order, precision, use_cache, reps)
