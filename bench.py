"""Throughput of the GB300 LGF-FMM solve, one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one whole solve u = G * f (every step of Sec. 3.1: forward FFTs,
regularization, near-field and interaction-list products, inverse FFTs,
interpolation) on the 128^3 torus workload (8^3 blocks of 16^3 points, 3
levels, interpolation order 8) in FP32, inputs resident in HBM.  L2 is flushed
(a 256 MiB write) before every timed step; steps are timed with CUDA events on
the solve stream.  Under torchrun each rank solves its own replica (weak
scaling, no data-path collective); rank 0 prints the max-over-ranks timing.

--impl reference times the CPU oracle (NumPy FP64, the paper's method step by
step) on the host cores, each step a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "LGF-FMM points/s at <=1e-5 rel err, FP32 vs FP64 on 1 GB300; serve p50/p99 ms"
WORKLOAD = "torus_box_128"
FP32_FMA_LANES_PER_SM = 128
N_SM = 152
SM_MAX_MHZ = 2070.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def measure_fma_peaks(lgfm, dev: int):
    """FP32 and FP64 fused multiply-add throughput of this GPU, measured by the
    library (lgf_measure_fma_peak: every SM, independent FMA chains, best of 5
    launches), with the SM clock sampled meanwhile.  TFLOP/s."""
    clk = ClockSampler(dev)
    clk.start()
    r = {name: lgfm.lgf_measure_fma_peak(kind, 5) for name, kind in (("fp64", 0), ("fp32", 1), ("fp32x2", 2))}
    c = clk.stop()
    out = {k: {"tflops": v[0] / 1e12, "ms": v[1]} for k, v in r.items()}
    out["fp32_best_tflops"] = max(out["fp32"]["tflops"], out["fp32x2"]["tflops"])
    out["clocks"] = c
    out["how"] = ("lgf_measure_fma_peak: every SM full of 256-thread CTAs, 16 independent fma.rn chains per "
                  "thread (f64 / f32 / f32x2), CUDA events, best of 5; 2 flop per FMA lane")
    return out


def profiled_traffic(name: str):
    """DRAM bytes per launch of the dominant kernel from its committed ncu
    summary (profiles/<kernel>_torus_box_128_fp32.md), or None when there is
    none or the kernel sources changed after that capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{name}_{WORKLOAD}_fp32.md")
    csrc = os.path.join(ROOT, "paper_1402_6081_gb300", "csrc")
    try:
        text = open(path).read()
        h = hashlib.sha256(open(os.path.join(csrc, "kernels_impl.cuh"), "rb").read()
                           + open(os.path.join(csrc, "fft_device.cuh"), "rb").read()).hexdigest()[:16]
        kv = dict(line.split(": ", 1) for line in text.splitlines() if ": " in line and "_" in line.split(": ")[0]
                  and " " not in line.split(": ")[0])
        if kv.get("kernel_source_sha256_16") != h:
            return None
        return int(kv["traffic_bytes_per_launch"])
    except Exception:
        return None


def interaction_pairs(blocks: np.ndarray, n_levels: int):
    """Source-target interval pairs per level: level 0 near pairs, level l >= 1
    interaction-list pairs (Sec. 3.1 lists), for the roofline's work count."""
    out = {}
    b = np.asarray(blocks, dtype=np.int64)
    for l in range(0, n_levels):
        iv = np.unique(b >> max(l - 1, 0), axis=0)
        keys = set(map(tuple, iv))
        n = 0
        for p in map(tuple, iv):
            if l == 0:
                n += sum((p[0] + dx, p[1] + dy, p[2] + dz) in keys
                         for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1))
                continue
            pp = (p[0] >> 1, p[1] >> 1, p[2] >> 1)
            for ex in (-1, 0, 1):
                for ey in (-1, 0, 1):
                    for ez in (-1, 0, 1):
                        for c in range(8):
                            q = (2 * (pp[0] + ex) + (c & 1), 2 * (pp[1] + ey) + ((c >> 1) & 1),
                                 2 * (pp[2] + ez) + (c >> 2))
                            if q in keys and max(abs(q[0] - p[0]), abs(q[1] - p[1]), abs(q[2] - p[2])) > 1:
                                n += 1
        out[l] = n
    return out


def cpu_oracle_rate(p, spectra=None):
    """Oracle FMM on the host cores: (points/s, seconds, cores used, solution)."""
    from oracle import fmm
    sp = spectra if spectra is not None else fmm.Spectra(p.n_b)
    if spectra is None:      # kernel spectra are plan-time work: precompute outside the timing
        fmm.fmm_solve(p.blocks[:1], p.f[:1], p.n_b, 1, p.order, spectra=sp)
    t0, c0 = time.perf_counter(), time.process_time()
    u = fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order, spectra=sp)
    dt, dc = time.perf_counter() - t0, time.process_time() - c0
    return p.n_points / dt, dt, max(1, round(dc / dt)), u


def direct_sum_rate():
    """The exact O(N^2) lattice sum (the oracle's C/OpenMP direct sum, all host
    threads) on the 32^3 two-level workload: one warm-up, median of three."""
    from oracle import direct
    p = W.config(0)
    direct.direct_sum(p.blocks, p.n_b, p.f)
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        direct.direct_sum(p.blocks, p.n_b, p.f)
        ts.append(time.perf_counter() - t0)
    dt = statistics.median(ts)
    n = p.n_points
    return {"value": n / dt, "unit": "points/s", "pairs_per_s": n * n / dt, "seconds": dt,
            "threads": os.cpu_count(), "kind": "oracle direct sum (exact)",
            "sample": f"gaussian_box_32: {n} points, {n * n:.3g} pair terms, median of 3 after 1 warm-up"}


def reference_sample():
    """Bounded sample of the workload for the CPU arm: the 64^3 window (4^3
    blocks of 16^3, 2 levels) of the 128^3 torus at the same order."""
    full = W.config(1)
    sel = np.all(full.blocks < 4, axis=1)
    return W.Problem(full.blocks[sel].copy(), full.f[sel].copy(), 16, 2, full.order, "torus_box_128_window64")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import fmm
    p = reference_sample()
    sp = fmm.Spectra(p.n_b)
    for _ in range(args.warmup):
        fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order, spectra=sp)
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(args.steps):
        fmm.fmm_solve(p.blocks, p.f, p.n_b, p.n_levels, p.order, spectra=sp)
    dt, dc = time.perf_counter() - t0, time.process_time() - c0
    value = p.n_points * args.steps / dt
    cores = max(1, round(dc / dt))
    sample = "oracle FMM (NumPy FP64) on the 64^3 window (4^3 blocks of 16^3, 2 levels, order 8) of the 128^3 torus"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "window64", "points": p.n_points},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "nproc": os.cpu_count(), "cpu_model": cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def replica_rate(total_ms: float, points: int, steps: int, world: int, dist=None, device: str = "cpu"):
    """Weak scaling over replicas: every rank solves its own copy of the
    workload; the job's time is the slowest rank's (max over ranks), and the
    job's rate counts the points of all ranks.  Returns (max ms, points/s)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * points * steps / (total_ms * 1e-3)


def batch_run(torch, lgfm, steps: int, warmup: int, flush):
    """64 independent uneven solves (log-uniform 32^3..192^3 boxes, 8^3 or 16^3
    blocks, Gaussian-blob sources) as one CUDA-graph batch: one multi-problem
    plan per block size (one launch per phase for all its problems), options
    from the autotuner.  Returns the JSON object of the batched workload."""
    from paper_1402_6081_gb300 import autotune
    probs = W.batch_problems(64, seed=3)
    specs = [(p.blocks, p.n_b, p.n_levels, p.order) for p in probs]
    opts = {}
    for n_b in sorted({p.n_b for p in probs}):
        ps = [p for p in probs if p.n_b == n_b]
        opts[n_b] = autotune.tune_multi([p.blocks for p in ps], n_b, [p.n_levels for p in ps], ps[0].order,
                                        lgfm.LGF_FP32)
    stream = torch.cuda.Stream()
    res = {}
    for prec in (lgfm.LGF_FP32, lgfm.LGF_FP64):
        dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
        bs = lgfm.BatchSolver(specs, prec, use_graph=1, options=opts if prec == lgfm.LGF_FP32 else None)
        bs.set_sources([torch.from_numpy(p.f).to(dt) for p in probs])
        launches = sum(lgfm.lgf_plan_timings(pl)[1] for pl in bs.plans)
        k = steps if prec == lgfm.LGF_FP32 else max(3, steps // 5)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                bs(stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for a, b in ev:
                flush.fill_(1.0)
                a.record(stream)
                bs(stream)
                b.record(stream)
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        npts = bs.n_points()
        r = {"value": npts / (ms * 1e-3), "unit": "points/s", "ms_per_step": ms, "steps": k,
             "gpu_launches_per_step": int(launches), "plans": len(bs.plans)}
        if prec == lgfm.LGF_FP32:
            # end to end: pinned host sources in, results out, every step
            fh = [torch.cat([bs.f_view(i).reshape(-1).cpu() for i in range(len(probs)) if bs.where[i][0] == c])
                  .pin_memory() for c in range(len(bs.plans))]
            uh = [torch.empty_like(x).pin_memory() for x in fh]
            ke = max(3, k // 4)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(ke):
                with torch.cuda.stream(stream):
                    for c in range(len(bs.plans)):
                        bs.f[c].copy_(fh[c], non_blocking=True)
                    bs(stream)
                    for c in range(len(bs.plans)):
                        uh[c].copy_(bs.u[c], non_blocking=True)
                stream.synchronize()
            e2e = (time.perf_counter() - t0) / ke
            nbytes = int(sum(x.numel() for x in fh) * 4)
            r["e2e"] = {"value": npts / e2e, "unit": "points/s", "h2d_bytes_per_step": nbytes,
                        "d2h_bytes_per_step": nbytes, "steps": ke}
            r["options"] = {str(kk): v for kk, v in opts.items()}
            u32 = [bs.u_view(i).double().cpu().numpy() for i in range(len(probs))]
        else:
            err = 0.0
            for i in range(len(probs)):
                u64 = bs.u_view(i).cpu().numpy()
                err = max(err, float(np.abs(u32[i] - u64).max() / np.abs(u64).max()))
            r["rel_err_fp32_vs_fp64_max"] = err
        bs.close()
        res["fp32" if prec == lgfm.LGF_FP32 else "fp64"] = r
    out = dict(res["fp32"])
    out["fp64"] = res["fp64"]
    out["config"] = {"workload": "batch64", "problems": len(probs), "points": npts,
                     "l2": "flushed: 256 MiB write before every timed step", "graph": True}
    return out


def irregular_run(torch, lgfm, steps: int, flush):
    """The 512^3 irregular domain (12 tori, 7252 blocks of 16^3, 22% occupancy,
    5 levels, order 8): points/s and the error of each interpolation mode
    against the plain FP64 form on the same GPU (which the parity tests tie to
    the FP64 oracle at 1e-12 on the other configs)."""
    p = W.tori_irregular(2)
    stream = torch.cuda.Stream()
    # "fp32": the library's default (compensated Reg/Interp sums at this depth);
    # "fp32_plain": plain FP32 sums
    modes = {"fp32": lgfm.LGF_INTERP_NATIVE, "fp32_plain": lgfm.LGF_INTERP_PLAIN,
             "bf16": lgfm.LGF_INTERP_BF16, "fp16": lgfm.LGF_INTERP_FP16, "bf16x3": lgfm.LGF_INTERP_BF16X3}

    def run(prec, mode, k):
        dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
        s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, prec, interp_mode=mode)
        f = torch.from_numpy(p.f).to(dt).cuda()
        u = torch.empty_like(f)
        with torch.cuda.stream(stream):
            for _ in range(3):
                s(f, u, stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for a, b in ev:
                flush.fill_(1.0)
                a.record(stream)
                s(f, u, stream)
                b.record(stream)
        lgfm.lgf_plan_sync(s.plan)
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        out = u.double().cpu().numpy()
        s.close()
        return ms, out

    ms64, u64 = run(lgfm.LGF_FP64, lgfm.LGF_INTERP_NATIVE, 3)
    scale = float(np.abs(u64).max())
    res = {"fp64": {"value": p.n_points / (ms64 * 1e-3), "ms_per_step": ms64}}
    for name, mode in modes.items():
        ms, u = run(lgfm.LGF_FP32, mode, steps)
        res[name] = {"value": p.n_points / (ms * 1e-3), "ms_per_step": ms,
                     "rel_err_vs_fp64": float(np.abs(u - u64).max()) / scale}
    out = dict(res["fp32"])
    out.update({"unit": "points/s", "modes": res,
                "config": {"workload": "tori_irregular_512", "points": p.n_points, "blocks": len(p.blocks),
                           "levels": p.n_levels, "interp_order": p.order,
                           "l2": "flushed: 256 MiB write before every timed step"}})
    return out


def fft_conv_run(torch, lgfm, steps: int, flush, peak_tf: float):
    """The FFT-convolution special case (Sec. 4, "FFT Conv."): every 16^3 block
    an isolated one-block domain, u_b = G * f_b by one padded 32^3 R2C, one
    spectral product and one truncated C2R, the 512 blocks of the 128^3 torus
    per step, FP32.  The timed form is lgf_conv_blocks: all three steps in one
    kernel with the spectra in shared memory; the three-launch form
    (lgf_solve_blocks_noalloc, spectra through device memory) is timed beside
    it.  Work is counted as 5 N log2 N flop per real 32^3 transform (both
    directions) plus the product; the fraction is of the FP32 FMA peak."""
    p = W.config(1)
    n_b = p.n_b
    per_call = lgfm.lgf_noalloc_max_blocks(n_b, lgfm.LGF_FP32)
    f = torch.from_numpy(p.f).float().cuda()
    u = torch.empty_like(f)
    nblk = len(p.blocks)
    stream = torch.cuda.Stream()

    def fused():
        lgfm.lgf_conv_blocks(f, u, nblk, n_b, lgfm.LGF_FP32, stream)

    def three_launch():
        for b0 in range(0, nblk, per_call):
            nb = min(per_call, nblk - b0)
            lgfm.lgf_solve_blocks_noalloc(f[b0:b0 + nb], u[b0:b0 + nb], nb, n_b, lgfm.LGF_FP32, stream)

    def timed(one_pass):
        with torch.cuda.stream(stream):
            for _ in range(4):
                one_pass()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for a, b in ev:
                flush.fill_(1.0)
                a.record(stream)
                one_pass()
                b.record(stream)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    ms3 = timed(three_launch)
    ms = timed(fused)
    S = 2 * n_b
    n3 = S ** 3
    flops_block = 2 * 5.0 * n3 * np.log2(n3) / 2 + 8.0 * (S // 2 + 1) * S * S
    tf = nblk * flops_block / (ms * 1e-3) / 1e12
    return {"value": p.n_points / (ms * 1e-3), "unit": "points/s", "ms_per_step": ms, "steps": steps,
            "launch_calls_per_step": 1,
            "three_launch": {"value": p.n_points / (ms3 * 1e-3), "ms_per_step": ms3,
                             "launch_calls_per_step": -(-nblk // per_call)},
            "roofline": {"bound": "alu", "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s", "frac": tf / peak_tf,
                         "peak_source": "measured FP32 FMA peak (lgf_measure_fma_peak)",
                         "algorithmic": "per block: 5 N log2 N / 2 per real 32^3 transform x 2 + 8 flop per "
                                        "complex product",
                         "hbm_gbs_f_and_u": 8.0 * p.n_points / (ms * 1e-3) / 1e9},
            "config": {"workload": "fft_conv_16cubed_blocks", "blocks": nblk, "points": p.n_points,
                       "l2": "flushed: 256 MiB write before every timed step"}}


def error_sweep_run(torch, lgfm, diameter: int = 128):
    """The paper's error experiment on the GPU (Sec. 4.1): exact manufactured
    solutions on a cube, a sphere and a spherical shell of the same diameter,
    n_max = 10, n_I = n_b + 1 = 11..27; relative L-infinity error of the FP64
    form, its fitted power of n_I (the paper: -10.7 for n_I = 11..28) over the
    whole range and over n_I <= 23 (above that the error reaches the FP64
    rounding floor of these badly conditioned random sources), and the FP32 /
    FP64 rates.  Also the Sec. 2.5 parameter choice for three targets."""
    sizes = (10, 12, 14, 16, 18, 20, 22, 24, 26)
    out = {"config": {"workload": "manufactured_sweep", "diameter": diameter, "n_max": 10,
                      "n_I": [n + 1 for n in sizes]}}
    for shape in ("box", "sphere", "shell"):
        rows = []
        for n_b in sizes:
            blocks = W.shape_blocks(shape, diameter, n_b)
            L = W.levels_for(int(np.ceil(diameter / n_b)))
            m = W.manufactured(blocks, n_b, L, 9, seed=11)
            row = {"n_I": n_b + 1, "points": m.n_points, "levels": L}
            for prec, name in ((lgfm.LGF_FP64, "fp64"), (lgfm.LGF_FP32, "fp32")):
                dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
                s = lgfm.Solver(m.blocks, n_b, L, 9, prec)
                f = torch.from_numpy(m.f).to(dt).cuda()
                u = torch.empty_like(f)
                s(f, u)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(3):
                    s(f, u)
                b.record()
                b.synchronize()
                row[f"{name}_points_per_s"] = 3 * m.n_points / (a.elapsed_time(b) * 1e-3)
                row[f"{name}_rel_err_vs_exact"] = float(np.abs(u.double().cpu().numpy() - m.u_exact).max()
                                                        / np.abs(m.u_exact).max())
                s.close()
            rows.append(row)
        def slope(rs):
            return float(np.polyfit(np.log([r["n_I"] for r in rs]), np.log([r["fp64_rel_err_vs_exact"] for r in rs]),
                                    1)[0])
        out[shape] = {"rows": rows, "fp64_error_slope_vs_n_I": slope(rows),
                      "fp64_error_slope_n_I_11_23": slope([r for r in rows if r["n_I"] <= 23])}
    sel = {}
    for eps, prec, name in ((1e-5, lgfm.LGF_FP32, "fp32_1e-5"), (1e-9, lgfm.LGF_FP64, "fp64_1e-9"),
                            (1.25e-12, lgfm.LGF_FP64, "fp64_1.25e-12")):
        sel[name] = lgfm.lgf_select_interp(eps, prec)
    out["interp_selection"] = sel
    return out


def serve_run(torch, lgfm, n_requests: int = 2200, n_warm: int = 200, precisions=None, server_opts=None):
    """Poisson arrivals (200/s, seed 1) of torus solves with point counts
    log-uniform in 2^12..2^24, admitted under a 120 GB HBM budget, FP32 form
    and plain FP64 form, plus one 512^3 fully occupied solve in the stream and
    alone.  Latency: arrival to the result copied back to host memory."""
    from paper_1402_6081_gb300.serve import GpuServer, Request, summarize
    arr = W.arrival_stream(n_requests, 200.0, seed=1)
    shapes = sorted({(n_b, nb) for _, n_b, nb in arr})
    problems = {k: W.request_problem(k[0], k[1], seed=i) for i, k in enumerate(shapes)}
    big = ("full", 512)
    problems[big] = W.torus_box(seed=7, nb=32, n_b=16, radius=0.3 * 512, sigma=0.06 * 512, noise=0.05, order=8)
    reqs = [Request(i, t, (n_b, nb), problems[(n_b, nb)].n_points) for i, (t, n_b, nb) in enumerate(arr)]
    t_big = arr[(n_warm + n_requests) // 2][0]
    reqs.append(Request(n_requests, t_big, big, problems[big].n_points))
    npts = {r.rid: r.n_points for r in reqs}
    out = {}
    for prec in precisions or (lgfm.LGF_FP32, lgfm.LGF_FP64):
        name = "fp32" if prec == lgfm.LGF_FP32 else "fp64"
        srv = GpuServer(prec, problems, budget_bytes=120e9, n_streams=16, **(server_opts or {}))
        srv.warm(shapes + [big])
        done, rejected = srv.run(reqs)
        timed = [d for d in done if n_warm <= d.rid < n_requests]
        s = summarize(timed, lambda rid: npts[rid])
        bigd = [d for d in done if d.rid == n_requests]
        s["big_512_in_stream_ms"] = 1e3 * bigd[0].latency if bigd else None
        if bigd:
            # the same statistics without the requests whose lifetime overlaps
            # the 512^3 request's (they queue behind its solve on the device)
            b0, b1 = bigd[0].arrival, bigd[0].finish
            clear = [d for d in timed if d.finish < b0 or d.arrival > b1]
            sc = summarize(clear, lambda rid: npts[rid])
            s["without_big_overlap"] = {"requests": sc["requests"], "p50_ms": sc["p50_ms"], "p99_ms": sc["p99_ms"],
                                        "max_ms": sc["max_ms"]}
        s["rejected"] = len(rejected)
        s["folded_requests"] = srv.folded
        s["plans_resident"] = sum(len(v) for v in srv.pools.slots.values())
        s["hbm_used_gb"] = srv.pools.used / 1e9
        # the same 512^3 request alone: the first run right after the stream
        # carries a one-time transient (56.8 ms against 25.2 ms in a probe), so
        # it is kept apart and the median of the three runs after it reported
        alone = [srv.run([Request(0, 0.0, big, problems[big].n_points)])[0][0].latency for _ in range(4)]
        s["big_512_alone_first_ms"] = 1e3 * alone[0]
        s["big_512_alone_ms"] = 1e3 * float(np.median(alone[1:]))
        # saturated: every timed request present at once (capacity); the
        # second pass, once the pools hold the plans this load needs
        sat = [Request(r.rid, 0.0, r.key, r.n_points) for r in reqs if n_warm <= r.rid < n_requests]
        srv.run(sat)
        f0 = srv.folded
        dsat, _ = srv.run(sat)
        ss = summarize(dsat, lambda rid: npts[rid])
        s["saturated"] = {"points_per_s": ss["points_per_s"], "p50_ms": ss["p50_ms"], "p99_ms": ss["p99_ms"],
                          "folded_requests": srv.folded - f0}
        if prec == lgfm.LGF_FP64:
            # the same requests at a quarter of the rate (arrival times x 4: a
            # Poisson stream at 50/s), below the FP64 form's capacity, so its
            # latency is a service time and not a queue
            slow = [Request(r.rid, 4.0 * r.arrival, r.key, r.n_points) for r in reqs[:600]]
            dslow, _ = srv.run(slow)
            ts = summarize([d for d in dslow if d.rid >= 100], lambda rid: npts[rid])
            s["at_50_per_s"] = {"requests": ts["requests"], "p50_ms": ts["p50_ms"], "p99_ms": ts["p99_ms"],
                                "points_per_s": ts["points_per_s"]}
        srv.close()
        out[name] = s
    out["config"] = {"workload": "serve_poisson200", "requests_timed": n_requests - n_warm, "warmup": n_warm,
                     "shapes": len(shapes), "hbm_budget_gb": 120, "streams": 16,
                     "latency": "arrival to result in pinned host memory",
                     "large_requests": "more than 2^25 points: default-priority stream, plan leaves 32 SMs free "
                                       "(others on high-priority streams)"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fft-size", type=int, default=0,
                    help="FFT length per axis at the interval levels (0 = library default)")
    ap.add_argument("--near-kernel", type=int, default=0, help="level-0 product kernel variant (0 = default)")
    ap.add_argument("--interval-kernel", type=int, default=0, help="interval product kernel variant (0 = default)")
    ap.add_argument("--free-sms", type=int, default=0,
                    help="SMs left to levels >= 2 beside the persistent products (-1: split schedule, 0: default)")
    ap.add_argument("--interp-mode", type=int, default=0,
                    help="Reg/Interp arithmetic (lgf_interp_mode: 0 native, 1 BF16, 2 FP16, 3 BF16x3, 4 compensated, "
                         "5 plain)")
    ap.add_argument("--symmetric-spectra", type=int, default=0,
                    help="1: reflection-reduced kernel tables at the one-CTA-per-chunk product levels")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-solve batched workload")
    ap.add_argument("--no-serve", action="store_true", help="skip the Poisson-arrival serving workload")
    ap.add_argument("--no-irregular", action="store_true", help="skip the 512^3 irregular-domain workload")
    ap.add_argument("--no-fft-conv", action="store_true", help="skip the single-block FFT-convolution workload")
    ap.add_argument("--no-sweep", action="store_true", help="skip the n_max = 10 error sweep")
    ap.add_argument("--profile-only", action="store_true",
                    help="only warmup + steps of the FP32 solve (for ncu captures); prints no JSON")
    ap.add_argument("--profile-workload", default=WORKLOAD,
                    choices=[WORKLOAD, "torus_box_144_nb18", "fft_conv_16cubed_blocks", "tori_irregular_512"],
                    help="with --profile-only: the workload solved (torus_box_144_nb18: 8^3 blocks of 18^3, "
                         "3 levels, the run-time-size kernels; fft_conv_16cubed_blocks: the 512 blocks of the "
                         "128^3 torus each alone, lgf_conv_blocks; tori_irregular_512: the 5-level irregular "
                         "domain)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch

    import paper_1402_6081_gb300 as lgfm
    from paper_1402_6081_gb300 import build as lgf_build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        lgf_build.build()
    if dist is not None:
        dist.barrier()
    lgfm.library()
    dev = torch.cuda.current_device()

    p = W.config(1)
    if args.profile_only and args.profile_workload == "torus_box_144_nb18":
        p = W.torus_box(seed=3, nb=8, n_b=18, radius=0.3 * 144, sigma=0.06 * 144, order=8, n_levels=3)
    if args.profile_only and args.profile_workload == "tori_irregular_512":
        p = W.config(2)
    if args.profile_only and args.profile_workload == "fft_conv_16cubed_blocks":
        fc = torch.from_numpy(p.f).float().cuda()
        uc = torch.empty_like(fc)
        for _ in range(args.warmup + args.steps):
            lgfm.lgf_conv_blocks(fc, uc, len(p.blocks), p.n_b, lgfm.LGF_FP32)
        torch.cuda.synchronize()
        return
    npts = p.n_points
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def make(prec):
        dt = torch.float64 if prec == lgfm.LGF_FP64 else torch.float32
        s = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, prec, fft_size_interval=args.fft_size,
                        near_kernel=args.near_kernel, interval_kernel=args.interval_kernel, free_sms=args.free_sms,
                        interp_mode=args.interp_mode if prec == lgfm.LGF_FP32 else 0,
                        symmetric_spectra=args.symmetric_spectra)
        f = torch.from_numpy(p.f).to(dt).cuda()
        u = torch.empty_like(f)
        return s, f, u

    def timed_steps(s, f, u, steps, warmup, timing_capacity=0):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                s(f, u, stream)
        torch.cuda.synchronize()
        if timing_capacity:
            lgfm.lgf_plan_set_timing(s.plan, timing_capacity)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for a, b in ev:
                flush.fill_(1.0)
                a.record(stream)
                s(f, u, stream)
                b.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if dist is not None:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, wall

    s32, f32, u32 = make(lgfm.LGF_FP32)
    with torch.cuda.stream(stream):
        s32(f32, u32, stream)
    torch.cuda.synchronize()
    per_solve_launches = None
    if args.profile_only:
        with torch.cuda.stream(stream):
            for _ in range(args.warmup + args.steps):
                s32(f32, u32, stream)
        torch.cuda.synchronize()
        s32.close()
        return

    clocks = ClockSampler(dev)
    clocks.start()
    # headline: uninstrumented solves
    ms, wall = timed_steps(s32, f32, u32, args.steps, args.warmup)
    clk = clocks.stop()
    total_ms, value = replica_rate(float(sum(ms)), npts, args.steps, world, dist, "cuda")
    # per-kernel times from a shorter pass with an event pair around every launch
    k_tr = max(3, min(200, args.steps // 10))
    ms_traced, _ = timed_steps(s32, f32, u32, k_tr, 3, timing_capacity=k_tr * 16)
    ktimes, per_solve_launches = lgfm.lgf_plan_timings(s32.plan)
    lgfm.lgf_plan_set_timing(s32.plan, 0)

    # the same kernels once more with every launch on one stream, so the
    # dominant kernel is also timed without other chains sharing the SMs
    s_iso = lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, lgfm.LGF_FP32, fft_size_interval=args.fft_size,
                        near_kernel=args.near_kernel, interval_kernel=args.interval_kernel, single_stream=1,
                        free_sms=args.free_sms, interp_mode=args.interp_mode,
                        symmetric_spectra=args.symmetric_spectra)
    k_iso = max(3, min(100, args.steps // 10))
    timed_steps(s_iso, f32, u32, k_iso, 3, timing_capacity=k_iso * 16)
    kt_iso, _ = lgfm.lgf_plan_timings(s_iso.plan)
    s_iso.close()

    # FP64 form on the same GPU (shorter run)
    s64, f64, u64 = make(lgfm.LGF_FP64)
    k64 = max(3, min(50, args.steps // 20))
    ms64, _ = timed_steps(s64, f64, u64, k64, 3)
    rate64 = npts / (statistics.mean(ms64) * 1e-3)

    # end to end through the C ABI with host buffers (pinned), copies inside
    fh = torch.from_numpy(p.f).float().pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    k_e2e = max(3, min(500, args.steps // 4))
    for _ in range(3):
        lgfm.lgf_solve_host(s32.plan, fh, uh, stream)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        lgfm.lgf_solve_host(s32.plan, fh, uh, stream)
    e2e_serial_s = (time.perf_counter() - t0) / k_e2e
    # pipelined, one C-ABI call for all steps (lgf_solve_host_pipelined): each
    # step's input copy runs ahead of its solve and its result copy behind it
    # on library-owned copy streams, through double-buffered device arrays;
    # every step still copies its input in and its result out
    uhs = [uh, torch.empty_like(uh).pin_memory()]
    lgfm.lgf_solve_host_pipelined(s32.plan, [fh] * 4, [uhs[k % 2] for k in range(4)], stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lgfm.lgf_solve_host_pipelined(s32.plan, [fh] * k_e2e, [uhs[k % 2] for k in range(k_e2e)], stream)
    e2e_s = (time.perf_counter() - t0) / k_e2e

    # measured FMA peaks (the denominator of the ALU rooflines)
    fma = measure_fma_peaks(lgfm, dev)
    # roofline of the dominant kernel
    dom = max(ktimes.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_tot, dom_cnt) = dom
    dom_ms = dom_tot / dom_cnt
    pk, src = peaks()
    st = s32.stats()
    pairs = {l: st["pairs"][l] for l in range(p.n_levels)}
    assert pairs == interaction_pairs(p.blocks, p.n_levels)
    S0, SI = st["fft_size_level0"], st["fft_size_interval"]
    nw = {0: st["nw"][0], 1: st["nw"][1]}
    # useful complex products per launch of each product kernel
    upper = [(l, st["pairs"][l], st["nw"][l]) for l in range(2, p.n_levels) if st["nw"][l]]
    work = {"mac_level0": (pairs[0] * nw[0], f"{pairs[0]} near pairs x {nw[0]} frequencies"),
            "mac_all_levels": ((pairs[0] + pairs[1]) * nw[0] + sum(a * b for _, a, b in upper),
                               f"({pairs[0]} near + {pairs[1]} level-1 interaction pairs) x {nw[0]} frequencies"
                               + "".join(f" + {a} level-{l} pairs x {b}" for l, a, b in upper)),
            "mac_level01": ((pairs[0] + pairs[1]) * nw[0],
                            f"({pairs[0]} near + {pairs[1]} level-1 interaction pairs) x {nw[0]} frequencies"),
            "mac_interval_l1": (pairs[1] * nw[1], f"{pairs[1]} interaction pairs x {nw[1]} frequencies")}
    roof = None
    if dom_name in work:
        flops = 8.0 * work[dom_name][0]                   # one complex MAC = 8 real flops
        derived_tf = N_SM * FP32_FMA_LANES_PER_SM * 2 * float(pk.get("sm_max_mhz", SM_MAX_MHZ)) * 1e6 / 1e12
        peak_tf = fma["fp32_best_tflops"]
        ach = flops / (dom_ms * 1e-3) / 1e12
        iso_ms = kt_iso[dom_name][0] / kt_iso[dom_name][1]
        roof = {"bound": "alu", "kernel": dom_name, "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": ach / peak_tf, "traffic": profiled_traffic(dom_name),
                "peak_source": "measured: lgf_measure_fma_peak, best of fma.rn.f32 and fma.rn.f32x2 on all SMs",
                "peak_derived": derived_tf, "frac_of_derived": ach / derived_tf,
                "algorithmic": "8 flop x " + work[dom_name][1],
                "ms_in_step": dom_ms, "ms_isolated": iso_ms,
                # the persistent products leave some SMs to the levels >= 2
                # chain: the fraction of the peak of the SMs they run on
                "sms": int(st.get("persistent_ctas") or N_SM),
                "frac_of_its_sms": ach / (peak_tf * (st.get("persistent_ctas") or N_SM) / N_SM),
                "frac_isolated": flops / (iso_ms * 1e-3) / 1e12 / peak_tf,
                # the streaming model (every complex MAC reads a source and a
                # kernel value, 16 B in FP32): what HBM would have to deliver
                # without on-chip reuse, against the measured copy bandwidth
                "streamed_model_gbs": 16.0 * work[dom_name][0] / (dom_ms * 1e-3) / 1e9,
                "streamed_model_frac_of_hbm": 16.0 * work[dom_name][0] / (dom_ms * 1e-3) / 1e9
                / float(pk.get("hbm_gbs", 6800.0))}
    else:
        roof = {"bound": "hbm", "kernel": dom_name, "achieved": None, "peak": pk.get("hbm_gbs"),
                "unit": "GB/s", "frac": None, "traffic": None}

    out = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "points": npts, "blocks": len(p.blocks), "n_b": p.n_b,
                   "levels": p.n_levels, "interp_order": p.order, "fft_sizes": [S0, SI],
                   "l2": "flushed: 256 MiB write before every timed step",
                   "parallelism": f"replicas x{world}"},
        "fp64": {"value": rate64, "unit": "points/s", "ms_per_step": statistics.mean(ms64), "steps": k64},
        "e2e": {"value": npts / e2e_s, "unit": "points/s", "h2d_bytes_per_step": int(fh.numel() * 4),
                "d2h_bytes_per_step": int(uh.numel() * 4), "steps": k_e2e,
                "how": "one lgf_solve_host_pipelined call (C ABI, pinned host buffers): every step's H2D copy "
                       "runs ahead of its solve and its D2H copy behind it on library-owned copy streams, "
                       "double-buffered device arrays; wall clock over all steps"},
        "e2e_serial": {"value": npts / e2e_serial_s, "unit": "points/s",
                       "how": "lgf_solve_host per step (copy in, solve, copy out, synchronize)"},
        "gpu_launches": int(per_solve_launches) * args.steps,
        "launches_per_step": int(per_solve_launches),
        "kernel_ms": {k: v[0] / v[1] for k, v in ktimes.items()},
        "ms_per_step_traced": statistics.mean(ms_traced),
        "kernel_ms_isolated": {k: v[0] / v[1] for k, v in kt_iso.items()},
        "roofline": roof, "peaks": src, "fma_peaks": fma,
        "clocks": clk, "wall_s_timed": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import fmm
        rate, secs, cores, uref = cpu_oracle_rate(p)
        torch.cuda.synchronize()
        got = u32.double().cpu().numpy()
        out["cpu_baseline"] = {"value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
                               "nproc": os.cpu_count(), "cpu_model": cpu_model(),
                               "sample": f"one full oracle FMM solve of the 128^3 torus ({secs:.1f} s, "
                                         "kernel spectra precomputed outside the timing)"}
        out["cpu_baseline"]["direct_sum"] = direct_sum_rate()
        out["rel_err_fp32_vs_oracle"] = fmm.rel_linf(got, uref)
        out["rel_err_fp64_vs_oracle"] = fmm.rel_linf(u64.double().cpu().numpy(), uref)
    if world == 1 and not args.no_batch:
        try:
            out["batch"] = batch_run(torch, lgfm, max(3, min(200, args.steps // 10)), 3, flush)
        except Exception as exc:       # reported in the line, the headline stands
            out["batch"] = {"error": f"{type(exc).__name__}: {exc}"}
    if world == 1 and not args.no_fft_conv:
        try:
            out["fft_conv"] = fft_conv_run(torch, lgfm, max(3, min(100, args.steps // 20)), flush,
                                           fma["fp32_best_tflops"])
        except Exception as exc:
            out["fft_conv"] = {"error": f"{type(exc).__name__}: {exc}"}
    if world == 1 and not args.no_irregular:
        try:
            out["irregular"] = irregular_run(torch, lgfm, max(3, min(50, args.steps // 40)), flush)
        except Exception as exc:
            out["irregular"] = {"error": f"{type(exc).__name__}: {exc}"}
    if world == 1 and not args.no_sweep:
        try:
            out["error_sweep"] = error_sweep_run(torch, lgfm)
        except Exception as exc:
            out["error_sweep"] = {"error": f"{type(exc).__name__}: {exc}"}
    if world == 1 and not args.no_serve:
        try:
            out["serve"] = serve_run(torch, lgfm)
        except Exception as exc:
            out["serve"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(out))
    s32.close()
    s64.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
