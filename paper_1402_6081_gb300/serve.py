"""Continuous-batching solve server.

Requests (a block-structured domain and its source) arrive over time.  The
server keeps plans resident in pools keyed by problem shape, admits an arrived
request as soon as a plan for its shape is idle or a new one fits the HBM
budget (evicting idle plans of other shapes if needed), and runs it on one of
a pool of CUDA streams: host-to-device copy of f, the solve, device-to-host
copy of u, a completion event.  Requests that arrive while others run are
admitted as plans and memory free up, so their work overlaps on the device.
Latency is measured from arrival to completion of the copy of u.

The admission logic runs on the host and takes a plan factory and a
submit/poll pair, so it runs the same with fake plans on a simulated clock.
A request whose plan must first be made does not hold up the others: with an
executor the plan is built on a worker thread (host tables, kernel spectra,
uploads) while the loop keeps admitting and polling, and arrived requests
behind a waiting one are admitted when an idle plan of their shape exists.
Dropping an idle plan never waits for the device (the library frees a plan's
workspace in stream order, after its own last solve).
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the run
    key: tuple              # problem shape (n_b, blocks per axis, ...)
    n_points: int


@dataclasses.dataclass
class Done:
    rid: int
    arrival: float
    start: float
    finish: float

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


class AdmissionError(RuntimeError):
    pass


class _Slot:
    """One resident plan with its device and pinned host buffers."""

    def __init__(self, key, handle, nbytes):
        self.key = key
        self.handle = handle
        self.nbytes = nbytes
        self.busy = False
        self.last_used = 0.0


class PlanPools:
    """Plans per shape under an HBM budget.  make(key) -> (handle, bytes);
    drop(handle) frees one.  With an executor (concurrent.futures), a new plan
    whose size is known or estimated is made on it: its bytes are reserved
    against the budget meanwhile and acquire returns None until it is ready."""

    def __init__(self, make, drop, budget_bytes: float, executor=None):
        self.make = make
        self.drop = drop
        self.budget = float(budget_bytes)
        self.used = 0.0
        self.slots: dict = collections.defaultdict(list)
        self.known: dict = {}               # shape -> bytes of its plan
        self.executor = executor
        self.making: dict = {}              # shape -> (future, reserved bytes)

    def _collect(self, key, now: float):
        """The plan made for this shape on the executor, once it is ready."""
        fut, reserved = self.making[key]
        if not fut.done():
            return None
        del self.making[key]
        self.used -= reserved
        handle, nbytes = fut.result()
        self.known[key] = nbytes
        s = _Slot(key, handle, nbytes)
        s.busy = True
        s.last_used = now
        self.slots[key].append(s)
        self.used += nbytes                 # may pass the budget by the estimate's error
        return s

    def acquire(self, key, now: float, need_bytes=None, allow_new: bool = True):
        """An idle plan of this shape, else a new one if it fits the budget
        (evicting idle plans, least recently used first), else None (wait).
        The size of a new plan is the one measured for this shape before, else
        need_bytes; with neither, the plan is made and then checked.
        allow_new=False only takes an idle plan."""
        for s in self.slots[key]:
            if not s.busy:
                s.busy = True
                s.last_used = now
                return s
        if key in self.making:
            return self._collect(key, now)
        if not allow_new:
            return None
        est = self.known.get(key, need_bytes)
        if est is not None:
            if est > self.budget:
                raise AdmissionError(f"request {key} needs {est:.3e} B, above the budget {self.budget:.3e} B")
            if not self._make_room(est):
                return None
            if self.executor is not None:
                self.used += est
                self.making[key] = (self.executor.submit(self.make, key), est)
                return None
        handle, nbytes = self.make(key)
        self.known[key] = nbytes
        if self.used + nbytes > self.budget and not self._make_room(nbytes):
            self.drop(handle)
            if nbytes > self.budget:
                raise AdmissionError(f"request {key} needs {nbytes:.3e} B, above the budget {self.budget:.3e} B")
            return None
        s = _Slot(key, handle, nbytes)
        s.busy = True
        s.last_used = now
        self.slots[key].append(s)
        self.used += nbytes
        return s

    def _make_room(self, nbytes) -> bool:
        idle = sorted((s for ss in self.slots.values() for s in ss if not s.busy), key=lambda s: s.last_used)
        while self.used + nbytes > self.budget and idle:
            self._evict(idle.pop(0))
        return self.used + nbytes <= self.budget

    def release(self, slot, now: float):
        slot.busy = False
        slot.last_used = now

    def _evict(self, slot):
        self.slots[slot.key].remove(slot)
        self.used -= slot.nbytes
        self.drop(slot.handle)

    def close(self):
        for fut, _ in self.making.values():
            self.drop(fut.result()[0])
        self.making.clear()
        for ss in self.slots.values():
            for s in ss:
                self.drop(s.handle)
        self.slots.clear()
        self.used = 0.0


def run_stream(requests, pools: PlanPools, submit, poll, clock=time.perf_counter, max_inflight: int = 64,
               need_bytes=None, idle_wait: float = 20e-6, sleep=time.sleep, fold=None):
    """Drive a request stream.  submit(slot, requests) starts the work of a
    list of requests on one plan and returns a token; poll(token) -> bool says
    whether it finished.  need_bytes(key) (optional) estimates a new plan's
    bytes before creating it.  fold(key) (optional) gives the largest number
    of requests of one shape to solve together: when several requests of a
    shape are pending at the same moment they take one plan of key (key, k),
    k a power of two (a multi-problem plan, one launch per phase for all k),
    if one is idle or can be made, else they run one by one.
    Returns the list of Done records and the rejected request ids."""
    pending = sorted(requests, key=lambda r: r.arrival)
    inflight = []
    done, rejected = [], []
    t0 = clock()

    def try_fold(i, now, allow_new):
        """A folded plan for pending[i] and the arrived requests of its shape
        behind it: (slot, indices) or None."""
        kmax = fold(pending[i].key) if fold else 1
        if kmax < 2:
            return None
        same = [j for j in range(i, len(pending))
                if pending[j].arrival <= now and pending[j].key == pending[i].key][:kmax]
        k = 1
        while 2 * k <= len(same):
            k *= 2
        while k >= 2:
            key = (pending[i].key, k)
            try:
                slot = pools.acquire(key, now, need_bytes(key) if need_bytes else None, allow_new=allow_new)
            except AdmissionError:
                slot = None
            if slot is not None:
                return slot, same[:k]
            k //= 2
        return None

    while pending or inflight:
        now = clock() - t0
        progressed = False
        # arrived requests in arrival order; once one has to wait, later ones
        # only take idle plans of their shape (no new plans ahead of it)
        i, waiting = 0, False
        while i < len(pending) and pending[i].arrival <= now and len(inflight) < max_inflight:
            r = pending[i]
            folded = try_fold(i, now, not waiting)
            if folded is not None:
                slot, idx = folded
                group = [pending[j] for j in idx]
                for j in reversed(idx):
                    del pending[j]
                start = clock() - t0
                inflight.append((group, slot, submit(slot, group), start))
                progressed = True
                continue
            try:
                slot = pools.acquire(r.key, now, need_bytes(r.key) if need_bytes else None, allow_new=not waiting)
            except AdmissionError:
                del pending[i]
                rejected.append(r.rid)
                progressed = True
                continue
            if slot is None:
                waiting = True              # memory, or its plan is being made
                i += 1
                continue
            del pending[i]
            start = clock() - t0
            inflight.append(([r], slot, submit(slot, [r]), start))
            progressed = True
        still = []
        for item in inflight:
            group, slot, tok, start = item
            if poll(tok):
                fin = clock() - t0
                for r in group:
                    done.append(Done(r.rid, r.arrival, start, fin))
                pools.release(slot, fin)
                progressed = True
            else:
                still.append(item)
        inflight = still
        if not progressed:
            if pending and not inflight and not pools.making and pending[0].arrival > now:
                sleep(min(pending[0].arrival - now, 1e-3))
            else:
                sleep(idle_wait)
    return done, rejected


def summarize(done, n_points_of) -> dict:
    lat = np.array([d.latency for d in done]) * 1e3
    t_first = min(d.arrival for d in done)
    t_last = max(d.finish for d in done)
    pts = sum(n_points_of(d.rid) for d in done)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "max_ms": float(lat.max()), "points_per_s": pts / (t_last - t_first),
            "span_s": t_last - t_first}


class _MultiPlan:
    """k copies of one problem in one multi-problem plan (lgf_plan_create_multi):
    one launch per phase solves all of them, each to the result it has alone."""

    def __init__(self, lgfm, p, k, precision, opts):
        self.lgfm = lgfm
        self.plan = lgfm.lgf_plan_create_multi([p.blocks] * k, p.n_b, [p.n_levels] * k, p.order, precision, **opts)

    def __call__(self, f, u, stream=None):
        self.lgfm.lgf_solve(self.plan, f, u, stream)
        return u

    def workspace_bytes(self):
        return self.lgfm.lgf_plan_workspace_bytes(self.plan)

    def close(self):
        if self.plan:
            self.lgfm.lgf_destroy(self.plan)
            self.plan = None


class GpuServer:
    """The CUDA side: plans per shape, device buffers, pinned host buffers and
    a pool of streams.  problems maps a shape key to a workloads-style problem
    (blocks, n_b, n_levels, order, f); source(request) optionally gives the
    request's own pinned host source (default: the shape's f).

    Folding: up to fold_max requests of one shape pending together (shapes of
    at most fold_points points) run as one multi-problem plan of key (shape,
    k).  k is limited so that the folded plan picks the same product-kernel
    form at every level as the plan of one request (the persistent form is
    chosen per level by its number of sibling groups, 48 or more), so every
    folded result has the bits of the same request solved alone.

    Large requests (more than big_points points) run on a stream of the
    default priority and their plans leave big_free_sms SMs to everything
    else (option free_sms, unless the tuned options set it): the persistent
    products of a large solve would otherwise hold every SM for milliseconds,
    and the requests that arrive meanwhile (their streams at high priority)
    would wait for them.  The large solve itself takes longer; the others see
    the free SMs."""

    def __init__(self, precision: int, problems: dict, budget_bytes: float = 120e9, n_streams: int = 16,
                 tuned_options=None, source=None, keep_results: bool = False, background_plans: bool = True,
                 fold_max: int = 8, fold_points: int = 1 << 18, big_points: int = 1 << 25,
                 big_free_sms: int = 32):
        import concurrent.futures

        import torch

        import paper_1402_6081_gb300 as lgfm
        self.torch = torch
        self.lgfm = lgfm
        self.precision = precision
        self.dtype = torch.float64 if precision == lgfm.LGF_FP64 else torch.float32
        self.problems = problems
        self.tuned = tuned_options or {}
        self.streams = [torch.cuda.Stream(priority=-1) for _ in range(n_streams)]   # high priority
        self.big_stream = torch.cuda.Stream(priority=0)
        self.big_points = big_points
        self.big_free_sms = big_free_sms
        self.next_stream = 0
        self.source = source
        self.host_f = {} if source else {k: torch.from_numpy(p.f).to(self.dtype).pin_memory()
                                         for k, p in problems.items()}
        self.keep_results = keep_results
        self.results = {}
        self.largest = {}                   # n_b -> (points, bytes) of the largest plan made
        self.groups = {}                    # shape -> sibling groups per level of its one-request plan
        self.fold_max = fold_max
        self.fold_points = fold_points
        self.folded = 0                     # requests served in folded plans
        self.device = torch.cuda.current_device()
        self.executor = concurrent.futures.ThreadPoolExecutor(1) if background_plans else None
        self.pools = PlanPools(self._make, self._drop, budget_bytes, executor=self.executor)

    @staticmethod
    def _split(key):
        """(shape, copies) of a pool key: a shape, or (shape, k) for a folded plan."""
        if isinstance(key, tuple) and len(key) == 2 and isinstance(key[1], int) and isinstance(key[0], tuple):
            return key[0], key[1]
        return key, 1

    def points(self, key) -> int:
        shape, k = self._split(key)
        p = self.problems[shape]
        return k * len(p.blocks) * p.n_b ** 3

    def need_bytes(self, key):
        """Size of a new plan of this shape: measured before for the shape, else
        scaled by points from the largest plan of the same block size (25%
        margin; small plans carry more per-point overhead), else unknown."""
        if key in self.pools.known:
            return self.pools.known[key]
        big = self.largest.get(self.problems[self._split(key)[0]].n_b)
        return None if big is None else 1.25 * big[1] * self.points(key) / big[0]

    def fold(self, shape) -> int:
        """Largest number of pending requests of this shape to solve together."""
        if self.fold_max < 2 or shape not in self.groups or self.points(shape) > self.fold_points:
            return 1
        k = 1
        while 2 * k <= self.fold_max and all((g >= 48) == (2 * k * g >= 48) for g in self.groups[shape]):
            k *= 2
        return k

    def _make(self, key):
        self.torch.cuda.set_device(self.device)     # also on the plan-making thread
        shape, k = self._split(key)
        p = self.problems[shape]
        opts = dict(self.tuned.get(shape, {}))
        if self.points(key) > self.big_points and "free_sms" not in opts:
            opts["free_sms"] = self.big_free_sms
        if k == 1:
            s = self.lgfm.Solver(p.blocks, p.n_b, p.n_levels, p.order, self.precision, **opts)
            st = s.stats()
            self.groups[shape] = [g for g in st["groups"][: st["top_product_level"] + 1]]
        else:
            s = _MultiPlan(self.lgfm, p, k, self.precision, opts)
        dims = (k * len(p.blocks), p.n_b, p.n_b, p.n_b)
        f = self.torch.empty(dims, dtype=self.dtype, device="cuda")
        u = self.torch.empty_like(f)
        uh = self.torch.empty(dims, dtype=self.dtype).pin_memory()
        nbytes = s.workspace_bytes() + 2 * f.numel() * f.element_size()
        if k == 1 and self.points(key) > self.largest.get(p.n_b, (0, 0))[0]:
            self.largest[p.n_b] = (self.points(key), nbytes)
        return (s, f, u, uh), nbytes

    def _drop(self, handle):
        # only idle plans are dropped (their last solve and copies completed);
        # the library releases the workspace in stream order, without waiting
        s, f, u, uh = handle
        s.close()

    def submit(self, slot, reqs):
        s, f, u, uh = slot.handle
        if self.points(slot.key) > self.big_points:
            st = self.big_stream
        else:
            st = self.streams[self.next_stream]
            self.next_stream = (self.next_stream + 1) % len(self.streams)
        nb = f.shape[0] // len(reqs)
        with self.torch.cuda.stream(st):
            for i, req in enumerate(reqs):
                src = self.source(req) if self.source else self.host_f[req.key]
                f[i * nb:(i + 1) * nb].copy_(src, non_blocking=True)
            s(f, u, st)
            uh.copy_(u, non_blocking=True)
            ev = self.torch.cuda.Event()
            ev.record(st)
        if len(reqs) > 1:
            self.folded += len(reqs)
        return (ev, uh, [r.rid for r in reqs], nb)

    def poll(self, tok):
        if not tok[0].query():
            return False
        if self.keep_results:
            ev, uh, rids, nb = tok
            for i, rid in enumerate(rids):
                self.results[rid] = uh[i * nb:(i + 1) * nb].numpy().copy()
        return True

    def warm(self, keys):
        """One resident plan per shape, made before the stream starts (largest
        first; each plan's size is measured, not estimated)."""
        keys = sorted(keys, key=self.points, reverse=True)
        slots = []
        for k in keys:
            sl = self.pools.acquire(k, 0.0)
            while sl is None and k in self.pools.making:
                time.sleep(1e-3)
                sl = self.pools.acquire(k, 0.0)
            slots.append(sl)
        for sl in slots:
            if sl is not None:
                self.pools.release(sl, 0.0)

    def run(self, requests, **kw):
        return run_stream(requests, self.pools, self.submit, self.poll, need_bytes=self.need_bytes,
                          fold=self.fold, **kw)

    def close(self):
        self.torch.cuda.synchronize()
        self.pools.close()
        if self.executor is not None:
            self.executor.shutdown(wait=True)
