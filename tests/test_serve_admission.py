"""Host logic of the solve server: admission under the HBM budget, plan reuse
and eviction, overlap of requests, latency accounting.  A simulated clock and
fake plans stand in for the GPU (each fake solve takes a fixed time)."""
import numpy as np
import pytest

from paper_1402_6081_gb300.serve import AdmissionError, PlanPools, Request, run_stream, summarize


class Sim:
    def __init__(self, sizes, service):
        self.t = 0.0
        self.sizes = sizes            # key -> plan bytes
        self.service = service        # key -> seconds per solve
        self.live = {}
        self.used = 0
        self.max_used = 0
        self.made = 0
        self.running = 0
        self.max_running = 0
        self.next = 0

    def clock(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)

    def make(self, key):
        self.made += 1
        h = self.next
        self.next += 1
        self.live[h] = self.sizes[key]
        self.used += self.sizes[key]
        self.max_used = max(self.max_used, self.used)
        return h, self.sizes[key]

    def drop(self, h):
        self.used -= self.live.pop(h)

    def submit(self, slot, reqs):
        self.running += 1
        self.max_running = max(self.max_running, self.running)
        key = reqs[0].key
        return [self.t + self.service[key[0] if isinstance(key, tuple) else key], False]

    def poll(self, tok):
        if self.t >= tok[0] and not tok[1]:
            tok[1] = True
            self.running -= 1
        return tok[1]


def _requests(keys, rate, n, seed=0):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    return [Request(i, float(t[i]), keys[int(rng.integers(len(keys)))], 1000) for i in range(n)]


def test_all_served_within_budget_with_plan_reuse():
    sim = Sim({"a": 30, "b": 50, "c": 20}, {"a": 2e-3, "b": 5e-3, "c": 1e-3})
    pools = PlanPools(sim.make, sim.drop, budget_bytes=400)
    reqs = _requests(["a", "b", "c"], rate=2000.0, n=300)
    done, rejected = run_stream(reqs, pools, sim.submit, sim.poll, clock=sim.clock, sleep=sim.sleep,
                                need_bytes=lambda k: sim.sizes[k])
    assert not rejected and len(done) == 300
    assert sorted(d.rid for d in done) == list(range(300))
    assert sim.max_used <= 400
    assert sim.made <= 60                      # plans are kept and reused (>= 80% of requests)
    assert sim.max_running > 1                 # arrivals overlap running work
    for d in done:
        assert d.arrival <= d.start <= d.finish


def test_oversize_request_is_rejected_and_others_run():
    sim = Sim({"a": 30, "huge": 1000}, {"a": 1e-3, "huge": 1e-3})
    pools = PlanPools(sim.make, sim.drop, budget_bytes=100)
    reqs = [Request(0, 0.0, "a", 1), Request(1, 0.001, "huge", 1), Request(2, 0.002, "a", 1)]
    done, rejected = run_stream(reqs, pools, sim.submit, sim.poll, clock=sim.clock, sleep=sim.sleep,
                                need_bytes=lambda k: sim.sizes[k])
    assert rejected == [1]
    assert sim.made == 1                       # the oversize plan is never made
    assert sorted(d.rid for d in done) == [0, 2]
    assert sim.max_used <= 100
    with pytest.raises(AdmissionError):
        pools.acquire("huge", 0.0, need_bytes=1000)


def test_idle_plans_of_other_shapes_are_evicted():
    sim = Sim({"a": 60, "b": 60}, {"a": 1e-3, "b": 1e-3})
    pools = PlanPools(sim.make, sim.drop, budget_bytes=100)
    reqs = [Request(i, 0.01 * i, "ab"[i % 2], 1) for i in range(10)]
    done, rejected = run_stream(reqs, pools, sim.submit, sim.poll, clock=sim.clock, sleep=sim.sleep,
                                need_bytes=lambda k: sim.sizes[k])
    assert len(done) == 10 and not rejected
    assert sim.max_used <= 100
    assert sim.made == 10                      # each switch evicts the idle plan of the other shape


def test_request_waits_for_memory_instead_of_failing():
    # two concurrent "a" requests need two plans but only one fits: the second waits
    sim = Sim({"a": 60}, {"a": 5e-3})
    pools = PlanPools(sim.make, sim.drop, budget_bytes=100)
    reqs = [Request(0, 0.0, "a", 1), Request(1, 1e-4, "a", 1)]
    done, rejected = run_stream(reqs, pools, sim.submit, sim.poll, clock=sim.clock, sleep=sim.sleep)
    assert not rejected
    d = {x.rid: x for x in done}
    assert d[1].start >= d[0].finish - 1e-9
    assert sim.made == 1


def test_latency_equals_service_time_without_queueing():
    sim = Sim({"a": 10}, {"a": 2e-3})
    pools = PlanPools(sim.make, sim.drop, budget_bytes=100)
    reqs = [Request(i, 0.01 * i, "a", 100) for i in range(20)]
    done, _ = run_stream(reqs, pools, sim.submit, sim.poll, clock=sim.clock, sleep=sim.sleep)
    s = summarize(done, lambda rid: 100)
    assert s["requests"] == 20
    assert abs(s["p50_ms"] - 2.0) < 0.1 and abs(s["p99_ms"] - 2.0) < 0.1


def test_sizes_learned_from_the_first_plan_of_a_shape():
    # without estimates only the first plan of each shape may be made before
    # its size is known; later ones are admitted against the learned size
    sim = Sim({"a": 30, "b": 50, "c": 20}, {"a": 2e-3, "b": 5e-3, "c": 1e-3})
    pools = PlanPools(sim.make, sim.drop, budget_bytes=400)
    reqs = _requests(["a", "b", "c"], rate=2000.0, n=300, seed=4)
    done, rejected = run_stream(reqs, pools, sim.submit, sim.poll, clock=sim.clock, sleep=sim.sleep)
    assert len(done) == 300 and not rejected
    assert pools.known == {"a": 30, "b": 50, "c": 20}
    assert pools.used <= 400


def test_plan_made_in_the_background_does_not_block_others():
    # a shape whose plan takes long to make: with an executor the loop keeps
    # serving the requests of a shape that has an idle plan meanwhile
    import concurrent.futures
    import threading
    import time as _time

    sim = Sim({"fast": 10, "slow": 10}, {"fast": 1e-3, "slow": 1e-3})
    lock = threading.Lock()
    release = threading.Event()

    def make(key):
        if key == "slow":
            release.wait(5.0)            # held until the fast requests went through
        with lock:
            return sim.make(key)

    def drop(h):
        with lock:
            sim.drop(h)

    ex = concurrent.futures.ThreadPoolExecutor(1)
    pools = PlanPools(make, drop, budget_bytes=100, executor=ex)
    warm = pools.acquire("fast", 0.0, need_bytes=10)
    assert warm is None                  # made on the executor
    while pools.acquire("fast", 0.0) is None:
        _time.sleep(1e-3)
    pools.release(pools.slots["fast"][0], 0.0)
    reqs = [Request(0, 0.0, "slow", 1)] + [Request(i, 1e-3 * i, "fast", 1) for i in range(1, 11)]
    n_fast_done = []

    def poll(tok):
        done = sim.poll(tok)
        if done:
            n_fast_done.append(1)
            if len(n_fast_done) >= 10:
                release.set()
        return done

    done, rejected = run_stream(reqs, pools, sim.submit, poll, clock=sim.clock, sleep=sim.sleep,
                                need_bytes=lambda k: sim.sizes[k])
    pools.close()
    ex.shutdown()
    assert not rejected and len(done) == 11
    d = {x.rid: x for x in done}
    # every fast request finished before the slow one could start
    assert all(d[i].finish <= d[0].start for i in range(1, 11))
    assert sim.made == 2


def test_requests_pending_together_are_folded():
    # eight requests of one shape arrive at once: with fold allowing 4, they
    # run as two folded plans of 4 (key ("a", 4)), each completing all four
    sizes = {"a": 10, ("a", 4): 30, ("a", 2): 18}
    sim = Sim(sizes, {"a": 1e-3})
    pools = PlanPools(sim.make, sim.drop, budget_bytes=100)
    submitted = []

    def submit(slot, reqs):
        submitted.append((slot.key, [r.rid for r in reqs]))
        return sim.submit(slot, reqs)

    reqs = [Request(i, 0.0, "a", 1) for i in range(8)] + [Request(8, 0.5, "a", 1)]
    done, rejected = run_stream(reqs, pools, submit, sim.poll, clock=sim.clock, sleep=sim.sleep,
                                need_bytes=lambda k: sizes[k], fold=lambda key: 4)
    assert not rejected and sorted(d.rid for d in done) == list(range(9))
    assert [k for k, _ in submitted[:2]] == [("a", 4), ("a", 4)]
    assert sorted(r for _, rids in submitted[:2] for r in rids) == list(range(8))
    assert submitted[-1] == ("a", [8])             # alone: nothing pending beside it
    d = {x.rid: x for x in done}
    assert len({d[i].finish for i in range(4)}) == 1   # a folded group completes together
