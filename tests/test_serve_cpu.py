"""The serving scheduler's host logic on the CPU: a fake engine (fixed number
of ticks per request, fixed bytes) and a fake clock."""
import math

import pytest

from paper_2209_06478_b300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeEngine:
    def __init__(self, clock, tick_s=0.001, mem=0):
        self.clock = clock
        self.tick_s = tick_s
        self.mem = mem
        self.running = {}
        self.admit_order = []
        self.peak = 0
        self.evictions = 0

    def bytes_needed(self, req):
        return req.size

    def bytes_in_use(self):
        return self.mem

    def evict(self, need):
        self.evictions += 1
        return False

    def admit(self, slot, req):
        assert slot not in self.running
        self.running[slot] = [req, math.ceil(req.size / 10)]
        self.mem += req.size
        self.peak = max(self.peak, self.mem)
        self.admit_order.append(req.rid)
        return True

    def step(self, iters):
        self.clock.t += self.tick_s
        done = []
        for slot, rec in self.running.items():
            rec[1] -= 1
            if rec[1] <= 0:
                done.append(slot)
        return done

    def result(self, slot):
        return {"status": 0, "iterations": 1, "true_rel_residual": 1e-11}

    def retire(self, slot):
        req, _ = self.running.pop(slot)
        self.mem -= req.size


def test_poisson_requests_are_deterministic_and_ordered():
    a = serve.make_requests(50, 20.0, seed=3)
    b = serve.make_requests(50, 20.0, seed=3)
    assert [(r.arrival, r.kind, r.size) for r in a] == [(r.arrival, r.kind, r.size) for r in b]
    assert all(a[i].arrival < a[i + 1].arrival for i in range(49))
    # mean gap close to 1/rate
    gaps = [a[0].arrival] + [a[i + 1].arrival - a[i].arrival for i in range(49)]
    assert 0.02 < sum(gaps) / 50 < 0.09
    assert {r.kind for r in serve.make_requests(400, 10.0)} >= {"stencil27", "stencil7"}


def test_scheduler_fifo_budget_and_latency():
    clk = FakeClock()
    eng = FakeEngine(clk)
    reqs = [serve.Request(i, 0.0005 * i, "stencil27", 30 + (i % 3) * 20, i) for i in range(30)]
    sch = serve.Scheduler(eng, max_slots=4, budget=200, iterations_per_tick=8, clock=clk,
                          sleep=clk.sleep)
    recs = sch.run(reqs)
    assert len(recs) == 30 and all(r.status == 0 for r in recs.values())
    assert eng.admit_order == sorted(eng.admit_order)          # FIFO
    assert eng.peak <= 200                                      # budget respected
    for r in recs.values():
        assert r.arrival <= r.admitted <= r.done
    s = sch.summary()
    assert s["requests"] == 30 and s["p99_ms"] >= s["p50_ms"] > 0


def test_scheduler_fills_free_slots_continuously():
    clk = FakeClock()
    eng = FakeEngine(clk)
    # one long request and many short ones arriving together: short ones flow
    # through the other slots while the long one runs
    reqs = [serve.Request(0, 0.0, "stencil27", 1000, 0)]
    reqs += [serve.Request(i, 0.0, "stencil27", 10, i) for i in range(1, 9)]
    sch = serve.Scheduler(eng, max_slots=2, budget=10**9, clock=clk, sleep=clk.sleep)
    recs = sch.run(reqs)
    assert max(recs[i].done for i in range(1, 9)) < recs[0].done


def test_scheduler_reports_unadmittable_request():
    clk = FakeClock()
    eng = FakeEngine(clk)
    reqs = [serve.Request(0, 0.0, "stencil27", 500, 0)]
    sch = serve.Scheduler(eng, max_slots=2, budget=100, clock=clk, sleep=clk.sleep)
    with pytest.raises(RuntimeError, match="never be admitted"):
        sch.run(reqs)


def test_scheduler_sjf_admits_least_work_first_and_lowers_mean_latency():
    # everything queued at once, one slot: shortest-first is the order of
    # estimated work, and its mean latency is below FIFO's
    sizes = [90, 10, 50, 30, 70, 20]
    mean = {}
    for policy in ("fifo", "sjf"):
        clk = FakeClock()
        eng = FakeEngine(clk)
        reqs = [serve.Request(i, 0.0, "stencil27", s, i) for i, s in enumerate(sizes)]
        sch = serve.Scheduler(eng, max_slots=1, budget=10**9, clock=clk, sleep=clk.sleep,
                              policy=policy)
        recs = sch.run(reqs)
        if policy == "sjf":
            assert [sizes[i] for i in eng.admit_order] == sorted(sizes)
        else:
            assert eng.admit_order == list(range(len(sizes)))
        mean[policy] = sum(r.done - r.arrival for r in recs.values()) / len(recs)
    assert mean["sjf"] < mean["fifo"]
    # the estimate: n^4 for an n^3 stencil, rows x 30 for an irregular matrix
    assert serve.request_work(serve.Request(0, 0.0, "stencil27", 64, 0)) == 64 ** 4
    assert serve.request_work(serve.Request(0, 0.0, "powerlaw", 100000, 0)) == 3_000_000


class PausingEngine(FakeEngine):
    """A fake engine whose running requests advance only when the scheduler
    lets them run (set_running), as the batched engine's paused slots do. A
    tick costs tick_s while the rows it runs fit in `fill` rows and grows in
    proportion beyond that (a saturated GPU). Without set_running (run=None)
    every admitted request runs, as in sjf."""

    def __init__(self, clock, fill, pausing=True, **kw):
        super().__init__(clock, **kw)
        self.fill = fill
        self.pausing = pausing
        self.run = None
        self.ran = []

    def set_running(self, slots):
        self.run = set(slots)

    def step(self, iters):
        run = self.run if self.run is not None else set(self.running)
        rows = sum(serve.request_rows(self.running[s][0]) for s in run)
        self.clock.t += self.tick_s * max(1.0, rows / self.fill)
        self.ran.append(sorted(self.running[s][0].rid for s in run))
        done = []
        for slot, rec in self.running.items():
            if slot not in run:
                continue
            rec[1] -= 1
            if rec[1] <= 0:
                done.append(slot)
        return done


class NonPausingEngine(PausingEngine):
    """The same cost model with every admitted request in every tick."""
    set_running = property()  # no set_running: the scheduler cannot pause


def test_srpt_runs_the_least_remaining_work_and_lowers_the_median():
    """A large request is admitted first and small ones arrive just after:
    with every admitted request in every tick (sjf) the small ones share slow
    ticks with the large one; srpt runs the small ones alone (they fill the
    GPU's row budget), so they all finish before the large one and the
    median latency drops."""
    p50 = {}
    for policy in ("sjf", "srpt"):
        clk = FakeClock()
        eng = (PausingEngine if policy == "srpt" else NonPausingEngine)(clk, fill=16000)
        reqs = [serve.Request(0, 0.0, "stencil27", 100, 0)]           # 10^6 rows, 10 ticks
        reqs += [serve.Request(i, 0.0001, "stencil27", 20, i) for i in range(1, 9)]  # 8000 rows
        sch = serve.Scheduler(eng, max_slots=4, budget=10**9, clock=clk, sleep=clk.sleep,
                              policy=policy, sat_rows=16000)
        recs = sch.run(reqs)
        assert all(r.status == 0 for r in recs.values())
        lat = sorted(r.done - r.arrival for r in recs.values())
        p50[policy] = lat[len(lat) // 2]
        if policy == "srpt":
            assert max(recs[i].done for i in range(1, 9)) < recs[0].done
    assert p50["srpt"] < 0.5 * p50["sjf"]


def test_srpt_does_not_starve_a_paused_request():
    """Small requests keep arriving; the large one is paused while they fill
    the ticks, but never for more than max_wait ticks in a row."""
    clk = FakeClock()
    eng = PausingEngine(clk, fill=8000)
    reqs = [serve.Request(0, 0.0, "stencil27", 100, 0)]
    reqs += [serve.Request(i, 0.0005 * i, "stencil27", 20, i) for i in range(1, 60)]
    sch = serve.Scheduler(eng, max_slots=4, budget=10**9, clock=clk, sleep=clk.sleep,
                          policy="srpt", sat_rows=8000, max_wait=3)
    recs = sch.run(reqs)
    assert all(r.status == 0 for r in recs.values())
    ticks = [t for t, ran in enumerate(eng.ran) if 0 in ran]
    assert len(ticks) == 10                       # its ten ticks all ran
    assert ticks[0] <= 4                          # admitted at once, paused at most 3 ticks
    assert all(b - a <= 4 for a, b in zip(ticks, ticks[1:]))
