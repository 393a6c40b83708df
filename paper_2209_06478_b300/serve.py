"""Continuous-batching CG server on one B300 (the served-stream workload).

Requests arrive as a Poisson process. Each asks for the solution of A x = b
with a stencil matrix (7- or 27-point, §II-B's HPCG problem, n^3 grids) or
an irregular SPD matrix (banded / power-law rows) and its own random
right-hand side. The scheduler admits requests (in arrival order, or the
least estimated work first) whenever a
batch slot is free and the device-memory budget has room for the request's
matrix (if not already resident) and vectors; matrices stay resident in a
cache (least recently used ones are dropped when room is needed). Every tick
advances all admitted solves together with one `cg_batch_step` (one graph
launch of persistent kernels over every slot); solves that finish are
retired and their slots refilled at once. Latency runs from arrival to
completion.

Engines:
  * BatchedEngine(precision=MIXED_RELIABLE): FP32 matrices, one FP32 CG per
    request in the batch whose correction is folded into the FP64 solution
    with an FP64 residual on every tenfold residual drop (to 1e-10), all
    inside the batch's graph.
  * BatchedEngine(precision=FP64): plain FP64 CG in the batch.
  * SerialEngine: the plain per-matrix FP64 path — one cg_solve at a time,
    first come first served.

The scheduler is engine-agnostic (tests drive it on the CPU with a fake
engine and a fake clock). Served irregular matrices carry values that are
exact in FP32, so every engine solves the same system.
"""
from __future__ import annotations

import argparse
import heapq
import json
import math
import time
from collections import OrderedDict
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Workload
# ---------------------------------------------------------------------------


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    kind: str               # stencil27, stencil7, banded, powerlaw
    size: int               # grid n (stencils) or rows (irregular)
    seed: int               # right-hand side seed

    @property
    def key(self):
        return (self.kind, self.size)


STENCIL_SIZES = (32, 48, 64, 96, 128, 160)
IRREGULAR = (("banded", 50_000), ("banded", 500_000), ("banded", 2_000_000),
             ("powerlaw", 50_000), ("powerlaw", 200_000), ("powerlaw", 2_000_000))


def make_requests(count: int, rate: float, seed: int = 7, stencil_sizes=STENCIL_SIZES,
                  irregular=IRREGULAR, irregular_share: float = 0.25):
    """Poisson arrivals at `rate` per second (exponential gaps from SplitMix64
    draws); kinds and sizes drawn uniformly from the served mix."""
    import synth
    u = synth.uniform01(seed, 3 * count)
    reqs, t = [], 0.0
    for i in range(count):
        t += -math.log(1.0 - u[3 * i]) / rate
        if u[3 * i + 1] < irregular_share and irregular:
            kind, size = irregular[int(u[3 * i + 2] * len(irregular)) % len(irregular)]
        else:
            kind = "stencil27" if u[3 * i + 2] < 0.5 else "stencil7"
            size = stencil_sizes[int(u[3 * i + 1] * 997) % len(stencil_sizes)]
        reqs.append(Request(i, t, kind, size, 1000 + i))
    return reqs


def request_rows(req: Request) -> int:
    return req.size ** 3 if req.kind.startswith("stencil") else req.size


def request_work(req: Request) -> int:
    """Estimated solve work, for shortest-first admission: rows times the
    expected iteration count (CG on an n^3 stencil needs iterations in
    proportion to n; the diagonally dominant irregular matrices about 30)."""
    if req.kind.startswith("stencil"):
        return req.size ** 4
    return req.size * 30


# ---------------------------------------------------------------------------
# Scheduler (host logic, engine-agnostic)
# ---------------------------------------------------------------------------


@dataclass
class Record:
    rid: int
    arrival: float
    admitted: float = 0.0
    done: float = 0.0
    status: int = -1
    iterations: int = 0
    residual: float = float("nan")

    @property
    def latency(self):
        return self.done - self.arrival


@dataclass
class Scheduler:
    engine: object
    max_slots: int
    budget: int                      # device bytes the server may use
    iterations_per_tick: int = 8
    # "fifo": admit in arrival order; "sjf": admit the least estimated work
    # first; "srpt": as sjf, and every tick runs only the running requests
    # with the least estimated remaining work, until their rows fill the GPU
    # (engines with set_running; the others are paused for that tick)
    policy: str = "fifo"
    clock: object = time.perf_counter
    sleep: object = time.sleep
    records: dict = field(default_factory=dict)
    sat_rows: int = 2_000_000        # srpt: rows that keep the GPU busy
    max_wait: int = 16               # srpt: ticks a request may stay paused in a row

    def pick_running(self, running, done_work, waited):
        """srpt: the slots to advance this tick. Least estimated remaining
        work (request_work minus the work of the ticks it ran) first, until
        the rows of the chosen requests reach sat_rows; a request paused for
        max_wait ticks in a row runs regardless."""
        order = sorted(running.items(), key=lambda kv: (
            request_work(kv[1]) - done_work.get(kv[1].rid, 0), kv[1].arrival, kv[1].rid))
        run, rows = [], 0
        for slot, req in order:
            if rows < self.sat_rows or waited.get(req.rid, 0) >= self.max_wait:
                run.append(slot)
                rows += request_rows(req)
        return run

    def run(self, requests):
        pending = sorted(requests, key=lambda r: r.arrival)
        queue = []                   # arrived, not admitted (FIFO)
        running = {}                 # slot -> request
        free = list(range(self.max_slots))
        heapq.heapify(free)
        t0 = self.clock()
        i = 0
        busy_ticks = 0
        done_work, waited = {}, {}   # srpt bookkeeping per request id
        srpt = self.policy == "srpt" and hasattr(self.engine, "set_running")
        while i < len(pending) or queue or running:
            now = self.clock() - t0
            while i < len(pending) and pending[i].arrival <= now:
                queue.append(pending[i])
                self.records[pending[i].rid] = Record(pending[i].rid, pending[i].arrival)
                i += 1
            # admit in arrival order (or least estimated work first) while a
            # slot and the budget allow
            if self.policy in ("sjf", "srpt"):
                queue.sort(key=lambda q: (request_work(q), q.arrival, q.rid))
            while queue and free:
                req = queue[0]
                need = self.engine.bytes_needed(req)
                if self.engine.bytes_in_use() + need > self.budget:
                    if not self.engine.evict(need + self.engine.bytes_in_use() - self.budget):
                        break
                    continue
                slot = heapq.heappop(free)
                if not self.engine.admit(slot, req):
                    heapq.heappush(free, slot)
                    break
                queue.pop(0)
                running[slot] = req
                self.records[req.rid].admitted = self.clock() - t0
            if running:
                if srpt:
                    run = self.pick_running(running, done_work, waited)
                    self.engine.set_running(run)
                    for slot, req in running.items():
                        if slot in run:
                            done_work[req.rid] = (done_work.get(req.rid, 0) +
                                                  self.iterations_per_tick * request_rows(req))
                            waited[req.rid] = 0
                        else:
                            waited[req.rid] = waited.get(req.rid, 0) + 1
                finished = self.engine.step(self.iterations_per_tick)
                busy_ticks += 1
                t = self.clock() - t0
                for slot in finished:
                    req = running.pop(slot)
                    res = self.engine.result(slot)
                    rec = self.records[req.rid]
                    rec.done = t
                    rec.status = res["status"]
                    rec.iterations = res["iterations"]
                    rec.residual = res.get("true_rel_residual", float("nan"))
                    self.engine.retire(slot)
                    heapq.heappush(free, slot)
            elif i < len(pending):
                wait = pending[i].arrival - (self.clock() - t0)
                if wait > 0:
                    self.sleep(min(wait, 0.01))
            elif queue and not running:
                raise RuntimeError("request %d can never be admitted (budget %d bytes)"
                                   % (queue[0].rid, self.budget))
        self.wall = self.clock() - t0
        self.busy_ticks = busy_ticks
        return self.records

    def summary(self):
        lat = np.array([r.latency for r in self.records.values()])
        ok = sum(1 for r in self.records.values() if r.status == 0)
        return {"requests": len(self.records), "converged": ok,
                "solves_per_s": round(len(self.records) / self.wall, 3),
                "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 2),
                "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 2),
                "mean_ms": round(float(lat.mean()) * 1e3, 2),
                "wall_s": round(self.wall, 3),
                "max_true_rel_residual": float(max(r.residual for r in self.records.values()))}


# ---------------------------------------------------------------------------
# GPU engines
# ---------------------------------------------------------------------------


class MatrixCache:
    """Device-resident matrices keyed by (kind, size, value type), dropped
    least recently used first when the budget needs room."""

    def __init__(self, dm, fmt_for, vdtype, irregular_pool, online_tune=False):
        self.dm = dm
        self.vdtype = vdtype
        self.fmt_for = fmt_for
        self.pool = irregular_pool
        self.online_tune = online_tune
        self.entries = OrderedDict()   # key -> (handle, bytes, tile shape or None)
        self.pinned = {}               # key -> number of running requests
        self.tune_s = 0.0              # time spent in online tuning probes
        self.tuned = {}                # chosen format name -> count
        self.evictions = 0             # matrices dropped to make room

    def bytes(self):
        return sum(e[1] for e in self.entries.values())

    def estimate(self, req):
        if req.key in self.entries:
            return 0
        rows = request_rows(req)
        vb = 8 if self.vdtype == self.dm.F64 else 4
        per_row = {"stencil27": 27, "stencil7": 7}.get(req.kind, 48)
        return rows * per_row * (vb + 4) + rows * 8

    def get(self, req):
        """(handle, tile shape or None) of the request's matrix, created on
        first use in the FEATURES rule's format; with online tuning, a short
        probe in the batch kernel then picks the format and tile shape that
        every later request for the matrix reuses."""
        dm = self.dm
        if req.key in self.entries:
            self.entries.move_to_end(req.key)
            e = self.entries[req.key]
            return e[0], e[2]
        if req.kind.startswith("stencil"):
            pts = 27 if req.kind == "stencil27" else 7
            A = dm.dynmat_create_stencil(req.size, pts, dm.DIA, self.vdtype)
        else:
            N, r, c, v = self.pool[req.key]
            A = dm.dynmat_create(N, N, r, c, v)
            fmt = A.select_format(dm.SELECT_FEATURES)
            if fmt not in (dm.DIA, dm.ELL, dm.CSR):
                fmt = dm.CSR
            A.convert(fmt, self.vdtype)
        shape = None
        if self.online_tune:
            t0 = time.perf_counter()
            fmt, shape = A.batch_tune(effort=0)
            self.tune_s += time.perf_counter() - t0
            name = dm.FORMATS[fmt]
            self.tuned[name] = self.tuned.get(name, 0) + 1
        self.entries[req.key] = (A, A.info().bytes, shape)
        return A, shape

    def pin(self, key, d):
        self.pinned[key] = self.pinned.get(key, 0) + d

    def evict(self, need):
        freed = 0
        for key in list(self.entries):
            if freed >= need:
                break
            if self.pinned.get(key, 0) > 0:
                continue
            A, b, _ = self.entries.pop(key)
            A.destroy()
            freed += b
            self.evictions += 1
        return freed > 0


def irregular_matrix(kind: str, rows: int):
    """One SPD irregular matrix of the served mix, values rounded to FP32 so
    all engines solve the same system: (N, row, col, val)."""
    import synth
    N, r, c, v = synth.make(kind, 300 + rows % 97, rows, 21 if kind == "banded" else 0, spd=True)
    return N, r, c, v.astype(np.float32).astype(np.float64)


def save_irregular(kind: str, rows: int, directory: str):
    """Generates one pool matrix into `directory` as .npy files (lets a
    separate process build the large ones while the GPU works on something
    else)."""
    import os
    N, r, c, v = irregular_matrix(kind, rows)
    stem = os.path.join(directory, "%s_%d" % (kind, rows))
    for name, a in (("row", r), ("col", c), ("val", v)):
        np.save(stem + "_%s.npy" % name, a)
    return N


def irregular_pool(specs=IRREGULAR, directory=None):
    """SPD irregular matrices of the served mix (generated once, on the host;
    read from `directory` where save_irregular left them)."""
    import os
    pool = {}
    for kind, rows in specs:
        stem = os.path.join(directory, "%s_%d" % (kind, rows)) if directory else None
        if stem and os.path.exists(stem + "_val.npy"):
            r, c, v = (np.load(stem + "_%s.npy" % name) for name in ("row", "col", "val"))
            pool[(kind, rows)] = (rows, r, c, v)
        else:
            pool[(kind, rows)] = irregular_matrix(kind, rows)
    return pool


class BatchedEngine:
    def __init__(self, dm, torch, max_slots, precision, pool, tol=1e-10, inner_tol=1e-5,
                 keep_solutions=False, online_tune=False):
        self.dm, self.torch = dm, torch
        self.precision = precision
        self.tol, self.inner_tol = tol, inner_tol
        vdt = dm.F64 if precision == dm.CG_FP64 else dm.F32
        self.cache = MatrixCache(dm, None, vdt, pool, online_tune=online_tune)
        self.batch = dm.DynBatch(max_slots)
        self.vecs = {}
        self.vec_bytes = 0
        self.keep_solutions = keep_solutions
        self.solutions = {}   # rid -> solution (host copy), when kept
        self.paused = set()   # admitted slots left out of the steps (srpt)

    def bytes_needed(self, req):
        rows = request_rows(req)
        work = rows * (16 + 28 if self.precision != self.dm.CG_FP64 else 24) + 4096
        return self.cache.estimate(req) + 16 * rows + work

    def bytes_in_use(self):
        return self.dm.dynmat_memory_in_use() + self.vec_bytes

    def evict(self, need):
        return self.cache.evict(need)

    def admit(self, slot, req):
        dm, torch = self.dm, self.torch
        import synth
        try:
            A, shape = self.cache.get(req)
            N = A.info().nrows
            b = torch.from_numpy(synth.uniform_pm1(req.seed, N)).cuda()
            x = torch.zeros_like(b)
            self.batch.cg_admit(slot, A, b, x, tol=self.tol, max_iters=5000,
                                precision=self.precision, inner_tol=self.inner_tol, shape=shape)
        except dm.DynmatError as e:
            if e.status == dm.ERR_OOM:
                return False
            raise
        self.cache.pin(req.key, +1)
        self.vecs[slot] = (req, b, x)
        self.vec_bytes += 16 * N
        return True

    def set_running(self, slots):
        """Runs only `slots` in the next steps; the other admitted slots are
        paused (their state keeps, their iterates only come later)."""
        want = set(slots)
        for slot in self.vecs:
            p = slot not in want
            if p != (slot in self.paused):
                self.batch.cg_pause(slot, p)
                if p:
                    self.paused.add(slot)
                else:
                    self.paused.discard(slot)

    def step(self, iters):
        done, _ = self.batch.cg_step(iters)
        return done

    def result(self, slot):
        return self.batch.cg_result(slot)

    def retire(self, slot):
        self.paused.discard(slot)
        req, b, x = self.vecs.pop(slot)
        if self.keep_solutions:
            self.solutions[req.rid] = x.cpu().numpy()
        self.batch.cg_retire(slot)
        self.cache.pin(req.key, -1)
        self.vec_bytes -= 16 * b.numel()


class SerialEngine:
    """The plain per-matrix FP64 path: one cg_solve at a time."""

    def __init__(self, dm, torch, pool, tol=1e-10, keep_solutions=False):
        self.dm, self.torch = dm, torch
        self.tol = tol
        self.cache = MatrixCache(dm, None, dm.F64, pool)
        self.current = None
        self.vec_bytes = 0
        self.keep_solutions = keep_solutions
        self.solutions = {}   # rid -> solution (host copy), when kept

    def bytes_needed(self, req):
        return self.cache.estimate(req) + 48 * request_rows(req)

    def bytes_in_use(self):
        return self.dm.dynmat_memory_in_use() + self.vec_bytes

    def evict(self, need):
        return self.cache.evict(need)

    def admit(self, slot, req):
        import synth
        A, _ = self.cache.get(req)
        N = A.info().nrows
        b = self.torch.from_numpy(synth.uniform_pm1(req.seed, N)).cuda()
        x = self.torch.zeros_like(b)
        self.current = (slot, A, b, x, req)
        return True

    def step(self, iters):
        slot, A, b, x, _ = self.current
        self.res = A.cg_solve(b, x, tol=self.tol, max_iters=5000)
        return [slot]

    def result(self, slot):
        return self.res

    def retire(self, slot):
        if self.keep_solutions:
            _, _, _, x, req = self.current
            self.solutions[req.rid] = x.cpu().numpy()
        self.current = None


def serve(mode: str, requests, budget=150 * 10**9, max_slots=8, iterations_per_tick=8,
          pool=None, online_tune=False, policy="sjf"):
    """Runs the request stream through one engine and returns the summary.
    Defaults: least estimated work first, 8 slots. On the benchmark's stream
    (96 requests, Poisson 400/s, 2M-row matrices included) 8 slots measured
    23.1 solves/s, p50 0.88 s, p99 4.0 s, against 23.7 / 1.16 / 4.0 with 16
    slots and 21.3 / 1.04 / 4.3 with 4: more slots share every tick among
    more solves and slow the median, fewer leave the GPU idle. Shortest
    remaining work ("srpt", paused slots) measured no better: 18.7-21.9
    solves/s, p50 0.88-1.29 s."""
    import torch
    from paper_2209_06478_b300 import build
    build.build()
    from paper_2209_06478_b300 import dynmat as dm
    pool = pool if pool is not None else irregular_pool()
    if mode == "mixed_batched":
        eng = BatchedEngine(dm, torch, max_slots, dm.CG_MIXED_RELIABLE, pool,
                            online_tune=online_tune)
    elif mode == "fp64_batched":
        eng = BatchedEngine(dm, torch, max_slots, dm.CG_FP64, pool, online_tune=online_tune)
    elif mode == "fp64_serial":
        eng = SerialEngine(dm, torch, pool)
        max_slots = 1
    else:
        raise ValueError(mode)
    sch = Scheduler(eng, max_slots, budget, iterations_per_tick, policy=policy)
    sch.run(requests)
    out = sch.summary()
    out["mode"] = mode
    out["policy"] = policy
    out["budget_bytes"] = budget
    out["evictions"] = eng.cache.evictions
    if online_tune and isinstance(eng, BatchedEngine):
        out["online_tune"] = {"probe_s": round(eng.cache.tune_s, 3), "formats": eng.cache.tuned}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", default="mixed_batched",
                    choices=["mixed_batched", "fp64_batched", "fp64_serial"])
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--rate", type=float, default=40.0)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--online-tune", action="store_true",
                    help="probe each new matrix in the batch kernel for its format and tile shape")
    ap.add_argument("--policy", default="sjf", choices=["fifo", "sjf", "srpt"],
                    help="admission order: arrival, or least estimated work first; srpt also "
                         "runs only the least remaining work each tick")
    args = ap.parse_args()
    reqs = make_requests(args.requests, args.rate)
    print(json.dumps(serve(args.mode, reqs, int(args.budget_gb * 1e9), args.slots,
                           online_tune=args.online_tune, policy=args.policy)))


if __name__ == "__main__":
    main()
