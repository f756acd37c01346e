"""Continuous-batching request server for SRT forward and adjoint solves.

Requests arrive with a geometry, a direction (forward A f or adjoint A^T p)
and a host payload.  The server:
  * keeps one Plan per geometry resident on the GPU (built on first use) and
    admits work by an HBM budget covering plans and execution buffers,
    evicting idle executors and plans least-recently-used first;
  * queues requests per (geometry, direction) and turns each queue into one
    batched transform: B same-plan volumes share one pass over the sparse
    operators (the batched products of the library).  B is a power of two <=
    max_batch (each (plan, direction, B) has one reusable executor), taken
    DOWN from the queue length so no batch slot computes padding, and capped
    so that B times the measured device time per volume of that (plan,
    direction) stays within batch_budget_s: small transforms batch wide,
    large ones run alone instead of holding a stream for a long batch;
  * runs each executor's transform as a captured CUDA graph on one of several
    streams, so batches of different geometries overlap on the device, while
    new arrivals are admitted as slots and memory free up (continuous
    batching, not a queue drained one request at a time);
  * completes batches by polling CUDA events from the host with a deadline
    (no device-side waits), and reports p50/p99 latency and throughput.

Every transform runs in the library's CUDA kernels; this module only moves
payloads, schedules and keeps time.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .srt import Geometry, Plan

FWD, ADJ = "fwd", "adj"


@dataclass
class Request:
    rid: int
    key: str
    direction: str
    payload: torch.Tensor          # host float32, f_shape (fwd) or p_shape (adj)
    t_arrival: float = 0.0
    t_done: float | None = None
    result: torch.Tensor | None = None
    error: str | None = None
    cancelled: bool = False
    batch: int = 0

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_arrival


class Executor:
    """Device buffers (and a CUDA graph) for one (plan, direction, batch) shape.
    Payloads are copied straight from the requests' host tensors into the
    batch slots, and results straight into per-request pinned host tensors
    (torch's caching host allocator recycles them), so the server thread does
    no host-side copies of its own."""

    def __init__(self, plan: Plan, direction: str, batch: int, use_graph: bool):
        g = plan.geom
        self.plan, self.direction, self.batch = plan, direction, batch
        ishape = g.f_shape if direction == FWD else g.p_shape
        self.oshape = tuple(g.p_shape if direction == FWD else g.f_shape)
        dev = plan.device
        self.d_in = torch.zeros((batch, *ishape), dtype=torch.float32, device=dev)
        self.d_out = torch.zeros((batch, *self.oshape), dtype=torch.float32, device=dev)
        self.ws = torch.empty(plan.workspace_bytes(batch), dtype=torch.uint8, device=dev)
        self.bytes = (self.d_in.numel() + self.d_out.numel()) * 4 + self.ws.numel()
        self.graph = None
        self.busy = False
        self.last_used = 0.0
        if use_graph:
            s = torch.cuda.Stream(device=dev)
            with torch.cuda.stream(s):
                self._launch(s)          # warm-up outside capture
            s.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=s):
                self._launch(torch.cuda.current_stream())

    def _launch(self, stream):
        if self.direction == FWD:
            self.plan.forward(self.d_in, out=self.d_out, workspace=self.ws, stream=stream)
        else:
            self.plan.adjoint(self.d_in, out=self.d_out, workspace=self.ws, stream=stream)

    def run(self, stream, payloads):
        """Enqueue the H2D copies of the payloads into slots 0..n-1, the
        transform (graph replay) and the D2H copies of those slots on stream.
        Slots n..B-1 keep stale inputs: batch columns are independent, and
        their outputs are not read.  Returns (event, host outputs, (t0, t1))
        with timing events around the transform."""
        outs = []
        with torch.cuda.stream(stream):
            for i, pl in enumerate(payloads):
                self.d_in[i].copy_(pl, non_blocking=True)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            if self.graph is not None:
                self.graph.replay()
            else:
                self._launch(stream)
            t1.record(stream)
            for i in range(len(payloads)):
                o = torch.empty(self.oshape, dtype=torch.float32, pin_memory=True)
                o.copy_(self.d_out[i], non_blocking=True)
                outs.append(o)
            ev = torch.cuda.Event()
            ev.record(stream)
        return ev, outs, (t0, t1)


def batch_size(queued: int, max_batch: int, per_volume_s, budget_s: float) -> int:
    """Volumes to take from a queue of `queued`: at most max_batch, at most
    budget_s / per_volume_s when the device time per volume is known, and a
    power of two (rounded down, so no batch slot computes padding)."""
    n = min(queued, max_batch)
    if per_volume_s is not None and per_volume_s > 0:
        n = min(n, max(1, int(budget_s / per_volume_s)))
    n = max(1, n)
    return 1 << (n.bit_length() - 1)


@dataclass
class _InFlight:
    ex: Executor
    reqs: list
    event: object
    slot: int
    deadline: float
    outs: list
    timing: tuple


@dataclass
class ServerStats:
    completed: int = 0
    failed: int = 0
    cancelled: int = 0
    batches: int = 0
    batch_hist: collections.Counter = field(default_factory=collections.Counter)
    plan_builds: int = 0
    evictions: int = 0
    deferred: int = 0


class Server:
    def __init__(self, geometries: dict, budget_bytes: int, max_batch: int = 16, n_streams: int = 4,
                 use_graphs: bool = True, batching: bool = True, deadline_s: float = 30.0,
                 batch_budget_s: float = 0.010,
                 plan_factory=Plan, clock=time.perf_counter):
        self.geoms = dict(geometries)
        self.budget = int(budget_bytes)
        self.max_batch = max(1, int(max_batch)) if batching else 1
        self.use_graphs = use_graphs
        self.deadline_s = deadline_s
        self.batch_budget_s = batch_budget_s
        self.cost: dict = {}           # (key, dir) -> device seconds per volume (EMA)
        self.plan_factory = plan_factory
        self.clock = clock
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.free_slots = list(range(n_streams))
        self.plans: dict = {}
        self.plan_used: dict = {}
        self.bad_keys: dict = {}
        self.executors: dict = {}      # (key, dir, B) -> [Executor]
        self.queues: dict = collections.OrderedDict()
        self.inflight: list = []
        self.done: list = []
        self.stats = ServerStats()
        self._ids = 0

    # ------------------------------------------------------------ memory
    def used_bytes(self):
        b = sum(p.info["device_bytes"] for p in self.plans.values())
        b += sum(e.bytes for lst in self.executors.values() for e in lst)
        return b

    def _evict(self, need: int, protect: str | None) -> bool:
        """Free idle executors, then idle plans, LRU first, until need fits."""
        while self.used_bytes() + need > self.budget:
            idle = [(e.last_used, k, e) for k, lst in self.executors.items() for e in lst
                    if not e.busy]
            if idle:
                _, k, e = min(idle, key=lambda t: t[0])
                self.executors[k].remove(e)
                if not self.executors[k]:
                    del self.executors[k]
                self.stats.evictions += 1
                continue
            busy_keys = {k[0] for k, lst in self.executors.items() for e in lst if e.busy}
            queued = {k[0] for k, q in self.queues.items() if q}
            idle_plans = [(self.plan_used[k], k) for k in self.plans
                          if k != protect and k not in busy_keys and k not in queued]
            if not idle_plans:
                return False
            _, k = min(idle_plans)
            self.plans.pop(k).close()
            self.stats.evictions += 1
        return True

    def _plan(self, key):
        if key in self.plans:
            self.plan_used[key] = self.clock()
            return self.plans[key]
        geom = self.geoms[key]
        plan = self.plan_factory(geom)
        self.stats.plan_builds += 1
        self.plans[key] = plan
        self.plan_used[key] = self.clock()
        if self.used_bytes() > self.budget and not self._evict(0, protect=key):
            self.plans.pop(key).close()
            raise MemoryError(f"plan {key} exceeds the HBM budget")
        return plan

    def _executor(self, key, direction, B):
        for e in self.executors.get((key, direction, B), []):
            if not e.busy:
                return e
        plan = self.plans[key]
        g = plan.geom
        ni = int(np.prod(g.f_shape if direction == FWD else g.p_shape))
        no = int(np.prod(g.p_shape if direction == FWD else g.f_shape))
        need = B * (ni + no) * 4 + plan.workspace_bytes(B)
        if not self._evict(need, protect=key):
            return None
        e = Executor(plan, direction, B, self.use_graphs)
        self.executors.setdefault((key, direction, B), []).append(e)
        return e

    # ------------------------------------------------------------ requests
    def submit(self, key: str, direction: str, payload: torch.Tensor, t_arrival=None) -> Request:
        self._ids += 1
        r = Request(self._ids, key, direction, payload,
                    self.clock() if t_arrival is None else t_arrival)
        if key not in self.geoms or direction not in (FWD, ADJ):
            return self._fail(r, "unknown geometry or direction")
        if key in self.bad_keys:
            return self._fail(r, self.bad_keys[key])
        g = self.geoms[key]
        shape = tuple(g.f_shape if direction == FWD else g.p_shape)
        if tuple(payload.shape) != shape or payload.dtype != torch.float32:
            return self._fail(r, f"payload must be float32 {shape}")
        self.queues.setdefault((key, direction), collections.deque()).append(r)
        return r

    def cancel(self, r: Request):
        r.cancelled = True
        q = self.queues.get((r.key, r.direction))
        if q and r in q:
            q.remove(r)
            self.stats.cancelled += 1

    def _fail(self, r, msg):
        r.error = msg
        r.t_done = self.clock()
        self.stats.failed += 1
        self.done.append(r)
        return r

    # ------------------------------------------------------------ scheduling
    def _complete(self):
        still = []
        now = self.clock()
        for f in self.inflight:
            if f.event.query():
                t0, t1 = f.timing
                per = t0.elapsed_time(t1) / 1e3 / f.ex.batch
                ck = (f.reqs[0].key, f.reqs[0].direction)
                old = self.cost.get(ck)
                self.cost[ck] = per if old is None else 0.8 * old + 0.2 * per
                for i, r in enumerate(f.reqs):
                    if r.error is not None:  # already failed at the deadline
                        continue
                    if r.cancelled:
                        self.stats.cancelled += 1
                        continue
                    r.result = f.outs[i]
                    r.t_done = self.clock()
                    r.batch = len(f.reqs)
                    self.stats.completed += 1
                    self.done.append(r)
                f.ex.busy = False
                f.ex.last_used = now
                self.free_slots.append(f.slot)
            elif now > f.deadline:
                # the host stops waiting on these requests; the buffers stay
                # busy until the batch completes, and its late results are
                # dropped (each request is answered once)
                for r in f.reqs:
                    if not r.cancelled:
                        self._fail(r, "timeout")
                f.deadline = math.inf
                still.append(f)
            else:
                still.append(f)
        self.inflight = still

    def _launch_ready(self):
        for qkey in list(self.queues.keys()):
            q = self.queues[qkey]
            if not q or not self.free_slots:
                continue
            key, direction = qkey
            try:
                self._plan(key)
            except MemoryError as exc:
                if not self.inflight and not self.plans:
                    while q:  # nothing left to evict: it can never fit
                        self._fail(q.popleft(), str(exc))
                else:
                    self.stats.deferred += 1
                continue
            except Exception as exc:  # malformed geometry, failed build
                self.bad_keys[key] = f"plan build failed: {exc}"
                while q:
                    self._fail(q.popleft(), self.bad_keys[key])
                continue
            B = batch_size(len(q), self.max_batch, self.cost.get(qkey), self.batch_budget_s)
            n = B
            ex = self._executor(key, direction, B)
            if ex is None:
                if not self.inflight:  # nothing will free memory: it can never fit
                    while q:
                        self._fail(q.popleft(), f"request for {key} exceeds the HBM budget")
                else:
                    self.stats.deferred += 1
                continue
            reqs = [q.popleft() for _ in range(n)]
            slot = self.free_slots.pop()
            ex.busy = True
            ev, outs, timing = ex.run(self.streams[slot], [r.payload for r in reqs])
            self.inflight.append(_InFlight(ex, reqs, ev, slot, self.clock() + self.deadline_s,
                                           outs, timing))
            self.stats.batches += 1
            self.stats.batch_hist[n] += 1
            self.queues.move_to_end(qkey)  # round robin between queues

    def step(self):
        self._complete()
        self._launch_ready()

    def pending(self):
        return bool(self.inflight) or any(self.queues.values())

    def drain(self, timeout_s: float = 120.0):
        t_end = self.clock() + timeout_s
        while self.pending() and self.clock() < t_end:
            self.step()
        if self.pending():
            raise TimeoutError("server did not drain in time")

    def close(self):
        torch.cuda.synchronize()
        self.executors.clear()
        for p in self.plans.values():
            p.close()
        self.plans.clear()


# ---------------------------------------------------------------------------
def latency_summary(reqs):
    lat = np.array([r.latency for r in reqs if r.latency is not None and r.error is None])
    if len(lat) == 0:
        return {"n": 0}
    return {"n": int(len(lat)), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)}


def serving_geometries(edges=(64, 96, 128, 192), n_phis=(128, 256)) -> dict:
    """The serving mix: cubes of each edge at 25.6 mm field of view, R = 20 mm,
    rings = edge, radius bins = 4 * edge, for each number of columns."""
    from . import inputs as I
    out = {}
    for e in edges:
        for nphi in n_phis:
            out[f"{e}^3/{nphi}"] = Geometry.from_sizes(I.sizes(I.serving_geometry(e, nphi)))
    return out


def poisson_run(server: Server, rate: float, duration_s: float, payloads: dict, seed: int = 3,
                max_requests: int | None = None, drop_results: bool = False):
    """Drive the server with Poisson arrivals (rate per second), 50/50 forward
    and adjoint, geometry uniform over the server's mix; payloads[(key, dir)]
    is a list of host tensors drawn from round robin.  Returns the requests.
    drop_results releases each result once it has been delivered (a long run
    at a high rate would otherwise hold every output in host memory)."""
    rng = np.random.default_rng(seed)
    keys = sorted(server.geoms)
    t0 = server.clock()
    t_next = t0 + rng.exponential(1.0 / rate)
    reqs = []
    counters = collections.Counter()
    seen = len(server.done)
    while True:
        now = server.clock()
        while t_next <= now and t_next - t0 < duration_s:
            key = keys[int(rng.integers(len(keys)))]
            d = FWD if rng.random() < 0.5 else ADJ
            pool = payloads[(key, d)]
            pl = pool[counters[(key, d)] % len(pool)]
            counters[(key, d)] += 1
            reqs.append(server.submit(key, d, pl, t_arrival=t_next))
            t_next += rng.exponential(1.0 / rate)
            if max_requests and len(reqs) >= max_requests:
                t_next = math.inf
        server.step()
        if drop_results:
            while seen < len(server.done):
                server.done[seen].result = None
                seen += 1
        if (t_next - t0 >= duration_s or t_next == math.inf) and not server.pending():
            break
    return reqs


def make_payloads(geoms: dict, per: int = 2, seed: int = 3) -> dict:
    """Seeded ball phantoms (forward) and N(0, 1) data (adjoint), pinned."""
    from . import inputs as I
    out = {}
    for i, (key, g) in enumerate(sorted(geoms.items())):
        rng = np.random.default_rng(seed + 17 * i)
        fw, ad = [], []
        for _ in range(per):
            f, _ = I.balls(g.ms, g.mz, g.dxy, g.dz, 8, rng)
            fw.append(torch.from_numpy(f.astype(np.float32)).pin_memory())
            ad.append(torch.from_numpy(rng.standard_normal(g.p_shape).astype(np.float32))
                      .pin_memory())
        out[(key, FWD)], out[(key, ADJ)] = fw, ad
    return out


def probe_costs(geoms: dict, batches=(1, 16), reps: int = 10):
    """Device milliseconds per volume of each (geometry, direction) at each
    batch size (CUDA events around reps back-to-back transforms)."""
    rows = []
    for key in sorted(geoms):
        g = geoms[key]
        plan = Plan(g)
        for d in (FWD, ADJ):
            ish, osh = (g.f_shape, g.p_shape) if d == FWD else (g.p_shape, g.f_shape)
            row = {"geometry": key, "direction": d}
            for B in batches:
                x = torch.randn((B, *ish), device=plan.device)
                y = torch.empty((B, *osh), device=plan.device)
                ws = plan.workspace(B)
                run = plan.forward if d == FWD else plan.adjoint
                run(x, out=y, workspace=ws)
                torch.cuda.synchronize()
                t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0.record()
                for _ in range(reps):
                    run(x, out=y, workspace=ws)
                t1.record()
                t1.synchronize()
                row[f"ms_per_volume_b{B}"] = t0.elapsed_time(t1) / reps / B
                del x, y, ws
            rows.append(row)
        plan.close()
    return rows


def copy_tail_probe(seconds: float, mib: int = 151, window_s: float = 10.0):
    """Pinned host->device and device->host copies of `mib` MiB on two streams,
    back to back with a 4 ms pause, for `seconds`; yields the median and p99
    copy times (CUDA events) of each window.  On the GB300 machines used here
    the medians stay flat while the p99 grows several-fold after about a
    minute, whatever runs on the GPU."""
    n = (mib << 20) // 4
    h_in = torch.empty(n).pin_memory()
    h_out = torch.empty(n).pin_memory()
    d_a = torch.empty(n, device="cuda")
    d_b = torch.empty(n, device="cuda")
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    t_start = time.perf_counter()
    win, k = [], 1
    while time.perf_counter() - t_start < seconds:
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(sa):
            e[0].record()
            d_a.copy_(h_in, non_blocking=True)
            e[1].record()
        with torch.cuda.stream(sb):
            e[2].record()
            h_out.copy_(d_b, non_blocking=True)
            e[3].record()
        e[1].synchronize()
        e[3].synchronize()
        win.append((e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])))
        time.sleep(0.004)
        if time.perf_counter() - t_start >= k * window_s:
            w = np.array(win)
            p50, p99 = np.median(w, axis=0), np.percentile(w, 99, axis=0)
            yield {"t_s": k * window_s, "copies": len(w),
                   "h2d_ms_p50": float(p50[0]), "h2d_ms_p99": float(p99[0]),
                   "d2h_ms_p50": float(p50[1]), "d2h_ms_p99": float(p99[1])}
            win, k = [], k + 1


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="SRT serving benchmark (continuous batching)")
    ap.add_argument("--rates", default="200",
                    help="comma-separated Poisson arrival rates (requests/s)")
    ap.add_argument("--duration", type=float, default=30.0,
                    help="arrival window in seconds at the first rate")
    ap.add_argument("--max-requests", type=int, default=12000,
                    help="arrivals per rate at most (bounds the overloaded runs)")
    ap.add_argument("--warmup-s", type=float, default=5.0,
                    help="untimed run before each mode (executors, graphs, pinned blocks)")
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--max-batch", type=int, default=16)
    ap.add_argument("--batch-budget-ms", type=float, default=10.0,
                    help="device time per batch the batch size is capped to")
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--edges", default="64,96,128,192")
    ap.add_argument("--baseline", action="store_true", help="also run unbatched, no graphs")
    ap.add_argument("--weights", choices=["fp32", "bf16", "both"], default="fp32",
                    help="entry type of the batched server's plans (both: one run each)")
    ap.add_argument("--segments", type=int, default=6,
                    help="arrival-window segments per rate; the modes alternate between them")
    ap.add_argument("--copy-probe", type=float, default=0.0, metavar="SECONDS",
                    help="only time pinned 151 MB host<->device copies for this long and "
                         "print median / p99 per 10 s")
    ap.add_argument("--probe", action="store_true",
                    help="only print the device time per volume of every geometry and "
                         "direction at batch 1 and at --max-batch")
    a = ap.parse_args(argv)
    geoms = serving_geometries(tuple(int(x) for x in a.edges.split(",")))
    if a.copy_probe > 0:
        for row in copy_tail_probe(a.copy_probe):
            print(json.dumps(row), flush=True)
        return
    wdts = ["fp32", "bf16"] if a.weights == "both" else [a.weights]
    if a.probe:
        for w in wdts:
            gw = {k: g.with_(weight_dtype=w) for k, g in geoms.items()}
            for row in probe_costs(gw, (1, a.max_batch)):
                print(json.dumps({**row, "weights": w}), flush=True)
        return
    payloads = make_payloads(geoms)
    rates = [float(x) for x in a.rates.split(",")]
    batched = dict(max_batch=a.max_batch, use_graphs=True, batching=True,
                   batch_budget_s=a.batch_budget_ms / 1e3)
    modes = [("batched" if w == "fp32" else "batched_bf16", batched, w) for w in wdts]
    if a.baseline:
        modes.append(("unbatched_fp32", dict(max_batch=1, use_graphs=False, batching=False),
                      "fp32"))
    out = {"duration_s": a.duration, "max_requests": a.max_requests, "warmup_s": a.warmup_s,
           "batch_budget_ms": a.batch_budget_ms,
           "budget_gb": a.budget_gb, "geometries": sorted(geoms), "runs": []}
    # Every mode's server stays resident, and each rate's arrival window is
    # cut into segments that visit the modes in alternating order with the
    # same seeded arrivals: host<->device copy tails on the box drift over a
    # run (see copy_tail_probe), so modes measured one after the other would
    # not see the same conditions.
    budget = int(min(a.budget_gb, 240.0 / len(modes)) * 2**30)
    servers = {}
    for name, kw, w in modes:
        gw = {k: g.with_(weight_dtype=w) for k, g in geoms.items()}
        srv = Server(gw, budget, n_streams=a.streams, **kw)
        for k in geoms:  # plans up front: latencies measure serving, not plan builds
            srv._plan(k)
        poisson_run(srv, rates[-1], a.warmup_s, payloads, seed=99, drop_results=True,
                    max_requests=min(a.max_requests, 3000))
        srv.done.clear()
        servers[name] = srv
    names = [m[0] for m in modes]
    out["segments"] = a.segments
    out["budget_gb_per_server"] = budget / 2**30
    for rate in rates:
        acc = {n: dict(reqs=[], wall=0.0, batches=0, hist=collections.Counter(), failed=0,
                       evictions=0, seg=[]) for n in names}
        for seg in range(a.segments):
            for name in (names if seg % 2 == 0 else names[::-1]):
                srv, ac = servers[name], acc[name]
                base = dict(srv.stats.__dict__)
                base_hist = collections.Counter(srv.stats.batch_hist)
                t0 = time.perf_counter()
                got = poisson_run(srv, rate, a.duration / a.segments, payloads,
                                  seed=3 + 1000 * seg, drop_results=True,
                                  max_requests=max(1, a.max_requests // a.segments))
                ac["reqs"] += got
                sl = latency_summary([r for r in got if r.error is None and not r.cancelled])
                if sl["n"]:
                    ac["seg"].append((round(sl["p50_ms"], 3), round(sl["p99_ms"], 3)))
                ac["wall"] += time.perf_counter() - t0
                ac["batches"] += srv.stats.batches - base["batches"]
                ac["hist"] += srv.stats.batch_hist - base_hist
                ac["failed"] += srv.stats.failed - base["failed"]
                ac["evictions"] += srv.stats.evictions - base["evictions"]
                srv.done.clear()
        for name in names:
            ac, srv = acc[name], servers[name]
            ok = [r for r in ac["reqs"] if r.error is None and not r.cancelled]
            out["runs"].append(dict(
                mode=name, rate_per_s=rate, requests=len(ac["reqs"]), wall_s=ac["wall"],
                throughput_rps=len(ok) / ac["wall"], **latency_summary(ok),
                failed=ac["failed"], batches=ac["batches"],
                mean_batch=len(ok) / max(1, ac["batches"]),
                batch_hist={int(k): int(v) for k, v in sorted(ac["hist"].items())},
                evictions=ac["evictions"], hbm_used_gb=srv.used_bytes() / 2**30,
                # the same arrivals segment by segment: the spread of p50 / p99
                # over segments is the run-to-run noise a mode difference must beat
                segment_p50_p99_ms=ac["seg"]))
            print(json.dumps(out["runs"][-1]), flush=True)
    for srv in servers.values():
        srv.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
