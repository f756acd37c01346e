"""The serving scheduler's host logic on the CPU, with the device replaced by
host fakes (no GPU, no library).

serving.Server takes its plan factory and clock as arguments; here the
module's Executor and torch's CUDA streams are swapped for fakes too.  A fake
executor "computes" on the host (2 * payload forward, payload + 1 adjoint)
and hands back an event that completes unless its geometry is held, and
timing events that report a chosen device time.  Checked here:
  * every request of a batch gets its own payload's result, batches are
    powers of two taken down from the queue;
  * the measured device time per volume caps later batch sizes;
  * queues take turns when streams are scarce (round robin);
  * the HBM budget: idle executors and then idle plans are evicted least
    recently used first, busy or queued plans never; work is deferred while
    something is in flight and failed when nothing could ever free memory;
  * the deadline: a batch that does not complete in time fails its requests
    ("timeout") while its buffers stay busy; when it completes later its
    results are dropped, so each request is answered exactly once; a
    request cancelled in flight is counted once, as cancelled.
Failures are made on the host (a held event, a clock moved forward); no GPU
is hung or faulted.
"""
import pytest
import torch

from paper_2402_15641_gb300 import serving as SV
from paper_2402_15641_gb300.srt import Geometry

HELD = set()          # geometry sizes (ms) whose batches do not complete
RUNS = []             # (key size, direction, number of payloads) per launch
DEVICE_MS = {}        # device time of one batch, by geometry size (default 1 ms)


def _geom(ms):
    return Geometry(ms=ms, mz=2, dxy=0.5, dz=0.5, radius=5.0, n_phi=2, phi0=0.0, n_zs=2, zs_lo=-0.5,
                    zs_hi=0.5, n_ell=3, ell_lo=4.0, ell_hi=6.0)


class FakePlan:
    def __init__(self, geom, nbytes=1000):
        self.geom, self.info, self.closed = geom, {"device_bytes": nbytes}, False

    def workspace_bytes(self, batch):
        return 0

    def close(self):
        self.closed = True


class _Event:
    def __init__(self, ms):
        self.ms = ms

    def query(self):
        return self.ms not in HELD


class _Timer:
    def __init__(self, t):
        self.t = t

    def elapsed_time(self, other):
        return other.t - self.t


class FakeExecutor:
    def __init__(self, plan, direction, batch, use_graph):
        g = plan.geom
        self.plan, self.direction, self.batch = plan, direction, batch
        n_f, n_p = g.ms * g.ms * g.mz, g.n_phi * g.n_zs * g.n_ell
        self.bytes = batch * (n_f + n_p) * 4 + plan.workspace_bytes(batch)
        self.busy, self.last_used = False, 0.0

    def run(self, stream, payloads):
        ms = self.plan.geom.ms
        RUNS.append((ms, self.direction, len(payloads)))
        outs = [2 * p if self.direction == SV.FWD else p + 1 for p in payloads]
        return _Event(ms), outs, (_Timer(0.0), _Timer(DEVICE_MS.get(ms, 1.0)))


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3
        return self.t


@pytest.fixture
def fake_device(monkeypatch):
    monkeypatch.setattr(SV, "Executor", FakeExecutor)
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: object())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    HELD.clear()
    RUNS.clear()
    DEVICE_MS.clear()
    yield
    HELD.clear()


def _server(geoms, budget=1 << 20, **kw):
    plans = {}

    def factory(g):
        p = FakePlan(g)
        plans.setdefault(g.ms, []).append(p)
        return p

    clock = Clock()
    srv = SV.Server(geoms, budget_bytes=budget, plan_factory=factory, clock=clock, **kw)
    return srv, plans, clock


def _payload(g, direction, seed):
    gen = torch.Generator().manual_seed(seed)
    return torch.rand(g.f_shape if direction == SV.FWD else g.p_shape, generator=gen)


def test_batches_return_each_request_its_own_result(fake_device):
    g = _geom(4)
    srv, _, _ = _server({"a": g})
    reqs = [srv.submit("a", SV.FWD, _payload(g, SV.FWD, i)) for i in range(5)]
    reqs += [srv.submit("a", SV.ADJ, _payload(g, SV.ADJ, 10 + i)) for i in range(3)]
    srv.drain()
    for r in reqs:
        assert r.error is None
        want = 2 * r.payload if r.direction == SV.FWD else r.payload + 1
        assert torch.equal(r.result, want)
    # powers of two taken down from the queue: 5 -> 4 + 1, 3 -> 2 + 1
    assert sorted(n for _, _, n in RUNS) == [1, 1, 2, 4]
    assert srv.stats.completed == 8 and srv.stats.failed == 0


def test_measured_device_time_caps_the_batch(fake_device):
    g = _geom(4)
    DEVICE_MS[4] = 24.0                        # 6 ms per volume in a batch of 4
    srv, _, _ = _server({"a": g}, batch_budget_s=0.010)
    for i in range(4):
        srv.submit("a", SV.FWD, _payload(g, SV.FWD, i))
    srv.drain()
    assert srv.cost[("a", SV.FWD)] == pytest.approx(0.006)
    for i in range(4):
        srv.submit("a", SV.FWD, _payload(g, SV.FWD, i))
    srv.drain()
    assert [n for _, _, n in RUNS] == [4, 1, 1, 1, 1]   # 10 ms budget / 6 ms: one at a time


def test_queues_take_turns(fake_device):
    ga, gb = _geom(4), _geom(6)
    srv, _, _ = _server({"a": ga, "b": gb}, n_streams=1, batching=False)
    for i in range(3):
        srv.submit("a", SV.FWD, _payload(ga, SV.FWD, i))
    for i in range(3):
        srv.submit("b", SV.FWD, _payload(gb, SV.FWD, i))
    srv.drain()
    assert [ms for ms, _, _ in RUNS] == [4, 6, 4, 6, 4, 6]


def test_budget_evicts_least_recently_used(fake_device):
    geoms = {k: _geom(ms) for k, ms in (("a", 4), ("b", 6), ("c", 8))}
    ex = {k: FakeExecutor(FakePlan(g), SV.FWD, 1, False).bytes for k, g in geoms.items()}
    # room for two plans and their executors, not three
    budget = 2000 + ex["b"] + ex["c"] + 1
    srv, plans, _ = _server(geoms, budget=budget, batching=False)
    for k in ("a", "b", "a", "c"):
        r = srv.submit(k, SV.FWD, _payload(geoms[k], SV.FWD, 0))
        srv.drain()
        assert r.error is None
    # "b" was used least recently: its plan went, "a" stayed
    assert plans[6][0].closed and not plans[4][0].closed
    assert set(srv.plans) == {"a", "c"}
    assert srv.used_bytes() <= budget
    assert srv.stats.evictions >= 3          # two idle executors, then plan "b"


def test_budget_defers_while_in_flight_and_fails_when_nothing_can_free(fake_device):
    ga, gb = _geom(4), _geom(6)
    ex = max(FakeExecutor(FakePlan(g), SV.FWD, 1, False).bytes for g in (ga, gb))
    # room for one plan and its executor at a time
    srv, plans, _ = _server({"a": ga, "b": gb}, budget=1000 + ex + 10, batching=False)
    HELD.add(4)
    ra = srv.submit("a", SV.FWD, _payload(ga, SV.FWD, 0))
    srv.step()                                 # a in flight and held
    rb = srv.submit("b", SV.FWD, _payload(gb, SV.FWD, 1))
    for _ in range(3):
        srv.step()
    assert rb.error is None and rb.result is None and srv.stats.deferred >= 3
    assert not plans[4][0].closed              # a busy plan is never evicted
    HELD.discard(4)
    srv.drain()
    assert ra.error is None and rb.error is None
    assert torch.equal(rb.result, 2 * rb.payload)
    assert plans[4][0].closed                  # evicted once idle, to admit b
    tiny, _, _ = _server({"a": ga}, budget=100)
    r = tiny.submit("a", SV.FWD, _payload(ga, SV.FWD, 0))
    tiny.drain()
    assert r.error and "budget" in r.error and tiny.stats.failed == 1


def test_deadline_fails_once_and_drops_the_late_result(fake_device):
    g = _geom(4)
    srv, _, clock = _server({"a": g}, deadline_s=0.5, n_streams=2)
    HELD.add(4)
    reqs = [srv.submit("a", SV.FWD, _payload(g, SV.FWD, i)) for i in range(2)]
    kept = srv.submit("a", SV.ADJ, _payload(g, SV.ADJ, 5))
    srv.step()                                 # both queues launched, both held
    srv.cancel(kept)                           # cancelled in flight
    clock.t += 1.0                             # past the deadline
    srv.step()
    assert all(r.error == "timeout" for r in reqs)
    assert kept.error is None and kept.cancelled
    assert srv.stats.failed == 2
    assert len(srv.free_slots) == 0            # buffers stay busy
    assert srv.pending()
    with pytest.raises(TimeoutError):
        srv.drain(timeout_s=0.05)
    HELD.discard(4)                            # the batches complete late
    srv.drain()
    assert all(r.result is None and r.error == "timeout" for r in reqs)
    assert kept.result is None
    assert srv.stats.completed == 0 and srv.stats.failed == 2 and srv.stats.cancelled == 1
    assert sorted(r.rid for r in srv.done) == sorted(r.rid for r in reqs)
    assert len(srv.free_slots) == 2
    # the server goes on serving
    r = srv.submit("a", SV.FWD, _payload(g, SV.FWD, 9))
    srv.drain()
    assert torch.equal(r.result, 2 * r.payload) and srv.stats.completed == 1
