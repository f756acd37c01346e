"""Serving loop: continuous batching over resident plans with CUDA graphs.
Each result must equal the same request computed alone; admission honours
the HBM budget; failures stay on the host (bad geometry, failed plan build,
budget exhaustion, cancellation)."""
import numpy as np
import pytest

from paper_2402_15641_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2402_15641_gb300 import build, serving as SV
    from paper_2402_15641_gb300.srt import Geometry, Plan
    assert torch.cuda.is_available()
    build.build()
    geoms = {
        "a": Geometry.from_sizes(I.sizes(I.serving_geometry(16, 32))),
        "b": Geometry.from_sizes(I.sizes(I.serving_geometry(24, 48))),
        "c": Geometry.from_sizes(I.sizes(I.serving_geometry(20, 40))),
    }
    payloads = SV.make_payloads(geoms, per=3)
    return SV, Plan, geoms, payloads


_ALONE = {}


def _alone(Plan, geoms, r):
    k = (r.key, geoms[r.key].weight_dtype)
    if k not in _ALONE:
        _ALONE[k] = Plan(geoms[r.key])
    plan = _ALONE[k]
    x = r.payload.cuda()
    out = plan.forward(x) if r.direction == "fwd" else plan.adjoint(x)
    return out.cpu()


@pytest.mark.parametrize("graphs,wdt", [(True, "fp32"), (False, "fp32"), (True, "bf16")])
def test_results_in_the_mix_equal_results_alone(env, graphs, wdt):
    import torch
    SV, Plan, geoms, payloads = env
    geoms = {k: g.with_(weight_dtype=wdt) for k, g in geoms.items()}
    srv = SV.Server(geoms, budget_bytes=8 << 30, max_batch=16, n_streams=3, use_graphs=graphs)
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(60):
        key = "abc"[int(rng.integers(3))]
        d = "fwd" if rng.random() < 0.5 else "adj"
        reqs.append(srv.submit(key, d, payloads[(key, d)][i % 3]))
        if i % 7 == 0:
            srv.step()  # arrivals interleaved with completions
    srv.drain()
    assert all(r.error is None and r.result is not None for r in reqs)
    assert max(srv.stats.batch_hist) > 1  # same-plan requests were batched
    for r in reqs:
        assert torch.equal(r.result, _alone(Plan, geoms, r)), (r.rid, r.key, r.direction)
    srv.close()


def test_budget_evicts_and_serves_alternating_plans(env):
    SV, Plan, geoms, payloads = env
    pa, pb = Plan(geoms["a"]), Plan(geoms["b"])
    plans = [pa.info["device_bytes"], pb.info["device_bytes"]]
    execs = [(int(np.prod(geoms[k].f_shape)) + int(np.prod(geoms[k].p_shape))) * 4
             + p.workspace_bytes(1) for k, p in (("a", pa), ("b", pb))]
    budget = max(plans) + max(execs) + (64 << 10)  # room for one plan and one executor
    assert budget < sum(plans) + sum(execs)
    pa.close(), pb.close()
    srv = SV.Server({k: geoms[k] for k in "ab"}, budget_bytes=budget, max_batch=1, n_streams=1)
    reqs = []
    for i in range(8):
        key = "ab"[i % 2]
        reqs.append(srv.submit(key, "fwd", payloads[(key, "fwd")][0]))
        srv.drain()
    assert all(r.error is None for r in reqs)
    assert srv.stats.evictions > 0 and srv.used_bytes() <= budget
    srv.close()


def test_host_side_failures(env):
    import torch
    SV, Plan, geoms, payloads = env
    bad = geoms["a"].with_(radius=0.1)  # sensors inside the volume: rejected by srt_plan

    def factory(g):
        if g.ms == 24:
            raise RuntimeError("injected plan-build failure")
        return Plan(g)

    srv = SV.Server({"a": geoms["a"], "b": geoms["b"], "bad": bad}, budget_bytes=8 << 30,
                    plan_factory=factory)
    ok = srv.submit("a", "fwd", payloads[("a", "fwd")][0])
    r_bad = srv.submit("bad", "fwd", payloads[("a", "fwd")][0])
    r_inj = srv.submit("b", "adj", payloads[("b", "adj")][0])
    r_unknown = srv.submit("zzz", "fwd", payloads[("a", "fwd")][0])
    r_shape = srv.submit("a", "adj", payloads[("a", "fwd")][0])
    r_cancel = srv.submit("a", "adj", payloads[("a", "adj")][1])
    srv.cancel(r_cancel)
    srv.drain()
    assert ok.error is None and ok.result is not None
    assert "plan build failed" in r_bad.error
    assert "injected" in r_inj.error
    assert r_unknown.error and r_shape.error
    assert r_cancel.result is None and r_cancel.cancelled
    assert srv.stats.failed == 4 and srv.stats.cancelled == 1
    srv.close()
    tiny = SV.Server({"a": geoms["a"]}, budget_bytes=16 << 10)  # below any plan
    r = tiny.submit("a", "fwd", payloads[("a", "fwd")][0])
    tiny.drain()
    assert r.error and "budget" in r.error
    tiny.close()


def test_poisson_run_reports_latency(env):
    SV, Plan, geoms, payloads = env
    srv = SV.Server(geoms, budget_bytes=8 << 30)
    for k in geoms:
        srv._plan(k)
    reqs = SV.poisson_run(srv, rate=400.0, duration_s=1.0, payloads=payloads, seed=3)
    s = SV.latency_summary(reqs)
    assert s["n"] == len(reqs) > 100
    assert 0 < s["p50_ms"] <= s["p99_ms"]
    srv.close()


_SIZES = {"a": (16, 32), "b": (24, 48), "c": (20, 40)}


@pytest.mark.parametrize("wdt,tol", [("fp32", 1e-5), ("bf16", 5e-3)])
def test_served_results_match_the_oracle(env, orc, wdt, tol):
    """Every forward and adjoint served in a mixed run of the three test
    geometries, against the FP64 oracle in full (relative L2 <= 1e-5 with
    FP32 entries, <= 5e-3 with BF16 entries)."""
    SV, Plan, geoms, payloads = env
    geoms = {k: g.with_(weight_dtype=wdt) for k, g in geoms.items()}
    srv = SV.Server(geoms, budget_bytes=8 << 30, max_batch=16, n_streams=3)
    reqs = [srv.submit(k, d, payloads[(k, d)][i]) for i in range(2) for d in ("fwd", "adj")
            for k in "abc"]
    srv.drain()
    for r in reqs:
        o = orc.OracleGeometry.default(**I.sizes(I.serving_geometry(*_SIZES[r.key])))
        x = r.payload.double().numpy()
        want = orc.forward(o, x) if r.direction == "fwd" else orc.adjoint(o, x)
        got = r.result.double().numpy()
        err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        assert err <= tol, (r.key, r.direction, err)
    srv.close()


@pytest.mark.parametrize("edge,n_phi", [(64, 128), (128, 256)])
def test_serving_mix_geometries_against_the_oracle(env, orc, edge, n_phi):
    """Geometries of the serving mix itself (64^3 / 128 columns and 128^3 /
    256 columns, FP32 entries), served as batches of two: forward values on
    256 seeded shells and adjoint values on 12 seeded voxels against the
    FP64 oracle (relative L2 <= 1e-5)."""
    SV, Plan, _, _ = env
    from paper_2402_15641_gb300.srt import Geometry
    sz = I.sizes(I.serving_geometry(edge, n_phi))
    geoms = {"m": Geometry.from_sizes(sz)}
    pl = SV.make_payloads(geoms, per=2, seed=11)
    srv = SV.Server(geoms, budget_bytes=16 << 30, max_batch=16, n_streams=2)
    reqs = [srv.submit("m", d, pl[("m", d)][i]) for d in ("fwd", "adj") for i in range(2)]
    srv.drain()
    o = orc.OracleGeometry.default(**sz)
    rng = np.random.default_rng(edge)
    sh = np.stack([rng.integers(0, n, 256) for n in o.p_shape], axis=1)
    vx = np.stack([rng.integers(0, n, 12) for n in o.f_shape], axis=1)
    for r in reqs:
        x = r.payload.double().numpy()
        got = r.result.double().numpy()
        if r.direction == "fwd":
            want = orc.forward_shells(o, x, sh)
            have = got[sh[:, 0], sh[:, 1], sh[:, 2]]
        else:
            want = orc.adjoint_voxels(o, x, vx)
            have = got[vx[:, 0], vx[:, 1], vx[:, 2]]
        err = float(np.linalg.norm(have - want) / np.linalg.norm(want))
        print(f"PARITY serving {edge}^3/{n_phi} {r.direction}: rel-L2 {err:.2e}")
        assert err <= 1e-5, (r.direction, err)
    srv.close()
