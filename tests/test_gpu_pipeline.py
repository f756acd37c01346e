"""Pipelined host-buffer calls (srt_pipe_*): results bitwise equal to the
device-buffer calls for interleaved forward and adjoint sequences, with more
calls submitted than there are slots, waited in and out of order."""
import numpy as np
import pytest

from paper_2402_15641_gb300 import inputs as I
from tests.gpu_helpers import geom_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srt():
    import torch
    from paper_2402_15641_gb300 import build, srt as S
    assert torch.cuda.is_available()
    build.build()
    return S


@pytest.mark.parametrize("opts,slots", [({}, 2), ({}, 3), ({}, 4), ({"csr_only": True}, 3),
                                        ({"a1_rotation": True}, 3),
                                        ({"weight_dtype": "bf16", "rho_linear": True}, 2)])
@pytest.mark.parametrize("batch", [1, 2])
def test_pipeline_bitwise_equal_to_device_calls(srt, orc, opts, slots, batch):
    import torch
    g, _ = geom_pair(orc, **dict(I.sizes("srt32")), **opts)
    plan = srt.Plan(g)
    pipe = srt.Pipeline(plan, batch, slots=slots)
    rng = np.random.default_rng(23)
    dirs = ["forward", "adjoint", "forward", "forward", "adjoint", "adjoint", "forward"]
    calls = []
    for d in dirs:
        shp_in, shp_out = (g.f_shape, g.p_shape) if d == "forward" else (g.p_shape, g.f_shape)
        x = torch.from_numpy(rng.standard_normal((batch, *shp_in)).astype(np.float32)).pin_memory()
        y = torch.full((batch, *shp_out), float("nan"), dtype=torch.float32).pin_memory()
        calls.append((d, x, y, pipe.submit(d, x, y)))
    assert [c[3] for c in calls] == list(range(len(dirs)))
    order = [3, 0, 6, 1, 2, 5, 4]  # out of submission order
    for i in order:
        d, x, y, t = calls[i]
        r = pipe.wait(t)
        assert r is y or r is None  # None: released by the wait of a later ticket
        xd = x.cuda()
        want = plan.forward(xd) if d == "forward" else plan.adjoint(xd)
        np.testing.assert_array_equal(y.numpy().view(np.uint32), want.cpu().numpy().view(np.uint32))
    pipe.close()


def test_pipeline_stage_times_and_lagged_waits(srt, orc):
    """A forward/adjoint sequence waited one step behind (the pattern that
    keeps the device busy); stage times are kept for the last 8 calls."""
    import torch
    g, _ = geom_pair(orc, **dict(I.sizes("srt32")))
    plan = srt.Plan(g)
    pipe = srt.Pipeline(plan, 1)
    f = torch.rand(g.f_shape).pin_memory()
    y = torch.randn(g.p_shape).pin_memory()
    outs = {d: [torch.empty(s).pin_memory() for _ in range(2)]
            for d, s in (("forward", g.p_shape), ("adjoint", g.f_shape))}
    prev = None
    for k in range(12):
        cur = (pipe.submit("forward", f, outs["forward"][k % 2]),
               pipe.submit("adjoint", y, outs["adjoint"][k % 2]))
        if prev is not None:
            for t in prev:
                pipe.wait(t)
        prev = cur
    for t in prev:
        pipe.wait(t)
    for t in range(16, 24):
        h2d, comp, d2h, idle = pipe.stage_times(t)
        assert h2d > 0 and comp > 0 and d2h > 0 and idle >= 0
    with pytest.raises(srt.L.SrtError):
        pipe.stage_times(15)  # older than the last 8 calls
    pipe.close()


def test_pipeline_argument_errors(srt, orc):
    import torch
    g, _ = geom_pair(orc, **dict(I.sizes("srt16fd")))
    plan = srt.Plan(g)
    pipe = srt.Pipeline(plan, 1)
    f = torch.zeros(g.f_shape).pin_memory()
    p = torch.zeros(g.p_shape).pin_memory()
    with pytest.raises(ValueError):
        pipe.submit("forward", p, f)            # shapes swapped
    with pytest.raises(ValueError):
        pipe.submit("forward", f.cuda(), p)     # device tensor
    with pytest.raises(srt.L.SrtError):
        pipe.wait(0)                            # nothing submitted yet
    for bad in (1, 5):
        with pytest.raises(srt.L.SrtError):
            srt.Pipeline(plan, 1, slots=bad)    # slots outside 2-4
    t = pipe.submit("forward", f, p)
    assert pipe.wait(t) is p
    assert float(p.abs().max()) == 0.0
    pipe.close()
    with pytest.raises(RuntimeError):
        pipe.submit("forward", f, p)            # closed pipeline
    pipe2 = srt.Pipeline(plan, 1)
    plan.close()
    with pytest.raises(RuntimeError):
        pipe2.submit("forward", f, p)           # its plan was closed
    pipe2.close()
