"""Argument checks of the Python binding, on the CPU (no GPU, no library).

The library takes raw pointers and sizes, so the binding refuses, before any
call, a tensor on the wrong device, an output that cannot hold the result and
a workspace on another device; it passes the workspace size in bytes.  A plan
object is put together here without assembling anything, with a fake library
that records the calls it receives: the refusals must leave it untouched, the
accepted calls must reach it with the right pointers and sizes."""
import ctypes

import pytest
import torch

from paper_2402_15641_gb300 import srt as S

GEOM = S.Geometry(ms=4, mz=3, dxy=0.5, dz=0.5, radius=5.0, n_phi=4, phi0=0.0, n_zs=3,
                  zs_lo=-0.75, zs_hi=0.75, n_ell=5, ell_lo=3.6, ell_hi=6.4)
WS = 4096  # bytes per volume of the fake workspace


class FakeLib:
    def __init__(self):
        self.calls = []

    def _size(self, ref, v):
        ref._obj.value = v
        return 0

    def srt_workspace_bytes(self, h, batch, ref):
        return self._size(ref, WS * batch)

    def srt_host_workspace_bytes(self, h, batch, ref):
        return self._size(ref, 2 * WS * batch)

    def __getattr__(self, name):
        if name.startswith("srt_") and name != "srt_plan_destroy":
            def call(*args):
                self.calls.append((name, *args))
                return 0
            return call
        if name == "srt_plan_destroy":
            return lambda h: 0
        raise AttributeError(name)


class Stream:
    cuda_stream = 0


def _plan(device):
    p = S.Plan.__new__(S.Plan)
    p.geom, p.device, p._h, p._ws, p.info = GEOM, torch.device(device), ctypes.c_void_p(1), {}, {}
    p._lib = FakeLib()
    return p


def test_accepted_calls_reach_the_library_with_byte_sizes():
    plan = _plan("cpu")
    f = torch.rand(GEOM.f_shape)
    p = plan.forward(f, stream=Stream())
    name, _, fp, pp, B, wsp, nb, _ = plan._lib.calls[-1]
    assert (name, fp, pp, B, nb) == ("srt_forward", f.data_ptr(), p.data_ptr(), 1, WS)
    assert p.shape == GEOM.p_shape
    # a caller's float workspace: its size goes over in bytes, not elements
    ws = torch.empty(3 * WS // 4, dtype=torch.float32)
    y = torch.rand(2, *GEOM.p_shape)
    out = torch.empty(2, *GEOM.f_shape)
    plan.adjoint(y, out=out, workspace=ws, stream=Stream())
    name, _, yp, op, B, wsp, nb, _ = plan._lib.calls[-1]
    assert (name, yp, op, B, wsp, nb) == ("srt_adjoint", y.data_ptr(), out.data_ptr(), 2,
                                          ws.data_ptr(), 3 * WS)
    # an output of another shape with the right number of elements is accepted
    plan.forward(f, out=torch.empty(GEOM.n_phi * GEOM.n_zs * GEOM.n_ell), stream=Stream())


@pytest.mark.parametrize("case", ["input device", "out size", "out dtype", "out strided",
                                  "out device", "workspace device", "workspace strided"])
def test_refused_before_any_call(case):
    plan = _plan("cpu")
    f = torch.rand(GEOM.f_shape)
    kw = {}
    if case == "input device":
        f = torch.empty(GEOM.f_shape, device="meta")
    elif case == "out size":
        kw["out"] = torch.empty(2, *GEOM.p_shape)           # holds 2 volumes, not 1
    elif case == "out dtype":
        kw["out"] = torch.empty(GEOM.p_shape, dtype=torch.float64)
    elif case == "out strided":
        kw["out"] = torch.empty(GEOM.n_phi, GEOM.n_zs, 2 * GEOM.n_ell)[..., ::2]
    elif case == "out device":
        kw["out"] = torch.empty(GEOM.p_shape, device="meta")
    elif case == "workspace device":
        kw["workspace"] = torch.empty(WS, dtype=torch.uint8, device="meta")
    elif case == "workspace strided":
        kw["workspace"] = torch.empty(2 * WS, dtype=torch.uint8)[::2]
    with pytest.raises(ValueError):
        plan.forward(f, stream=Stream(), **kw)
    assert plan._lib.calls == []


def test_host_calls_want_host_tensors_that_fit():
    plan = _plan("meta")                       # the plan's device: not the host
    f_h, p_h = torch.rand(GEOM.f_shape), torch.empty(GEOM.p_shape)
    plan.forward_host(f_h, p_h, stream=Stream())
    name, _, fp, pp, B, _, nb, _ = plan._lib.calls[-1]
    assert (name, fp, pp, B, nb) == ("srt_forward_host", f_h.data_ptr(), p_h.data_ptr(), 1,
                                     2 * WS)
    n = len(plan._lib.calls)
    with pytest.raises(ValueError):
        plan.forward_host(torch.empty(GEOM.f_shape, device="meta"), p_h, stream=Stream())
    with pytest.raises(ValueError):
        plan.forward_host(f_h, torch.empty(GEOM.p_shape, device="meta"), stream=Stream())
    with pytest.raises(ValueError):
        plan.adjoint_host(p_h, torch.empty(GEOM.ms, GEOM.ms), stream=Stream())  # too small
    with pytest.raises(ValueError):
        plan.adjoint_host(p_h[None].expand(2, *GEOM.p_shape), torch.empty(2, *GEOM.f_shape),
                          stream=Stream())                                     # not contiguous
    assert len(plan._lib.calls) == n


def test_dot_needs_device_tensors():
    with pytest.raises(ValueError, match="CUDA"):
        S.dot_f64(torch.rand(5), torch.rand(5))
    with pytest.raises(ValueError, match="equal size"):
        S.dot_f64(torch.rand(5), torch.rand(6))
