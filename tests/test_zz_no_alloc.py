"""srt_forward_noalloc / srt_adjoint_noalloc: the transforms for callers that cannot allocate
device memory (their device memory belongs to another allocator, or they run
where an allocation is not allowed or too slow).  It uses scratch the library
keeps on each GPU instead of a caller workspace.

This file is collected last so that a failure here leaves every other test
already run.  It checks, through the C ABI, that two calls in a row give the
same output as srt_forward and srt_adjoint, bit for bit (the same kernels
run in the same order on the same inputs, so any difference, even one inside
the FP32 tolerance of the other parity tests, would be a fault), and that a
problem too large for the scratch is refused."""
import ctypes

import numpy as np
import pytest

from paper_2402_15641_gb300 import inputs as I

pytestmark = pytest.mark.gpu

def test_noalloc_forward_matches_forward_twice():
    import torch
    from paper_2402_15641_gb300 import build, _lib
    from paper_2402_15641_gb300.srt import Geometry, Plan
    assert torch.cuda.is_available()
    build.build()
    lib = _lib.lib()
    plan = Plan(Geometry.from_sizes(I.sizes("srt32")))
    assert plan.workspace_bytes(2) <= _lib.SRT_NOALLOC_WORKSPACE_BYTES
    rng = np.random.default_rng(77)
    stream = torch.cuda.current_stream()
    for call in range(2):  # two calls in a row: the shared scratch is reused
        f = torch.from_numpy(rng.uniform(0, 1, (2, *plan.geom.f_shape)).astype(np.float32)).cuda()
        want = plan.forward(f)
        got = torch.full_like(want, float("nan"))
        rc = lib.srt_forward_noalloc(plan._h, f.data_ptr(), got.data_ptr(), 2,
                                     ctypes.c_void_p(stream.cuda_stream))
        assert rc == _lib.SRT_OK, (call, rc)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert torch.equal(got, want), call
        y = torch.from_numpy(rng.standard_normal((2, *plan.geom.p_shape)).astype(np.float32)).cuda()
        want_a = plan.adjoint(y)
        got_a = torch.full_like(want_a, float("nan"))
        rc = lib.srt_adjoint_noalloc(plan._h, y.data_ptr(), got_a.data_ptr(), 2,
                                     ctypes.c_void_p(stream.cuda_stream))
        assert rc == _lib.SRT_OK, (call, rc)
        torch.cuda.synchronize()
        assert torch.isfinite(got_a).all()
        assert torch.equal(got_a, want_a), call


def test_noalloc_refuses_problems_larger_than_its_scratch():
    import torch
    from paper_2402_15641_gb300 import build, _lib
    from paper_2402_15641_gb300.srt import Geometry, Plan
    build.build()
    lib = _lib.lib()
    plan = Plan(Geometry.from_sizes(I.sizes("srt128")))
    assert plan.workspace_bytes(1) > _lib.SRT_NOALLOC_WORKSPACE_BYTES
    f = torch.zeros(plan.geom.f_shape, device="cuda")
    p = torch.zeros(plan.geom.p_shape, device="cuda")
    rc = lib.srt_forward_noalloc(plan._h, f.data_ptr(), p.data_ptr(), 1,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _lib.SRT_ERR_WORKSPACE
    assert lib.srt_forward_noalloc(None, f.data_ptr(), p.data_ptr(), 1, None) == _lib.SRT_ERR_ARG
    rc = lib.srt_adjoint_noalloc(plan._h, p.data_ptr(), f.data_ptr(), 1,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _lib.SRT_ERR_WORKSPACE
    assert lib.srt_adjoint_noalloc(None, p.data_ptr(), f.data_ptr(), 1, None) == _lib.SRT_ERR_ARG
