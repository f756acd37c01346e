"""Differentiation through the SRT (autograd backward = adjoint kernel):
central finite differences, the oracle's FP64 adjoint, and the least-squares
reconstruction on the 128^3 workload."""

import numpy as np
import pytest

from paper_2402_15641_gb300 import inputs as I
from tests.gpu_helpers import geom_pair, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    from paper_2402_15641_gb300 import build, srt as S, autograd as A
    assert torch.cuda.is_available()
    build.build()
    return S, A


def test_gradient_central_differences_16(mods, orc):
    """L(f) = 1/2 ||A f - p||^2 on the 16^3 geometry: the directional
    derivative from autograd matches central differences (h = 1e-3) along 20
    seeded unit directions, and the gradient matches A^T (A f - p) from the
    FP64 oracle."""
    import torch
    S, A = mods
    sz = dict(I.sizes("srt16fd"))
    g, o = geom_pair(orc, **sz)
    plan = S.Plan(g)
    f_np = I.phantom("srt16fd")
    p_np = I.probe("srt16fd")
    f = to_dev(f_np).requires_grad_(True)
    p = to_dev(p_np)
    r = A.srt(f, plan) - p
    loss = 0.5 * (r * r).sum()
    (grad,) = torch.autograd.grad(loss, f)
    want = orc.adjoint(o, orc.forward(o, f_np) - p_np)
    assert rel_l2(to_np(grad), want) <= 1e-5

    def L(x):
        rr = plan.forward(x) - p
        return 0.5 * S.dot_f64(rr, rr)

    rng = np.random.default_rng(I.SEED_FD)
    h = 1e-3
    gnorm = float(grad.norm())
    for _ in range(20):
        v = rng.standard_normal(g.f_shape)
        v /= np.linalg.norm(v)
        vd = to_dev(v)
        fd = (L(f.detach() + h * vd) - L(f.detach() - h * vd)) / (2 * h)
        an = S.dot_f64(grad, vd)
        assert abs(fd - an) <= 2e-3 * gnorm, (fd, an, gnorm)


def test_adjoint_function_backward_is_forward(mods, orc):
    import torch
    S, A = mods
    g, _ = geom_pair(orc, **dict(I.sizes("srt16fd")))
    plan = S.Plan(g)
    rng = np.random.default_rng(4)
    y = to_dev(rng.standard_normal(g.p_shape)).requires_grad_(True)
    w = to_dev(rng.standard_normal(g.f_shape))
    out = (A.srt_adjoint(y, plan) * w).sum()
    (gy,) = torch.autograd.grad(out, y)
    assert torch.equal(gy, plan.forward(w))


def test_least_squares_128(mods, orc):
    """Loss 1/2||A f - p||^2 + 1e-3 ||grad f||^2, 50 gradient iterations with
    step 1/L, p = forward of a seeded ball phantom plus 1% Gaussian noise."""
    import torch
    S, A = mods
    g = S.Geometry.from_sizes(I.sizes("srt128"))
    plan = S.Plan(g)
    w = dict(I.WORKLOADS["srt128"], n_blobs=0)
    f_true = to_dev(I.phantom(w))
    p, sigma = A.noisy_data(plan, f_true, 0.01)
    res = A.least_squares(plan, p, iters=50, reg=1e-3)
    losses = np.array(res.losses)
    assert res.lipschitz > 0 and np.isfinite(losses).all()
    assert np.all(np.diff(losses) <= 1e-6 * losses[0])      # monotone decrease
    assert losses[-1] < 0.05 * losses[0]
    err0 = 1.0
    err = float((res.f - f_true).norm() / f_true.norm())
    assert err < 0.9 * err0
    # the power-iteration estimate bounds the Rayleigh quotient of A^T A
    v = to_dev(np.random.default_rng(9).standard_normal(g.f_shape))
    rq = S.dot_f64(plan.forward(v), plan.forward(v)) / S.dot_f64(v, v)
    assert rq <= res.lipschitz * (1 + 1e-3)


class _Interrupted:
    """A real plan whose calls raise on the host after `fail_after` calls,
    before any further launch: the run stops between steps with nothing of
    its own in flight (the injected failure of a checkpoint / resume test)."""

    def __init__(self, plan, fail_after=None):
        self.plan, self.geom, self.device = plan, plan.geom, plan.device
        self.calls, self.fail_after = 0, fail_after

    def _tick(self):
        self.calls += 1
        if self.fail_after is not None and self.calls > self.fail_after:
            raise RuntimeError("injected failure")

    def forward(self, f, **kw):
        self._tick()
        return self.plan.forward(f, **kw)

    def adjoint(self, p, **kw):
        self._tick()
        return self.plan.adjoint(p, **kw)


def test_least_squares_resumes_bitwise_on_gpu(mods, orc, tmp_path):
    """Least squares on the 32^3 geometry with a checkpoint every 3
    iterations: a run stopped by a host-side failure in iteration 8 and
    resumed from its iteration-6 checkpoint computes the same iterates and
    losses, bit for bit, as a run that was never interrupted (the products
    hold no atomics; the iterate is saved exactly)."""
    import torch
    S, A = mods
    g, _ = geom_pair(orc, **dict(I.sizes("srt32")))
    plan = S.Plan(g)
    p = plan.forward(to_dev(I.phantom("srt32")))
    ref = A.least_squares(plan, p, iters=12, reg=1e-3)
    ck = str(tmp_path / "lsq32.pt")
    # 20 power-iteration calls (forward + adjoint each) and 2 per iteration:
    # the 8th iteration's first call fails
    with pytest.raises(RuntimeError, match="injected"):
        A.least_squares(_Interrupted(plan, fail_after=40 + 2 * 7), p, iters=12, reg=1e-3,
                        checkpoint=ck, every=3)
    st = torch.load(ck, weights_only=True)
    assert st["iter"] == 6 and len(st["losses"]) == 6
    again = _Interrupted(plan)
    res = A.least_squares(again, p, iters=12, reg=1e-3, checkpoint=ck, every=3)
    assert again.calls == 2 * 6 + 1  # resumed at iteration 7: no power iterations
    assert torch.equal(res.f, ref.f)
    assert res.losses == ref.losses and res.step == ref.step
