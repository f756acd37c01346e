"""Host logic of the least-squares driver, on the CPU (no GPU, no library).

A dense random matrix on the host stands in for the plan: least_squares only
calls plan.forward / plan.adjoint (through the autograd function) and reads
plan.geom and plan.device.  Checked here:
  * the step 1/L with L = lambda_max(A^T A) + 24 reg bounds the gradient's
    Lipschitz constant (||D^T D|| <= 12 for the forward-difference
    Laplacian), so by the descent lemma every step lowers the objective;
  * the gradient through the autograd function equals A^T (A f - p) +
    2 reg D^T D f, formed here from dense matrices;
  * checkpoint / resume: a run interrupted by a failure injected on the host
    and resumed from its last checkpoint gives the same iterates and losses,
    bitwise, as one that was never interrupted; a checkpoint written for
    other data, reg or geometry is refused.
"""
import numpy as np
import pytest
import torch

from paper_2402_15641_gb300 import autograd as A
from paper_2402_15641_gb300.srt import Geometry

GEOM = Geometry(ms=4, mz=3, dxy=0.5, dz=0.5, radius=5.0, n_phi=4, phi0=0.0, n_zs=3, zs_lo=-0.75,
                zs_hi=0.75, n_ell=5, ell_lo=3.6, ell_hi=6.4)


class DensePlan:
    """plan.forward / plan.adjoint from a dense matrix on the host."""

    def __init__(self, geom=GEOM, seed=0, fail_after=None):
        self.geom, self.device = geom, torch.device("cpu")
        nf = geom.ms * geom.ms * geom.mz
        npr = geom.n_phi * geom.n_zs * geom.n_ell
        g = torch.Generator().manual_seed(seed)
        self.M = torch.rand(npr, nf, generator=g) * (torch.rand(npr, nf, generator=g) < 0.3)
        self.calls, self.fail_after = 0, fail_after

    def _tick(self):
        self.calls += 1
        if self.fail_after is not None and self.calls > self.fail_after:
            raise RuntimeError("injected failure")

    def forward(self, f):
        self._tick()
        return (self.M @ f.reshape(-1)).reshape(self.geom.n_phi, self.geom.n_zs, self.geom.n_ell)

    def adjoint(self, p):
        self._tick()
        return (self.M.T @ p.reshape(-1)).reshape(self.geom.ms, self.geom.ms, self.geom.mz)


def _data(plan, seed=1):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(plan.geom.n_phi, plan.geom.n_zs, plan.geom.n_ell, generator=g)


def _diff_matrix(ms, mz):
    """Forward differences along x, y and z over interior pairs, f[x][y][z]."""
    idx = np.arange(ms * ms * mz).reshape(ms, ms, mz)
    rows = []
    for a, b in ((idx[1:], idx[:-1]), (idx[:, 1:], idx[:, :-1]), (idx[:, :, 1:], idx[:, :, :-1])):
        for i, j in zip(a.ravel(), b.ravel()):
            r = np.zeros(ms * ms * mz)
            r[i], r[j] = 1.0, -1.0
            rows.append(r)
    return np.array(rows)


def test_laplacian_bound_and_gradient():
    D = _diff_matrix(GEOM.ms, GEOM.mz)
    assert np.linalg.eigvalsh(D.T @ D).max() <= 12.0
    f = torch.randn(GEOM.ms, GEOM.ms, GEOM.mz, dtype=torch.float64)
    assert float(A.grad_energy(f)) == pytest.approx(float(np.sum((D @ f.numpy().ravel()) ** 2)),
                                                     rel=1e-12)
    plan = DensePlan()
    plan.M = plan.M.double()
    p, reg = _data(plan).double(), 0.3
    f.requires_grad_(True)
    r = A.srt(f, plan) - p
    loss = 0.5 * (r * r).sum() + reg * A.grad_energy(f)
    (g,) = torch.autograd.grad(loss, f)
    M = plan.M.numpy()
    want = M.T @ (M @ f.detach().numpy().ravel() - p.numpy().ravel()) \
        + 2 * reg * D.T @ D @ f.detach().numpy().ravel()
    assert np.allclose(g.numpy().ravel(), want, rtol=1e-12, atol=1e-12)


def test_every_step_lowers_the_objective():
    plan = DensePlan()
    p = _data(plan)
    lam_true = float(np.linalg.eigvalsh((plan.M.T @ plan.M).double().numpy()).max())
    res = A.least_squares(plan, p, iters=25, reg=0.05)
    assert res.lipschitz == pytest.approx(lam_true, rel=1e-3)
    assert res.step == pytest.approx(1.0 / (res.lipschitz + 24 * 0.05))
    assert len(res.losses) == 26
    assert all(b < a for a, b in zip(res.losses, res.losses[1:])), res.losses


def test_interrupted_run_resumes_bitwise(tmp_path):
    p = _data(DensePlan())
    ref = A.least_squares(DensePlan(), p, iters=12, reg=0.05)
    ck = str(tmp_path / "lsq.pt")
    # 20 power-iteration products plus 2 per descent iteration: fail in iteration 8
    with pytest.raises(RuntimeError, match="injected"):
        A.least_squares(DensePlan(fail_after=40 + 2 * 7), p, iters=12, reg=0.05, checkpoint=ck,
                        every=3)
    st = torch.load(ck, weights_only=True)
    assert st["iter"] == 6 and len(st["losses"]) == 6
    plan = DensePlan()
    res = A.least_squares(plan, p, iters=12, reg=0.05, checkpoint=ck, every=3)
    assert plan.calls == 2 * 6 + 1          # no power iterations, 6 iterations, final loss
    assert torch.equal(res.f, ref.f)
    assert res.losses == ref.losses and res.step == ref.step
    assert torch.load(ck, weights_only=True)["iter"] == 12
    # a finished checkpoint: nothing left to run
    again = A.least_squares(DensePlan(), p, iters=12, reg=0.05, checkpoint=ck)
    assert torch.equal(again.f, ref.f) and again.losses == ref.losses


def test_checkpoint_for_other_problem_is_refused(tmp_path):
    p = _data(DensePlan())
    ck = str(tmp_path / "lsq.pt")
    A.least_squares(DensePlan(), p, iters=3, reg=0.05, checkpoint=ck)
    with pytest.raises(ValueError, match="data"):
        A.least_squares(DensePlan(), p * 2, iters=6, reg=0.05, checkpoint=ck)
    with pytest.raises(ValueError, match="reg"):
        A.least_squares(DensePlan(), p, iters=6, reg=0.1, checkpoint=ck)
    with pytest.raises(ValueError, match="geom"):
        A.least_squares(DensePlan(geom=GEOM.with_(weight_dtype="bf16")), p, iters=6, reg=0.05,
                        checkpoint=ck)
    with pytest.raises(ValueError, match="every"):
        A.least_squares(DensePlan(), p, iters=6, reg=0.05, checkpoint=ck, every=0)
