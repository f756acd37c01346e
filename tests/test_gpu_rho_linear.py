"""GPU parity of the piecewise-linear intermediate (SRT_RHO_LINEAR) against
the oracle's linear mode.

The intermediate f^{1,2} is interpolated linearly in rho between the radius
nodes (Sec. 3.1 remarks that the two-stage method holds for other bases).
A1 is unchanged; A2's entries become hat integrals along the semicircles.
Checked here: A2's FP64 entries against the oracle's per-cell weights (1e-12
of the spacing), the CSR and Toeplitz-tap forms against each other, the
transforms against the oracle (FP32 1e-5, BF16 5e-3 relative L2, FP32
accumulation), the adjoint identity (1e-6), and that the basis changes the
result by far more than the tolerance.
"""
import math

import numpy as np
import pytest

from paper_2402_15641_gb300 import inputs as I
from tests.gpu_helpers import geom_pair, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

FP32_TOL, BF16_TOL, ADJ_TOL = 1e-5, 5e-3, 1e-6


@pytest.fixture(scope="module")
def srt():
    import torch
    from paper_2402_15641_gb300 import build, srt as S
    assert torch.cuda.is_available()
    build.build()
    return S


LIN = [
    dict(ms=5, mz=4, dxy=0.6, dz=0.45, radius=3.0, n_phi=6, n_zs=3, n_ell=12, phi0=0.37,
         zs=(-0.7, 1.1)),
    dict(I.sizes("srt32")),
    dict(ms=9, mz=3, dxy=0.3, dz=0.8, radius=2.5, n_phi=5, n_zs=7, n_ell=31, zs=(-2.0, 1.5)),
    dict(ms=1, mz=1, dxy=1.0, dz=1.0, radius=2.0, n_phi=1, n_zs=1, n_ell=2),
    dict(ms=6, mz=5, dxy=0.5, dz=0.4, radius=4.0, n_phi=4, n_zs=5, n_ell=1),
    dict(ms=12, mz=40, dxy=0.5, dz=0.2, radius=9.0, n_phi=8, n_zs=40, n_ell=19),
]


@pytest.mark.parametrize("sz", LIN)
def test_entries_match_oracle_hat_weights(srt, orc, sz):
    g, o = geom_pair(orc, keep_f64=True, csr_only=True, rho_linear=True, **sz)
    plan = srt.Plan(g)
    rp, col, v32, v64 = plan.export(2, f64=True)
    assert rp[-1] == len(col) == plan.info["nnz2"]
    for r in range(g.n_zs * g.n_ell):
        h, m = divmod(r, g.n_ell)
        seg = slice(rp[r], rp[r + 1])
        assert np.all(np.diff(col[seg]) > 0)
        got = dict(zip(col[seg].tolist(), v64[seg].tolist()))
        want = orc.semicircle_arcs(o, h, m)
        for k, v in want.items():
            assert abs(got.get(k, 0.0) - v) <= 1e-12 * g.dz, (r, k, got.get(k), v)
        assert set(got) <= set(want)
    np.testing.assert_array_equal(v32, v64.astype(np.float32))
    # A1 does not depend on the basis
    c = srt.Plan(g.with_(rho_linear=False))
    for which in (1, 3):
        a, b = plan.export(which), c.export(which)
        for x, y in zip(a[:3], b[:3]):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("sz", LIN[1:])
@pytest.mark.parametrize("wdt", ["fp32", "bf16"])
def test_transforms_match_oracle(srt, orc, sz, wdt):
    g, o = geom_pair(orc, weight_dtype=wdt, rho_linear=True, **sz)
    plan = srt.Plan(g)
    const = srt.Plan(g.with_(rho_linear=False))
    rng = np.random.default_rng(17)
    tol = FP32_TOL if wdt == "fp32" else BF16_TOL
    for batch in (1, 3):
        f = rng.uniform(0, 1, (batch, *g.f_shape))
        y = rng.standard_normal((batch, *g.p_shape))
        pf = np.stack([orc.forward(o, f[b]) for b in range(batch)])
        fa = np.stack([orc.adjoint(o, y[b]) for b in range(batch)])
        fd, yd = to_dev(f), to_dev(y)
        p_gpu, a_gpu = to_np(plan.forward(fd)), to_np(plan.adjoint(yd))
        e_p, e_a = rel_l2(p_gpu, pf), rel_l2(a_gpu, fa)
        if batch == 1:
            print(f"PARITY rho-linear {g.ms}x{g.mz} n_ell={g.n_ell} {wdt} "
                  f"(a2_taps={plan.info['a2_taps']}): forward rel-L2 {e_p:.3e}, "
                  f"adjoint rel-L2 {e_a:.3e}")
        assert e_p <= tol and e_a <= tol
        if g.n_ell > 2:  # the basis matters: the constant-basis plan is far off
            assert rel_l2(to_np(const.forward(fd)), pf) > 100 * FP32_TOL
        lhs, rhs = srt.dot_f64(plan.forward(fd), yd), srt.dot_f64(fd, plan.adjoint(yd))
        af = plan.forward(fd)
        assert abs(lhs - rhs) / math.sqrt(srt.dot_f64(af, af) * srt.dot_f64(yd, yd)) <= ADJ_TOL


TOEP = [dict(I.sizes("srt32")), dict(I.sizes("srt16fd")),
        dict(ms=12, mz=40, dxy=0.5, dz=0.2, radius=9.0, n_phi=8, n_zs=40, n_ell=19)]


@pytest.mark.parametrize("sz", TOEP)
def test_taps_equal_csr(srt, orc, sz):
    """Hats depend on rho only, so A2 stays Toeplitz in the ring offset: the
    taps plan stands for the CSR plan's A2 and gives the same transforms."""
    g, _ = geom_pair(orc, rho_linear=True, **sz)
    a, b = srt.Plan(g), srt.Plan(g.with_(csr_only=True))
    assert a.info["a2_taps"] == 1 and b.info["a2_taps"] == 0
    assert a.info["nnz2"] == b.info["nnz2"]
    for which in (2, 4):
        ra, ca, va, _ = a.export(which)
        rb, cb, vb, _ = b.export(which)
        np.testing.assert_array_equal(ra, rb)
        np.testing.assert_array_equal(ca, cb)
        assert rel_l2(va, vb) <= 1e-6
    rng = np.random.default_rng(9)
    f = to_dev(rng.uniform(0, 1, (2, *g.f_shape)))
    y = to_dev(rng.standard_normal((2, *g.p_shape)))
    assert rel_l2(to_np(a.forward(f)), to_np(b.forward(f))) <= 1e-5
    assert rel_l2(to_np(a.adjoint(y)), to_np(b.adjoint(y))) <= 1e-5


def test_with_a1_rotation_and_host_calls(srt, orc):
    sz = dict(I.sizes("srt32"))
    g, o = geom_pair(orc, rho_linear=True, a1_rotation=True, **sz)
    plan = srt.Plan(g)
    assert plan.info["a1_rot"] == 1
    import torch
    f = I.phantom("srt32")
    y = I.probe("srt32")
    p_host = plan.forward_host(torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)),
                               torch.empty(g.p_shape, dtype=torch.float32))
    a_host = plan.adjoint_host(torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)),
                               torch.empty(g.f_shape, dtype=torch.float32))
    assert rel_l2(p_host.double().numpy(), orc.forward(o, f)) <= FP32_TOL
    assert rel_l2(a_host.double().numpy(), orc.adjoint(o, y)) <= FP32_TOL
