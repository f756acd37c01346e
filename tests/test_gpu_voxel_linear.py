"""GPU parity of the piecewise-linear voxels (SRT_VOXEL_LINEAR) against the
oracle's voxel_linear mode.

The volume is the bilinear interpolation in (x, y) of its values at the
voxel centres (held constant across the outer half voxel), still constant
along z in a slab (Sec. 3.1 remarks that the two-stage method holds for
other bases).  A2 is unchanged; A1's entries become the nodes' bases
integrated along the in-plane circles.  Checked here: A1's FP64 entries
against the oracle's per-node weights (1e-11 of the spacing), the
transforms against the oracle (FP32 1e-5, BF16 5e-3 relative L2) in every
storage form of A1 (8-fold, quarter turns, every column, row by row), with
the piecewise-linear intermediate as well, the adjoint identity (1e-6), and
that the basis changes the result by far more than the tolerance.
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


VOX = [
    dict(ms=5, mz=4, dxy=0.6, dz=0.45, radius=3.0, n_phi=6, n_zs=3, n_ell=12, phi0=0.37,
         zs=(-0.7, 1.1)),
    dict(I.sizes("srt32")),
    dict(ms=10, mz=8, dxy=0.5, dz=0.5, radius=6.0, n_phi=16, n_zs=8, n_ell=13,
         zs=(-2.0 + 0.15, 2.0 + 0.15)),                   # 8-fold, odd radius count
    dict(ms=9, mz=3, dxy=0.3, dz=0.8, radius=2.5, n_phi=5, n_zs=7, n_ell=31, zs=(-2.0, 1.5)),
    dict(ms=1, mz=1, dxy=1.0, dz=1.0, radius=2.0, n_phi=1, n_zs=1, n_ell=2),
    dict(ms=2, mz=4, dxy=0.8, dz=0.5, radius=2.5, n_phi=8, n_zs=4, n_ell=9),
]


@pytest.mark.parametrize("sz", VOX)
def test_entries_match_oracle_node_weights(srt, orc, sz):
    g, o = geom_pair(orc, keep_f64=True, voxel_linear=True, **sz)
    plan = srt.Plan(g)
    rp, col, v32, v64 = plan.export(1, f64=True)
    assert rp[-1] == len(col) == plan.info["nnz1"]
    checked = 0
    for r in range(g.n_phi * g.n_ell):
        j, l = divmod(r, g.n_ell)
        seg = slice(rp[r], rp[r + 1])
        assert np.all(np.diff(col[seg]) > 0)
        got = dict(zip(col[seg].tolist(), v64[seg].tolist()))
        want = orc.circle_arcs(o, j, l)
        for k in set(got) | set(want):
            assert abs(got.get(k, 0.0) - want.get(k, 0.0)) <= 1e-11 * g.dxy, \
                (r, k, got.get(k), want.get(k))
        checked += len(got)
    assert checked > 0
    np.testing.assert_array_equal(v32, v64.astype(np.float32))
    # A2 does not depend on the voxel basis
    c = srt.Plan(g.with_(voxel_linear=False))
    for which in (2, 4):
        a, b = plan.export(which), c.export(which)
        for x, y in zip(a[:3], b[:3]):
            np.testing.assert_array_equal(x, y)


FORMS = [dict(), dict(a1_rotation=True), dict(a1_full=True), dict(rowwise=True)]


@pytest.mark.parametrize("sz", VOX[1:4])
@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("wdt", ["fp32", "bf16"])
def test_transforms_match_oracle(srt, orc, sz, form, wdt):
    g, o = geom_pair(orc, weight_dtype=wdt, voxel_linear=True, **sz)
    plan = srt.Plan(g.with_(**form))
    const = srt.Plan(g.with_(voxel_linear=False, **form))
    rng = np.random.default_rng(18)
    tol = FP32_TOL if wdt == "fp32" else BF16_TOL
    f = rng.uniform(0, 1, (2, *g.f_shape))
    y = rng.standard_normal((2, *g.p_shape))
    pf = np.stack([orc.forward(o, f[b]) for b in range(2)])
    fa = np.stack([orc.adjoint(o, y[b]) for b in range(2)])
    fd, yd = to_dev(f), to_dev(y)
    p_gpu, a_gpu = to_np(plan.forward(fd)), to_np(plan.adjoint(yd))
    e_p, e_a = rel_l2(p_gpu, pf), rel_l2(a_gpu, fa)
    print(f"PARITY voxel-linear {g.ms}x{g.mz} {form} {wdt} (a1_rot={plan.info['a1_rot']}): "
          f"forward rel-L2 {e_p:.3e}, adjoint rel-L2 {e_a:.3e}")
    assert e_p <= tol and e_a <= tol
    assert rel_l2(to_np(const.forward(fd)), pf) > 100 * FP32_TOL  # the basis matters
    af = plan.forward(fd)
    lhs, rhs = srt.dot_f64(af, yd), srt.dot_f64(fd, plan.adjoint(yd))
    assert abs(lhs - rhs) / math.sqrt(srt.dot_f64(af, af) * srt.dot_f64(yd, yd)) <= ADJ_TOL


@pytest.mark.parametrize("sz", [VOX[0], VOX[4], VOX[5]])
def test_small_and_degenerate_grids(srt, orc, sz):
    g, o = geom_pair(orc, voxel_linear=True, **sz)
    plan = srt.Plan(g)
    rng = np.random.default_rng(19)
    f = rng.uniform(0, 1, g.f_shape)
    y = rng.standard_normal(g.p_shape)
    assert rel_l2(to_np(plan.forward(to_dev(f))), orc.forward(o, f)) <= FP32_TOL
    assert rel_l2(to_np(plan.adjoint(to_dev(y))), orc.adjoint(o, y)) <= FP32_TOL


def test_with_linear_intermediate(srt, orc):
    """Both bases linear: bilinear voxels and the intermediate linear in rho."""
    g, o = geom_pair(orc, voxel_linear=True, rho_linear=True, **dict(I.sizes("srt32")))
    plan = srt.Plan(g)
    f = I.phantom("srt32")
    y = I.probe("srt32")
    assert rel_l2(to_np(plan.forward(to_dev(f))), orc.forward(o, f)) <= FP32_TOL
    assert rel_l2(to_np(plan.adjoint(to_dev(y))), orc.adjoint(o, y)) <= FP32_TOL


def test_sampled_shells_at_128(srt, orc):
    """128^3 (the bench launch configuration, 8-fold A1): sampled shells of
    the forward against the oracle's walk, sampled voxels of the adjoint
    against its per-node route."""
    sz = dict(I.sizes("srt128"))
    g, o = geom_pair(orc, voxel_linear=True, **{k: sz[k] for k in
                                                ("ms", "mz", "dxy", "dz", "radius", "n_phi",
                                                 "n_zs", "n_ell")})
    plan = srt.Plan(g)
    assert plan.info["a1_rot"] == 2
    f = I.phantom("srt128")
    y = I.probe("srt128")
    p = to_np(plan.forward(to_dev(f)))
    a = to_np(plan.adjoint(to_dev(y)))
    rng = np.random.default_rng(20)
    sh = np.stack([rng.integers(0, g.n_phi, 48), rng.integers(0, g.n_zs, 48),
                   rng.integers(0, g.n_ell, 48)], axis=1)
    want = orc.forward_shells(o, f, sh)
    got = p[sh[:, 0], sh[:, 1], sh[:, 2]]
    assert rel_l2(got, want) <= FP32_TOL
    vx = np.stack([rng.integers(0, g.ms, 12), rng.integers(0, g.ms, 12),
                   rng.integers(0, g.mz, 12)], axis=1)
    want = orc.adjoint_voxels(o, y, vx)
    got = a[vx[:, 0], vx[:, 1], vx[:, 2]]
    assert rel_l2(got, want) <= FP32_TOL
