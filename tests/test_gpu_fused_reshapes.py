"""The reshapes P2 (after A2) and P1^-1 (after A2^T) folded into the tile
products' epilogues, and P1 into the epilogue of the A1 product stored by
rotation (SRT_FUSE_RESHAPES; Algorithms 1 and 2: the same sums, written in
the next step's layout): bitwise equal to the default plan, which runs them
as kernels of their own, through device buffers and the host-buffer calls,
and within FP32 tolerance of the oracle."""
import numpy as np
import pytest

from paper_2402_15641_gb300 import inputs as I

from tests.gpu_helpers import geom_pair, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srt():
    import torch
    from paper_2402_15641_gb300 import build, srt as S
    assert torch.cuda.is_available()
    build.build()
    return S

FP32_TOL, BF16_TOL = 1e-5, 5e-3

GEOMS = [
    dict(I.sizes("srt32")),
    # odd radius count (partial 4-radius segments of p), 7 slabs (partial
    # 8-slab segments of F1), 11 rings offset from the slabs
    dict(ms=8, mz=7, dxy=0.4, dz=0.3, radius=5.0, n_phi=8, n_zs=11, n_ell=23, phi0=0.4,
         zs=(-1.65 - 0.57, -2.22 + 3.3)),
    # 260 dense columns: a full 256-column chunk and a 4-column one
    dict(ms=8, mz=12, dxy=0.5, dz=0.4, radius=6.0, n_phi=260, n_zs=5, n_ell=17, zs=(-1.0, 1.0)),
    # 12 columns: one 128-column chunk, mostly empty
    dict(ms=10, mz=16, dxy=0.4, dz=0.25, radius=6.0, n_phi=12, n_zs=16, n_ell=30),
    # 520 slabs: A1 (8-fold) in two blocks of 256 slabs and one of 8, odd
    # radius count (a half-empty radius pair in A1's fused blocks)
    dict(ms=8, mz=520, dxy=0.5, dz=0.05, radius=6.0, n_phi=8, n_zs=4, n_ell=11,
         zs=(-0.1, 0.1)),                                  # 4 rings spaced dz
]


def _fwd_launches(plan, g):
    """P1 folds into A1 where A1 is stored by rotation and n_phi, mz are
    multiples of 4; P2 into A2 whenever the tiles run."""
    return 2 if plan.info["a1_rot"] > 0 and g.n_phi % 4 == 0 and g.mz % 4 == 0 else 3


def _plans(srt, orc, sz, **kw):
    """The fused plan, the default (separate reshapes) plan, geometries."""
    g, o = geom_pair(orc, **sz, **kw)
    g = g.with_(fuse_reshapes=True)
    return srt.Plan(g), srt.Plan(g.with_(fuse_reshapes=False)), g, o


@pytest.mark.parametrize("sz", GEOMS)
@pytest.mark.parametrize("batch", [1, 2])
@pytest.mark.parametrize("wdt", ["fp32", "bf16"])
def test_fused_equals_separate(srt, orc, sz, batch, wdt):
    import torch
    plan, sep, g, o = _plans(srt, orc, sz, weight_dtype=wdt)
    assert plan.info["a2_taps"] == 1 and plan.info["tile_records"][0] > 0
    assert plan.launches_per_call(0, batch) == _fwd_launches(plan, g)
    assert plan.launches_per_call(1, batch) == 3
    assert sep.launches_per_call(0, batch) == 4 and sep.launches_per_call(1, batch) == 4
    rng = np.random.default_rng(7)
    f = to_dev(rng.uniform(0, 1, (batch, *g.f_shape)))
    y = to_dev(rng.standard_normal((batch, *g.p_shape)))
    pf, pa = plan.forward(f), plan.adjoint(y)
    assert torch.equal(pf, sep.forward(f))
    assert torch.equal(pa, sep.adjoint(y))
    if g.n_phi <= 32 and g.mz <= 32:
        tol = FP32_TOL if wdt == "fp32" else BF16_TOL
        assert rel_l2(to_np(pf[-1]), orc.forward(o, to_np(f)[-1])) <= tol
        assert rel_l2(to_np(pa[0]), orc.adjoint(o, to_np(y)[0])) <= tol
    plan.close()
    sep.close()


@pytest.mark.parametrize("sz", GEOMS[:2])
def test_fused_host_calls(srt, orc, sz):
    """The host-buffer calls copy p back in ring chunks as A2 writes them."""
    import torch
    plan, sep, g, _ = _plans(srt, orc, sz)
    rng = np.random.default_rng(8)
    B = 2
    f = rng.uniform(0, 1, (B, *g.f_shape)).astype(np.float32)
    y = rng.standard_normal((B, *g.p_shape)).astype(np.float32)
    pf_dev, pa_dev = sep.forward(to_dev(f)).cpu(), sep.adjoint(to_dev(y)).cpu()
    f_h, y_h = torch.from_numpy(f).pin_memory(), torch.from_numpy(y).pin_memory()
    p_h = torch.empty((B, *g.p_shape), dtype=torch.float32).pin_memory()
    a_h = torch.empty((B, *g.f_shape), dtype=torch.float32).pin_memory()
    plan.forward_host(f_h, p_h)
    plan.adjoint_host(y_h, a_h)
    assert torch.equal(p_h, pf_dev) and torch.equal(a_h, pa_dev)
    plan.close()
    sep.close()


def test_unfused_when_width_not_multiple_of_4(srt, orc):
    """Dense width batch x n_phi = 6: the tiles (and so the fusion) stand aside."""
    import torch
    sz = dict(ms=8, mz=8, dxy=0.5, dz=0.4, radius=6.0, n_phi=6, n_zs=8, n_ell=12)
    plan, sep, g, o = _plans(srt, orc, sz)
    assert plan.launches_per_call(0, 1) == 4
    assert plan.launches_per_call(0, 2) == 3
    rng = np.random.default_rng(9)
    f = to_dev(rng.uniform(0, 1, (1, *g.f_shape)))
    assert torch.equal(plan.forward(f), sep.forward(f))
    assert rel_l2(to_np(plan.forward(f)[0]), orc.forward(o, to_np(f)[0])) <= FP32_TOL
    plan.close()
    sep.close()


@pytest.mark.parametrize("sz", [GEOMS[0], GEOMS[2], GEOMS[4]])
@pytest.mark.parametrize("batch", [1, 3])
def test_fused_p1_with_rowwise_products(srt, orc, sz, batch):
    """Row-per-warp products (A1 by quarter turns, no register tiles): only
    P1 folds, into A1; the forward makes 3 launches, the adjoint 4."""
    import torch
    plan, sep, g, o = _plans(srt, orc, sz, rowwise=True)
    assert plan.info["a1_rot"] == 1 and plan.info["tile_records"][0] == 0
    assert plan.launches_per_call(0, batch) == 3 and plan.launches_per_call(1, batch) == 4
    rng = np.random.default_rng(10)
    f = to_dev(rng.uniform(0, 1, (batch, *g.f_shape)))
    assert torch.equal(plan.forward(f), sep.forward(f))
    plan.close()
    sep.close()
