"""Column-block plans on one GPU (the per-rank operators of the sharded
transform, paper_2402_15641_gb300/sharded.py): a plan for sensor columns
[j0, j1) of the aperture computes their angles exactly as the whole plan
does, so its forward is bitwise the whole forward's rows of those columns,
and the blocks' adjoints add up to the whole adjoint (FP32 summation order
apart); against the FP64 oracle within the FP32 tolerance."""
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


@pytest.mark.parametrize("sz,cuts", [(dict(I.sizes("srt32")), (0, 24, 64)),
                                     (dict(I.sizes("srt16fd")), (0, 11, 12, 32)),
                                     (dict(ms=9, mz=7, dxy=0.4, dz=0.3, radius=5.0, n_phi=7,
                                           n_zs=11, n_ell=23, phi0=0.4), (0, 3, 7))])
@pytest.mark.parametrize("wdt", ["fp32", "bf16"])
def test_column_blocks_compose_the_whole_transform(srt, orc, sz, cuts, wdt):
    import torch
    g, o = geom_pair(orc, weight_dtype=wdt, **sz)
    # a block stores A1 for each of its columns; so does the whole plan here
    # (by default it would keep a symmetric subset and derive the rest)
    whole = srt.Plan(g.with_(a1_full=True))
    rng = np.random.default_rng(41)
    f = to_dev(rng.uniform(0, 1, (2, *g.f_shape)))
    y = to_dev(rng.standard_normal((2, *g.p_shape)))
    pw, fw = whole.forward(f), whole.adjoint(y)
    acc = torch.zeros_like(fw)
    for j0, j1 in zip(cuts, cuts[1:]):
        blk = srt.Plan(g.column_block(j0, j1))
        assert blk.info["rows1"] == (j1 - j0) * g.n_ell
        assert torch.equal(blk.forward(f), pw[:, j0:j1])
        acc += blk.adjoint(y[:, j0:j1].contiguous())
    assert rel_l2(to_np(acc), to_np(fw)) <= 1e-6
    tol = 1e-5 if wdt == "fp32" else 5e-3
    assert rel_l2(to_np(acc[1]), orc.adjoint(o, to_np(y)[1])) <= tol


def test_column_shard_single_rank_is_the_plan(srt, orc):
    import torch
    from paper_2402_15641_gb300.sharded import ColumnShard
    g, _ = geom_pair(orc, **dict(I.sizes("srt16fd")))
    sh = ColumnShard(g)
    assert (sh.j0, sh.j1) == (0, g.n_phi)
    f = to_dev(np.random.default_rng(5).uniform(0, 1, g.f_shape))
    assert torch.equal(sh.gather(sh.forward(f)), srt.Plan(g).forward(f))
    sh.close()


def test_column_block_geometry_checks(srt, orc):
    from paper_2402_15641_gb300._lib import SrtError
    g, _ = geom_pair(orc, **dict(I.sizes("srt16fd")))
    with pytest.raises(ValueError):
        g.column_block(5, 5)
    with pytest.raises(SrtError):  # the block must lie inside the aperture
        srt.Plan(g.with_(n_phi=8, n_phi_total=g.n_phi, phi_first=g.n_phi - 4))
