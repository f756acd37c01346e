"""The column-sharded transform's host logic on CPU gloo ranks.

paper_2402_15641_gb300/sharded.py splits the sensor columns over ranks: the
forward needs no exchange, the adjoint one all-reduce of the volume (Sec. 2:
one A2 serves every column).  Here each rank's block operator is the FP64
oracle restricted to the block's shells (forward on those shells, adjoint of
data supported on them), so the partition, the all-gather of p and the
all-reduce of the adjoint run exactly as on GPUs, and the results must equal
the single-rank oracle transform."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SZ = dict(ms=6, mz=5, dxy=0.5, dz=0.5, radius=4.0, n_phi=8, n_zs=5, n_ell=10)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleBlock:
    """The oracle on the shells of columns [j0, j1): forward values of those
    shells, and the adjoint of data that is zero outside them."""

    def __init__(self, O, g, j0, j1):
        self.O, self.g = O, g
        jj, hh, mm = np.meshgrid(np.arange(j0, j1), np.arange(g.n_zs), np.arange(g.n_ell),
                                 indexing="ij")
        self.shells = np.stack([jj.ravel(), hh.ravel(), mm.ravel()], axis=1)
        self.shape = (j1 - j0, g.n_zs, g.n_ell)

    def forward(self, f):
        v = self.O.forward_shells(self.g, f.numpy(), self.shells)
        return torch.from_numpy(v.reshape(self.shape))

    def adjoint(self, p):
        return torch.from_numpy(self.O.adjoint_shells(self.g, self.shells, p.numpy().ravel()))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2402_15641_gb300.sharded import ColumnShard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = O.OracleGeometry.default(**SZ)
        sh = ColumnShard(g, make_op=lambda gg, j0, j1: OracleBlock(O, gg, j0, j1))
        rng = np.random.default_rng(3)
        f = torch.from_numpy(rng.uniform(0, 1, g.f_shape))
        p = torch.from_numpy(rng.standard_normal(g.p_shape))
        pl = sh.forward(f)
        p_all = sh.gather(pl)
        fa = sh.adjoint(p[sh.j0:sh.j1].contiguous())
        q.put((rank, sh.j0, sh.j1, p_all.numpy(), fa.numpy()))
    finally:
        dist.destroy_process_group()


def test_column_range_partition():
    from paper_2402_15641_gb300.sharded import column_range
    for n in (1, 2, 7, 8, 256):
        for world in range(1, min(n, 9) + 1):
            blocks = [column_range(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(b[1] == c[0] for b, c in zip(blocks, blocks[1:]))
            sizes = [b[1] - b[0] for b in blocks]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        column_range(3, 0, 4)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_transform_on_gloo_ranks_matches_single_rank(orc, world):
    g = orc.OracleGeometry.default(**SZ)
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 1, g.f_shape)
    p = rng.standard_normal(g.p_shape)
    want_p, want_f = orc.forward(g, f), orc.adjoint(g, p)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = sorted((q.get(timeout=180) for _ in range(world)), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert [(j0, j1) for _, j0, j1, _, _ in got] == [
        __import__("paper_2402_15641_gb300.sharded", fromlist=["x"]).column_range(SZ["n_phi"], r,
                                                                                    world)
        for r in range(world)]
    for rank, j0, j1, p_all, fa in got:
        # the forward of a block is the whole forward's rows (the same shell walks)
        np.testing.assert_array_equal(p_all, want_p)
        # the adjoint sums the ranks' shares: equal up to FP64 summation order
        assert np.linalg.norm(fa - want_f) <= 1e-13 * np.linalg.norm(want_f)


def test_single_rank_shard_is_the_whole_aperture(orc):
    from paper_2402_15641_gb300.sharded import ColumnShard
    g = orc.OracleGeometry.default(**SZ)
    sh = ColumnShard(g, make_op=lambda gg, j0, j1: OracleBlock(orc, gg, j0, j1))
    assert (sh.j0, sh.j1, sh.world) == (0, SZ["n_phi"], 1)
    f = torch.from_numpy(np.random.default_rng(4).uniform(0, 1, g.f_shape))
    np.testing.assert_array_equal(sh.gather(sh.forward(f)).numpy(), orc.forward(g, f.numpy()))
