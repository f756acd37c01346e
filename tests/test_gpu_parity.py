"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (stated for the workload in the benchmark spec and derived from
the arithmetic): relative L2 <= 1e-5 for FP32-stored entries, <= 5e-3 for
BF16-stored entries (FP32 accumulation in both), adjoint identity <= 1e-6
relative in FP32.  Assembly entries are compared in FP64 before rounding
(<= 1e-12 of the spacing per entry).
"""
import math

import numpy as np
import pytest

from paper_2402_15641_gb300 import inputs as I
from tests.gpu_helpers import bf16_is_rne_of, geom_pair, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

FP32_TOL, BF16_TOL, ADJ_TOL = 1e-5, 5e-3, 1e-6


@pytest.fixture(scope="module")
def srt():
    import torch
    from paper_2402_15641_gb300 import build, srt as S
    assert torch.cuda.is_available()
    build.build()
    return S


def _arcs_match(got_cols, got_vals, want: dict, scale):
    got = dict(zip(got_cols.tolist(), got_vals.tolist()))
    for k, v in want.items():
        if k in got:
            assert abs(got[k] - v) <= 1e-12 * scale, (k, got[k], v)
        else:
            assert v <= 1e-12 * scale, (k, v)  # dropped tangent touch
    for k in got:
        assert k in want, k


TINY = dict(ms=5, mz=4, dxy=0.6, dz=0.45, radius=3.0, n_phi=6, n_zs=3, n_ell=12, phi0=0.37,
            zs=(-0.7, 1.1))


@pytest.mark.parametrize("sz", [TINY, dict(I.sizes("srt32"))])
def test_assembly_entries_match_oracle_arcs(srt, orc, sz):
    g, o = geom_pair(orc, keep_f64=True, **sz)
    plan = srt.Plan(g)
    rp, col, v32, v64 = plan.export(1, f64=True)
    assert np.all(np.diff(rp) >= 0) and rp[-1] == len(col) == plan.info["nnz1"]
    for r in range(g.n_phi * g.n_ell):
        j, l = divmod(r, g.n_ell)
        seg = slice(rp[r], rp[r + 1])
        assert np.all(np.diff(col[seg]) > 0)
        _arcs_match(col[seg], v64[seg], orc.circle_arcs(o, j, l), g.dxy)
    np.testing.assert_array_equal(v32, v64.astype(np.float32))
    rp, col, v32, v64 = plan.export(2, f64=True)
    assert rp[-1] == plan.info["nnz2"]
    for r in range(g.n_zs * g.n_ell):
        h, m = divmod(r, g.n_ell)
        seg = slice(rp[r], rp[r + 1])
        assert np.all(np.diff(col[seg]) > 0)
        _arcs_match(col[seg], v64[seg], orc.semicircle_arcs(o, h, m), g.dz)
    np.testing.assert_array_equal(v32, v64.astype(np.float32))


def test_transposes_are_exact(srt, orc):
    import scipy.sparse as sp
    g, _ = geom_pair(orc, **dict(I.sizes("srt32")), weight_dtype="bf16")
    plan = srt.Plan(g)
    for a, t, shape in ((1, 3, (plan.info["rows1"], plan.info["cols1"])),
                        (2, 4, (plan.info["rows2"], plan.info["cols2"]))):
        rp, col, val, _ = plan.export(a)
        trp, tcol, tval, _ = plan.export(t)
        A = sp.csr_matrix((val, col, rp), shape=shape)
        AT = sp.csr_matrix((tval, tcol, trp), shape=shape[::-1])
        want = A.T.tocsr()
        want.sort_indices()
        np.testing.assert_array_equal(AT.indptr, want.indptr)
        np.testing.assert_array_equal(AT.indices, want.indices)
        np.testing.assert_array_equal(AT.data.view(np.uint32), want.data.view(np.uint32))


def test_bf16_entries_are_rne_of_fp64(srt, orc):
    g, _ = geom_pair(orc, **dict(I.sizes("srt32")), weight_dtype="bf16", keep_f64=True)
    plan = srt.Plan(g)
    for which in (1, 2, 3, 4):
        _, _, v, v64 = plan.export(which, f64=True)
        assert np.all(bf16_is_rne_of(v, v64))


@pytest.fixture(scope="module")
def c0(orc):
    sz = dict(I.sizes("srt32"))
    _, o = geom_pair(orc, **sz)
    f = I.phantom("srt32")
    g = I.probe("srt32")
    return sz, f, g, orc.forward(o, f), orc.adjoint(o, g)


@pytest.mark.parametrize("wdt,tol", [("fp32", FP32_TOL), ("bf16", BF16_TOL)])
def test_forward_adjoint_c0(srt, orc, c0, wdt, tol):
    sz, f, y, pf, fa = c0
    g, _ = geom_pair(orc, weight_dtype=wdt, **sz)
    plan = srt.Plan(g)
    p_gpu = to_np(plan.forward(to_dev(f)))
    f_gpu = to_np(plan.adjoint(to_dev(y)))
    print(f"PARITY srt32 {wdt}: forward rel-L2 {rel_l2(p_gpu, pf):.3e}, "
          f"adjoint rel-L2 {rel_l2(f_gpu, fa):.3e}")
    assert rel_l2(p_gpu, pf) <= tol
    assert rel_l2(f_gpu, fa) <= tol
    if wdt == "fp32":  # the BF16 error is large enough to be seen at all
        return
    assert rel_l2(p_gpu, pf) > 1e-5


@pytest.mark.parametrize("name", ["srt32", "srt16fd"])
def test_adjoint_identity_on_gpu(srt, orc, name):
    sz = dict(I.sizes(name))
    g, _ = geom_pair(orc, **sz)
    plan = srt.Plan(g)
    f = to_dev(I.phantom(name))
    y = to_dev(I.probe(name))
    af = plan.forward(f)
    aty = plan.adjoint(y)
    lhs = srt.dot_f64(af, y)
    rhs = srt.dot_f64(f, aty)
    nrm = math.sqrt(srt.dot_f64(af, af) * srt.dot_f64(y, y))
    print(f"PARITY {name} fp32: adjoint identity {abs(lhs - rhs) / nrm:.3e} "
          f"(/|<Af,g>| {abs(lhs - rhs) / abs(lhs):.3e})")
    assert abs(lhs - rhs) / nrm <= ADJ_TOL
    # the FP64 device dot agrees with a host FP64 dot of the same floats
    assert lhs == pytest.approx(float(np.dot(to_np(af).ravel(), to_np(y).ravel())), rel=1e-12)


RAGGED = [
    dict(ms=7, mz=5, dxy=0.5, dz=0.37, radius=6.0, n_phi=6, n_zs=3, n_ell=13, phi0=0.2),
    dict(ms=9, mz=3, dxy=0.3, dz=0.8, radius=2.5, n_phi=5, n_zs=7, n_ell=31, zs=(-2.0, 1.5)),
    dict(ms=16, mz=12, dxy=0.5, dz=0.5, radius=12.0, n_phi=32, n_zs=16, n_ell=48),
    dict(ms=1, mz=1, dxy=1.0, dz=1.0, radius=2.0, n_phi=1, n_zs=1, n_ell=2),
    dict(ms=20, mz=36, dxy=0.4, dz=0.25, radius=9.0, n_phi=12, n_zs=40, n_ell=57, phi0=1.1),
]


@pytest.mark.parametrize("sz", RAGGED)
@pytest.mark.parametrize("batch", [1, 3])
def test_ragged_geometries_full(srt, orc, sz, batch):
    g, o = geom_pair(orc, **sz)
    plan = srt.Plan(g)
    rng = np.random.default_rng(7)
    f = rng.uniform(0, 1, (batch, *g.f_shape))
    y = rng.standard_normal((batch, *g.p_shape))
    pf = np.stack([orc.forward(o, f[b]) for b in range(batch)])
    fa = np.stack([orc.adjoint(o, y[b]) for b in range(batch)])
    assert rel_l2(to_np(plan.forward(to_dev(f))), pf) <= FP32_TOL
    assert rel_l2(to_np(plan.adjoint(to_dev(y))), fa) <= FP32_TOL


@pytest.mark.parametrize("mode", [{}, dict(a1_rotation=True), dict(csr_only=True),
                                  dict(rho_linear=True)])
def test_tangent_geometry_entries_and_transforms(srt, orc, mode):
    """Circles that touch a pixel line from either side, or the box from
    outside (the tangent geometry of the oracle pins): every A1 and A2 entry
    against the oracle's arcs, and forward / adjoint against the oracle."""
    from tests.test_oracle_pins import TANGENT
    g, o = geom_pair(orc, keep_f64=True, **TANGENT, **mode)
    plan = srt.Plan(g)
    rp, col, _, v64 = plan.export(1, f64=True)
    for r in range(g.n_phi * g.n_ell):
        j, l = divmod(r, g.n_ell)
        _arcs_match(col[rp[r]:rp[r + 1]], v64[rp[r]:rp[r + 1]], orc.circle_arcs(o, j, l), g.dxy)
    # radius 1.5 touches the box from outside: no entry at all
    for j in range(g.n_phi):
        assert rp[j * g.n_ell + 1] == rp[j * g.n_ell]
    rp, col, _, v64 = plan.export(2, f64=True)
    for r in range(g.n_zs * g.n_ell):
        h, m = divmod(r, g.n_ell)
        _arcs_match(col[rp[r]:rp[r + 1]], v64[rp[r]:rp[r + 1]], orc.semicircle_arcs(o, h, m),
                    g.dz)
    rng = np.random.default_rng(17)
    f = rng.uniform(0, 1, (2, *g.f_shape))
    y = rng.standard_normal((2, *g.p_shape))
    pf = np.stack([orc.forward(o, f[b]) for b in range(2)])
    fa = np.stack([orc.adjoint(o, y[b]) for b in range(2)])
    assert rel_l2(to_np(plan.forward(to_dev(f))), pf) <= FP32_TOL
    assert rel_l2(to_np(plan.adjoint(to_dev(y))), fa) <= FP32_TOL


def test_fd16_full_and_batched_bitwise(srt, orc):
    import torch
    sz = dict(I.sizes("srt16fd"))
    g, o = geom_pair(orc, **sz)
    plan = srt.Plan(g)
    rng = np.random.default_rng(8)
    f = rng.uniform(0, 1, (4, *g.f_shape))
    y = rng.standard_normal((4, *g.p_shape))
    pb = plan.forward(to_dev(f))
    ab = plan.adjoint(to_dev(y))
    for b in range(4):
        assert torch.equal(plan.forward(to_dev(f[b])), pb[b])
        assert torch.equal(plan.adjoint(to_dev(y[b])), ab[b])
    assert rel_l2(to_np(pb[2]), orc.forward(o, f[2])) <= FP32_TOL
    assert rel_l2(to_np(ab[1]), orc.adjoint(o, y[1])) <= FP32_TOL


@pytest.mark.parametrize("wdt", ["fp32", "bf16"])
def test_batch16_bitwise_per_volume(srt, orc, wdt):
    """Batch 16 at 32^3: the second product's dense width is 16 x 64 = 1024
    columns (the 512-column kernel), the first product runs 16 volumes per
    launch; every batch item equals the single-volume result bitwise."""
    import torch
    g, o = geom_pair(orc, weight_dtype=wdt, **dict(I.sizes("srt32")))
    plan = srt.Plan(g)
    rng = np.random.default_rng(12)
    f = rng.uniform(0, 1, (16, *g.f_shape))
    y = rng.standard_normal((16, *g.p_shape))
    pb = plan.forward(to_dev(f))
    ab = plan.adjoint(to_dev(y))
    for b in (0, 5, 15):
        assert torch.equal(plan.forward(to_dev(f[b])), pb[b])
        assert torch.equal(plan.adjoint(to_dev(y[b])), ab[b])
    tol = FP32_TOL if wdt == "fp32" else BF16_TOL
    assert rel_l2(to_np(pb[15]), orc.forward(o, f[15])) <= tol
    assert rel_l2(to_np(ab[7]), orc.adjoint(o, y[7])) <= tol


@pytest.mark.parametrize("sz,rot", [(RAGGED[0], False), (RAGGED[3], False),
                                    (dict(I.sizes("srt32")), False), (dict(I.sizes("srt32")), True)])
def test_host_calls_chunked_equal_device(srt, orc, sz, rot):
    """The host-buffer calls compute the last product in row ranges and copy
    each back while the next is computed: results equal the device path
    bitwise, also when there are fewer rings or pixel columns than chunks and
    when A1^T comes from the stored quarter of A1."""
    import torch
    g, _ = geom_pair(orc, a1_rotation=rot, **sz)
    plan = srt.Plan(g)
    rng = np.random.default_rng(13)
    f = torch.from_numpy(rng.uniform(0, 1, (2, *g.f_shape)).astype(np.float32)).pin_memory()
    y = torch.from_numpy(rng.standard_normal((2, *g.p_shape)).astype(np.float32)).pin_memory()
    p_h = torch.full((2, *g.p_shape), float("nan"), dtype=torch.float32).pin_memory()
    f_h = torch.full((2, *g.f_shape), float("nan"), dtype=torch.float32).pin_memory()
    plan.forward_host(f, p_h)
    plan.adjoint_host(y, f_h)
    assert torch.equal(p_h, plan.forward(f.cuda()).cpu())
    assert torch.equal(f_h, plan.adjoint(y.cuda()).cpu())


def test_host_buffer_variants_equal_device(srt, orc):
    import torch
    g, _ = geom_pair(orc, **dict(I.sizes("srt16fd")))
    plan = srt.Plan(g)
    rng = np.random.default_rng(9)
    f = torch.from_numpy(rng.uniform(0, 1, (2, *g.f_shape)).astype(np.float32)).pin_memory()
    y = torch.from_numpy(rng.standard_normal((2, *g.p_shape)).astype(np.float32)).pin_memory()
    p_h = torch.empty((2, *g.p_shape), dtype=torch.float32).pin_memory()
    f_h = torch.empty((2, *g.f_shape), dtype=torch.float32).pin_memory()
    plan.forward_host(f, p_h)
    plan.adjoint_host(y, f_h)
    assert torch.equal(p_h, plan.forward(f.cuda()).cpu())
    assert torch.equal(f_h, plan.adjoint(y.cuda()).cpu())


def test_workspace_and_argument_errors(srt, orc):
    import torch
    from paper_2402_15641_gb300._lib import SrtError, SRT_ERR_WORKSPACE, SRT_ERR_ARG
    g, _ = geom_pair(orc, **dict(I.sizes("srt16fd")))
    plan = srt.Plan(g)
    f = torch.zeros(g.f_shape, device="cuda")
    small = torch.empty(plan.workspace_bytes(1) - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(SrtError) as e:
        plan.forward(f, workspace=small)
    assert e.value.code == SRT_ERR_WORKSPACE
    big = torch.empty(plan.workspace_bytes(1) + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(SrtError) as e:
        plan.forward(f, workspace=big[4:])  # misaligned
    assert e.value.code == SRT_ERR_WORKSPACE
    with pytest.raises(SrtError) as e:  # batch 2 does not fit a batch-1 workspace
        plan.forward(torch.zeros((2, *g.f_shape), device="cuda"), workspace=plan.workspace(1))
    assert e.value.code == SRT_ERR_WORKSPACE
    raw = torch.zeros(g.ms * g.ms * g.mz + 4, device="cuda")
    ws = plan.workspace(1)
    rc = plan._lib.srt_forward(plan._h, raw[1:].data_ptr(), raw.data_ptr(), 1, ws.data_ptr(),
                               ws.numel(), None)  # misaligned volume pointer
    assert rc == SRT_ERR_ARG


TOEP = [dict(I.sizes("srt32")), dict(I.sizes("srt16fd")),
        dict(ms=9, mz=7, dxy=0.4, dz=0.3, radius=5.0, n_phi=5, n_zs=11, n_ell=23, phi0=0.4,
             zs=(-1.65 - 0.57, -2.22 + 3.3)),              # 11 rings spaced dz, offset
        dict(ms=9, mz=7, dxy=0.4, dz=0.3, radius=5.0, n_phi=5, n_zs=7, n_ell=23, phi0=0.4),
        dict(ms=12, mz=40, dxy=0.5, dz=0.2, radius=9.0, n_phi=6, n_zs=40, n_ell=19)]


@pytest.mark.parametrize("sz", TOEP)
@pytest.mark.parametrize("wdt", ["fp32", "bf16"])
def test_toeplitz_second_stage(srt, orc, sz, wdt):
    """With the rings at the slab centres A2 and A2^T are applied from the
    taps of the master tensor T (A2 = T shifted per ring) and never stored:
    the A2 they stand for (exported by expanding T) has the pattern of the
    directly assembled one and its entries to FP64 rounding, the taps alone
    take less memory than A2 and A2^T (the 2 x 2 tile records add some, which
    on grids this small can outweigh what the taps save), and the transforms
    match the CSR plan and the oracle (dense widths 5 and 15 take the
    row-per-warp scalar kernel)."""
    g, o = geom_pair(orc, weight_dtype=wdt, **sz)
    a = srt.Plan(g)
    b = srt.Plan(g.with_(csr_only=True))
    assert a.info["a2_taps"] == 1 and a.info["n_taps"] > 0 and b.info["a2_taps"] == 0
    assert a.info["nnz2"] == b.info["nnz2"]
    assert srt.Plan(g.with_(rowwise=True)).info["device_bytes"] < b.info["device_bytes"]
    for which in (2, 4):
        ra, ca, va, _ = a.export(which)
        rb, cb, vb, _ = b.export(which)
        np.testing.assert_array_equal(ra, rb)
        np.testing.assert_array_equal(ca, cb)
        assert rel_l2(va, vb) <= 1e-6  # T is computed once per offset, rows per ring
    rng = np.random.default_rng(12)
    for batch in (1, 3):
        f = to_dev(rng.uniform(0, 1, (batch, *g.f_shape)))
        y = to_dev(rng.standard_normal((batch, *g.p_shape)))
        assert rel_l2(to_np(a.forward(f)), to_np(b.forward(f))) <= 1e-5
        assert rel_l2(to_np(a.adjoint(y)), to_np(b.adjoint(y))) <= 1e-5
    tol = FP32_TOL if wdt == "fp32" else BF16_TOL
    fv, yv = to_np(f)[-1], to_np(y)[-1]
    assert rel_l2(to_np(a.forward(f))[-1], orc.forward(o, fv)) <= tol
    assert rel_l2(to_np(a.adjoint(y))[-1], orc.adjoint(o, yv)) <= tol
    lhs = srt.dot_f64(a.forward(f), y)
    rhs = srt.dot_f64(f, a.adjoint(y))
    nrm = math.sqrt(srt.dot_f64(a.forward(f), a.forward(f)) * srt.dot_f64(y, y))
    assert abs(lhs - rhs) / nrm <= ADJ_TOL


SPACED = [  # rings spaced like the slabs (spacing dz = 0.5), off the slab centres
    dict(ms=10, mz=8, dxy=0.5, dz=0.5, radius=6.0, n_phi=8, n_zs=8, n_ell=21,
         zs=(-2.0 + 0.15, 2.0 + 0.15)),                     # shifted by 0.3 slab
    dict(ms=10, mz=8, dxy=0.5, dz=0.5, radius=6.0, n_phi=8, n_zs=13, n_ell=21,
         zs=(-3.2, 3.3)),                                   # more rings, past both ends
    dict(ms=10, mz=8, dxy=0.5, dz=0.5, radius=6.0, n_phi=8, n_zs=3, n_ell=21,
         zs=(-0.725, 0.775)),                               # fewer rings, off centre
]


@pytest.mark.parametrize("sz", SPACED)
def test_rings_spaced_like_slabs_use_taps(srt, orc, sz):
    """Rings spaced like the slabs, whatever their number and offset, make A2
    Toeplitz in the slab offset: the plan applies it from the taps of a
    master tensor assembled for a ring at that offset, and matches the
    oracle and the CSR plan."""
    g, o = geom_pair(orc, **sz)
    plan = srt.Plan(g)
    csr = srt.Plan(g.with_(csr_only=True))
    assert plan.info["a2_taps"] == 1 and plan.info["n_taps"] > 0
    assert plan.info["nnz2"] == csr.info["nnz2"]
    rng = np.random.default_rng(31)
    f = rng.uniform(0, 1, g.f_shape)
    y = rng.standard_normal(g.p_shape)
    assert rel_l2(to_np(plan.forward(to_dev(f))), orc.forward(o, f)) <= FP32_TOL
    assert rel_l2(to_np(plan.adjoint(to_dev(y))), orc.adjoint(o, y)) <= FP32_TOL
    for which in (2, 4):
        ra, ca, va, _ = plan.export(which)
        rb, cb, vb, _ = csr.export(which)
        np.testing.assert_array_equal(ra, rb)
        np.testing.assert_array_equal(ca, cb)
        assert rel_l2(va, vb) <= 1e-6


def test_rings_spaced_unlike_slabs_use_csr(srt, orc):
    g, o = geom_pair(orc, ms=10, mz=8, dxy=0.5, dz=0.5, radius=6.0, n_phi=8, n_zs=8, n_ell=21,
                     zs=(-2.0, 2.2))                        # spacing 0.525
    plan = srt.Plan(g)
    assert plan.info["a2_taps"] == 0 and plan.info["n_taps"] == 0
    f = np.random.default_rng(32).uniform(0, 1, g.f_shape)
    assert rel_l2(to_np(plan.forward(to_dev(f))), orc.forward(o, f)) <= FP32_TOL


def test_plan_info_and_timing(srt, orc):
    import torch
    g, _ = geom_pair(orc, **dict(I.sizes("srt32")))
    plan = srt.Plan(g)
    inf = plan.info
    assert inf["rows1"] == 64 * 96 and inf["cols1"] == 32 * 32
    assert inf["rows2"] == 32 * 96 and inf["cols2"] == 96 * 32
    assert inf["nnz1"] > 0 and inf["nnz2"] > 0 and inf["device_bytes"] > 0
    plan.set_timing(True)
    f = to_dev(I.phantom("srt32"))
    plan.forward(f)
    t = plan.stage_times(0)
    assert len(t) == 4 and all(x >= 0 for x in t)
    from paper_2402_15641_gb300._lib import SrtError
    with pytest.raises(SrtError):
        plan.stage_times(1)
    assert plan.launches_per_call(0) == 4 and plan.launches_per_call(1) == 4
    # A2 / A2^T tiles writing the reshaped layouts themselves, and A1 (8-fold)
    # writing Y1': 2 launches forward, 3 adjoint
    s = srt.Plan(g.with_(fuse_reshapes=True))
    assert s.launches_per_call(0) == 2 and s.launches_per_call(1) == 3
    assert inf["a2_taps"] == 1  # rings at the slab centres: A2 from the taps
    c = srt.Plan(g.with_(csr_only=True))
    assert c.info["a2_taps"] == 0 and c.info["n_taps"] == 0
    assert c.launches_per_call(0) == 4 and c.launches_per_call(1) == 4
    torch.cuda.synchronize()


ROT = [dict(I.sizes("srt32")),
       dict(ms=7, mz=5, dxy=0.5, dz=0.37, radius=6.0, n_phi=8, n_zs=3, n_ell=13, phi0=0.2),
       dict(ms=12, mz=9, dxy=0.4, dz=0.3, radius=6.0, n_phi=12, n_zs=5, n_ell=21, zs=(-1.0, 1.2)),
       dict(ms=10, mz=8, dxy=0.5, dz=0.5, radius=6.0, n_phi=16, n_zs=8, n_ell=13,
            zs=(-2.0 + 0.15, 2.0 + 0.15)),                 # 8-fold, odd radius count
       dict(ms=6, mz=4, dxy=0.5, dz=0.5, radius=4.0, n_phi=8, n_zs=4, n_ell=9)]  # q = 2


def _sym_form(sz, **form):
    """The symmetry form the plan should choose (srt.h, SRT_A1_FULL)."""
    if form.get("a1_full") or sz["n_phi"] % 4:
        return 0
    tiles = sz["ms"] % 2 == 0 and sz["mz"] % 4 == 0 and not form.get("rowwise")
    eight = tiles and sz["n_phi"] % 8 == 0 and sz.get("phi0", 0.0) == 0.0
    return 2 if eight and not form.get("a1_rotation") else 1


@pytest.mark.parametrize("sz", ROT)
@pytest.mark.parametrize("form", [{}, dict(a1_rotation=True), dict(rowwise=True)])
@pytest.mark.parametrize("wdt", ["fp32", "bf16"])
def test_a1_by_symmetry(srt, orc, sz, form, wdt):
    """By default the plan stores A1 for a fundamental set of sensor columns:
    the first n_phi/8 + 1 under quarter turns and the diagonal mirror (the
    8-fold form; n_phi % 8 == 0, phi0 = 0, ms even, mz % 4 == 0), else the
    first n_phi/4 under quarter turns.  The full A1 and A1^T it stands for
    (exported) have the pattern of the directly assembled ones and their FP64
    entries to rounding, and the transforms (tile and row-per-warp kernels)
    match the fully stored plan and the oracle (odd ms, a phase phi0, rings
    off the slab centres, an odd radius count, two stored columns that are
    both fixed by a mirror, BF16, batch 2)."""
    g, o = geom_pair(orc, weight_dtype=wdt, keep_f64=True, **sz)
    a = srt.Plan(g.with_(**form))
    b = srt.Plan(g.with_(a1_full=True, rowwise=True))
    assert a.info["a1_rot"] == _sym_form(sz, **form) and b.info["a1_rot"] == 0
    assert a.info["rows1"] == b.info["rows1"] and a.info["nnz1"] == b.info["nnz1"]
    if a.info["a1_rot"]:
        assert a.info["device_bytes"] < srt.Plan(g.with_(a1_full=True, **form)).info["device_bytes"]
    for which in (1, 3):
        ra, ca, va, da = a.export(which, f64=True)
        rb, cb, vb, db = b.export(which, f64=True)
        np.testing.assert_array_equal(ra, rb)
        np.testing.assert_array_equal(ca, cb)
        np.testing.assert_allclose(da, db, rtol=1e-12, atol=1e-12 * sz["dxy"])
        assert rel_l2(va, vb) <= 1e-6
    rng = np.random.default_rng(14)
    f = to_dev(rng.uniform(0, 1, (2, *g.f_shape)))
    y = to_dev(rng.standard_normal((2, *g.p_shape)))
    assert rel_l2(to_np(a.forward(f)), to_np(b.forward(f))) <= 1e-5
    assert rel_l2(to_np(a.adjoint(y)), to_np(b.adjoint(y))) <= 1e-5
    tol = FP32_TOL if wdt == "fp32" else BF16_TOL
    assert rel_l2(to_np(a.forward(f))[1], orc.forward(o, to_np(f)[1])) <= tol
    assert rel_l2(to_np(a.adjoint(y))[0], orc.adjoint(o, to_np(y)[0])) <= tol
    lhs, rhs = srt.dot_f64(a.forward(f), y), srt.dot_f64(f, a.adjoint(y))
    nrm = math.sqrt(srt.dot_f64(a.forward(f), a.forward(f)) * srt.dot_f64(y, y))
    assert abs(lhs - rhs) / nrm <= ADJ_TOL


@pytest.mark.parametrize("sz", [dict(I.sizes("srt32")), ROT[3], ROT[4],
                                dict(ms=14, mz=12, dxy=0.4, dz=0.4, radius=6.0, n_phi=6, n_zs=7,
                                     n_ell=18, phi0=0.3)])
@pytest.mark.parametrize("wdt", ["fp32", "bf16"])
@pytest.mark.parametrize("batch", [1, 3])
def test_a1_tiles_equal_rowwise(srt, orc, sz, wdt, batch):
    """With A1 stored for every column, the 2 x 2 pixel A1^T tiles sum every
    pixel's entries in the CSR order of A1^T (ascending (j, l)) and add only
    zeros besides, and the A2 tiles those of the taps: forward and adjoint
    equal the row-per-warp kernels bitwise (after +0.0, which equates the
    signs of zero sums)."""
    import torch
    g, _ = geom_pair(orc, weight_dtype=wdt, a1_full=True, **sz)
    a, b = srt.Plan(g), srt.Plan(g.with_(rowwise=True))
    rng = np.random.default_rng(33)
    f = to_dev(rng.uniform(0, 1, (batch, *g.f_shape)))
    y = to_dev(rng.standard_normal((batch, *g.p_shape)))
    assert torch.equal(a.forward(f) + 0.0, b.forward(f) + 0.0)
    assert torch.equal(a.adjoint(y) + 0.0, b.adjoint(y) + 0.0)


def test_concurrent_calls_on_one_plan(srt, orc):
    """The plan is immutable: forward and adjoint calls on different streams
    (each with its own workspace), and from two host threads, overlap on the
    device and give bitwise the results of sequential calls."""
    import threading
    import torch
    g, _ = geom_pair(orc, **dict(I.sizes("srt32")))
    plan = srt.Plan(g)
    rng = np.random.default_rng(15)
    fs = [to_dev(rng.uniform(0, 1, g.f_shape)) for _ in range(4)]
    ys = [to_dev(rng.standard_normal(g.p_shape)) for _ in range(4)]
    want_p = [plan.forward(f) for f in fs]
    want_a = [plan.adjoint(y) for y in ys]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(4)]
    nb = plan.workspace_bytes(1)
    wss = [torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(4)]
    outs_p = [torch.empty_like(w) for w in want_p]
    outs_a = [torch.empty_like(w) for w in want_a]
    for rep in range(3):
        for i, st in enumerate(streams):
            with torch.cuda.stream(st):
                plan.forward(fs[i], out=outs_p[i], workspace=wss[i], stream=st)
                plan.adjoint(ys[i], out=outs_a[i], workspace=wss[i], stream=st)
        torch.cuda.synchronize()
        for i in range(4):
            assert torch.equal(outs_p[i], want_p[i]) and torch.equal(outs_a[i], want_a[i])
    errors = []

    def worker(i):
        try:
            st = torch.cuda.Stream()
            ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
            with torch.cuda.stream(st):
                for _ in range(5):
                    p = torch.empty_like(want_p[i])
                    plan.forward(fs[i], out=p, workspace=ws, stream=st)
                    st.synchronize()
                    if not torch.equal(p, want_p[i]):
                        errors.append(i)
        except Exception as exc:  # reported below
            errors.append(repr(exc))

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors


TILE_GEOMS = [dict(I.sizes("srt32")), dict(I.sizes("srt16fd")),
              dict(ms=9, mz=7, dxy=0.4, dz=0.3, radius=5.0, n_phi=8, n_zs=11, n_ell=23, phi0=0.4,
                   zs=(-1.65 - 0.57, -2.22 + 3.3)),             # 11 rings spaced dz, offset
              dict(ms=8, mz=9, dxy=0.5, dz=0.4, radius=6.0, n_phi=12, n_zs=5, n_ell=17,
                   zs=(-1.0, 1.0))]                                  # 5 rings spaced dz


@pytest.mark.parametrize("sz", TILE_GEOMS)
@pytest.mark.parametrize("wdt", ["fp32", "bf16"])
@pytest.mark.parametrize("batch", [1, 3])
def test_tiles_equal_rowwise_taps(srt, orc, sz, wdt, batch):
    """The 2 x 2 row tiles sum every row in the order of the row-per-warp
    taps kernel and add only zeros besides, so forward and adjoint agree
    bitwise (after +0.0, which equates the signs of zero sums; A1 stored for
    every column in both plans, where its tiles are bitwise the CSR rows
    too); odd ring, slab and radius counts leave half-empty tiles at the
    edges."""
    import torch
    g, o = geom_pair(orc, weight_dtype=wdt, a1_full=True, **sz)
    gr, _ = geom_pair(orc, weight_dtype=wdt, a1_full=True, rowwise=True, **sz)
    plan, ref = srt.Plan(g), srt.Plan(gr)
    assert plan.info["a2_taps"] == 1
    rng = np.random.default_rng(31)
    f = to_dev(rng.uniform(0, 1, (batch, *g.f_shape)))
    y = to_dev(rng.standard_normal((batch, *g.p_shape)))
    assert torch.equal(plan.forward(f) + 0.0, ref.forward(f) + 0.0)
    assert torch.equal(plan.adjoint(y) + 0.0, ref.adjoint(y) + 0.0)
    tol = FP32_TOL if wdt == "fp32" else BF16_TOL
    assert rel_l2(to_np(plan.forward(f)[0]), orc.forward(o, to_np(f)[0])) <= tol
    assert rel_l2(to_np(plan.adjoint(y)[-1]), orc.adjoint(o, to_np(y)[-1])) <= tol


def _pair_records(orc, sz):
    """Records per radius pair of the 2 x 2 tiles of A2 (pairs of radii m)
    and A2^T (pairs of radius bins l), counted from the oracle's semicircle
    cells.  With the rings at the slab centres, T's taps are one ring's
    semicircle cells at every ring-to-slab offset d, which the middle ring
    of a volume 2 mz - 1 slabs tall sees.  A forward record is a distinct
    (l, d + i) and an adjoint record a distinct (i - d, m), i = 0, 1 the
    tile's two rings or slabs."""
    _, tall = geom_pair(orc, **dict(sz, mz=2 * sz["mz"] - 1, n_zs=2 * sz["n_zs"] - 1))
    h, n = sz["n_zs"] - 1, sz["n_ell"]
    cells = [{(c // tall.mz, c % tall.mz - h) for c, w in orc.semicircle_arcs(tall, h, m).items()
              if w != 0.0} for m in range(n)]
    by_l = {}
    for m, cs in enumerate(cells):
        for l, d in cs:
            by_l.setdefault(l, []).append((m, d))
    fwd, adj = [], []
    for p in range(0, n, 2):
        two = [q for q in (p, p + 1) if q < n]
        fwd.append(len({(l, d + i) for m in two for l, d in cells[m] for i in (0, 1)}))
        adj.append(len({(i - d, m) for l in two for m, d in by_l.get(l, ()) for i in (0, 1)}))
    return fwd, adj


@pytest.mark.parametrize("name", ["srt16fd", "srt32", "srt128"])
def test_tile_records_and_block_order(srt, orc, name):
    """The plan's tile records are the distinct (offset, row) pairs of T's
    taps per radius pair, and its blocks start at the end of the radius range
    whose first or last eighth of the pairs holds more records: A2's records
    grow with the radius up to the largest ring-to-slab offset, so its
    blocks run from the last radius pair down (bit 0 of tile_order); A2^T's
    fall from the first radius bins, so its blocks run upwards (bit 1
    clear).  test_tiles_equal_rowwise_taps checks the results in that order
    (srt32, srt16fd) bitwise."""
    sz = dict(I.sizes(name))
    g, _ = geom_pair(orc, **sz)
    info = srt.Plan(g).info
    fwd, adj = _pair_records(orc, sz)
    assert info["tile_records"][:2] == [sum(fwd), sum(adj)]

    def heavier_last(r):
        e = max(1, len(r) // 8)
        return sum(r[-e:]) > sum(r[:e])

    assert info["tile_order"] == (1 if heavier_last(fwd) else 0) | (2 if heavier_last(adj) else 0)
    assert info["tile_order"] == 1
    gr, _ = geom_pair(orc, rowwise=True, **sz)
    assert srt.Plan(gr).info["tile_order"] == 0
