"""GPU parity at the full workload sizes, on seeded samples the oracle can
evaluate one by one (forward: sampled shells; adjoint: sampled voxels via the
oracle's per-voxel weights), plus the adjoint identity on the whole output.

srt256 runs in the launch configuration the benchmark times (batch 1, FP32
entries) and in its BF16 form, on a phantom that is zero outside the central
64^3 voxels (the full 256^3 oracle is out of reach: ~5e12 weight
evaluations)."""
import math

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


def _samples(g, n_shells, n_vox, seed, crop=None):
    rng = np.random.default_rng(seed)
    sh = np.stack([rng.integers(0, g.n_phi, n_shells), rng.integers(0, g.n_zs, n_shells),
                   rng.integers(0, g.n_ell, n_shells)], axis=1)
    if crop is None:
        vx = np.stack([rng.integers(0, g.ms, n_vox), rng.integers(0, g.ms, n_vox),
                       rng.integers(0, g.mz, n_vox)], axis=1)
    else:
        a, b = (g.ms - crop) // 2, (g.mz - crop) // 2
        vx = np.stack([rng.integers(a, a + crop, n_vox), rng.integers(a, a + crop, n_vox),
                       rng.integers(b, b + crop, n_vox)], axis=1)
    return sh, vx


def _check(srt, orc, plan, o, f, y, sh, vx, tol):
    p_gpu = to_np(plan.forward(to_dev(f)))
    a_gpu = to_np(plan.adjoint(to_dev(y)))
    want_p = orc.forward_shells(o, f, sh)
    got_p = p_gpu[sh[:, 0], sh[:, 1], sh[:, 2]]
    want_a = orc.adjoint_voxels(o, y, vx)
    got_a = a_gpu[vx[:, 0], vx[:, 1], vx[:, 2]]
    e_p, e_a = rel_l2(got_p, want_p), rel_l2(got_a, want_a)
    assert e_p <= tol, e_p
    assert e_a <= tol, e_a
    return e_p, e_a


def test_srt128_sampled(srt, orc):
    sz = dict(I.sizes("srt128"))
    g, o = geom_pair(orc, **sz)
    plan = srt.Plan(g)
    f = I.phantom("srt128")
    y = I.probe("srt128")
    sh, vx = _samples(g, 2048, 48, 31)
    e_p, e_a = _check(srt, orc, plan, o, f, y, sh, vx, 1e-5)
    print(f"PARITY srt128 fp32 (2048 shells, 48 voxels): forward rel-L2 {e_p:.3e}, "
          f"adjoint rel-L2 {e_a:.3e}")
    fd, yd = to_dev(f), to_dev(y)
    af, aty = plan.forward(fd), plan.adjoint(yd)
    lhs, rhs = srt.dot_f64(af, yd), srt.dot_f64(fd, aty)
    assert abs(lhs - rhs) / math.sqrt(srt.dot_f64(af, af) * srt.dot_f64(yd, yd)) <= 1e-6


@pytest.fixture(scope="module")
def srt256_inputs():
    return I.crop_phantom("srt256", 64), I.probe("srt256")


@pytest.mark.parametrize("wdt,tol,csr,lin", [("fp32", 1e-5, False, False),
                                             ("bf16", 5e-3, False, False),
                                             ("fp32", 1e-5, True, False),
                                             ("fp32", 1e-5, False, True)])
def test_srt256_crop_sampled(srt, orc, srt256_inputs, wdt, tol, csr, lin):
    """The benchmark's configuration (A2 from the Toeplitz taps), the CSR
    form of A2 and the piecewise-linear intermediate, against the oracle on
    samples of the 64^3-crop workload."""
    sz = dict(I.sizes("srt256"))
    g, o = geom_pair(orc, weight_dtype=wdt, csr_only=csr, rho_linear=lin, **sz)
    plan = srt.Plan(g)
    f, y = srt256_inputs
    sh, vx = _samples(g, 4096, 96, 41, crop=64)
    e_p, e_a = _check(srt, orc, plan, o, f, y, sh, vx, tol)
    print(f"PARITY srt256 {wdt}{' csr' if csr else ''}{' rho-linear' if lin else ''}"
          f" (64^3 crop, 4096 shells, 96 voxels): forward rel-L2 {e_p:.3e},"
          f" adjoint rel-L2 {e_a:.3e}")
    fd, yd = to_dev(f), to_dev(y)
    af, aty = plan.forward(fd), plan.adjoint(yd)
    lhs, rhs = srt.dot_f64(af, yd), srt.dot_f64(fd, aty)
    assert abs(lhs - rhs) / math.sqrt(srt.dot_f64(af, af) * srt.dot_f64(yd, yd)) <= 1e-6


def test_srt256_bf16_against_fp32(srt, orc, srt256_inputs):
    """The precision comparison at 256^3: BF16-stored entries against FP32
    entries over the whole output (both FP32-accumulated)."""
    sz = dict(I.sizes("srt256"))
    g32, _ = geom_pair(orc, **sz)
    g16, _ = geom_pair(orc, weight_dtype="bf16", **sz)
    f, y = srt256_inputs
    fd, yd = to_dev(f), to_dev(y)
    a, b = srt.Plan(g32), srt.Plan(g16)
    e_p = rel_l2(to_np(b.forward(fd)), to_np(a.forward(fd)))
    e_a = rel_l2(to_np(b.adjoint(yd)), to_np(a.adjoint(yd)))
    print(f"PARITY srt256 bf16 vs fp32 entries (full output): forward rel-L2 {e_p:.3e}, "
          f"adjoint rel-L2 {e_a:.3e}")
    assert 1e-5 < e_p <= 5e-3 and 1e-5 < e_a <= 5e-3


def test_srt512_sampled_maximum_size(srt, orc):
    """The largest workload the suite runs: 512^3 voxels at 0.05 mm, 256
    sensor columns, 512 rings, 1536 radius bins (8x the benchmark's voxels,
    about 4 GB on the device), in the default form (8-fold A1, Toeplitz taps,
    register tiles).  Every index the kernels form (tile-record offsets,
    A1^T keys j << 16 | l, pixel indices under the multiply-shift quotient of
    the symmetry map, row offsets into 805 MB operands) is larger here than
    anywhere else; sampled shells and voxels against the oracle, on a volume
    that is random inside the central 48^3 voxels and zero elsewhere, and
    the adjoint identity over the whole output."""
    sz = dict(ms=512, mz=512, dxy=0.05, dz=0.05, radius=20.0, n_phi=256, n_zs=512, n_ell=1536)
    g, o = geom_pair(orc, **sz)
    plan = srt.Plan(g)
    assert plan.info["a1_rot"] == 2 and plan.info["a2_taps"] == 1
    assert min(plan.info["tile_records"]) > 0
    rng = np.random.default_rng(51)
    c = 48
    a = (g.ms - c) // 2
    f = np.zeros(g.f_shape, dtype=np.float32)
    f[a:a + c, a:a + c, a:a + c] = rng.uniform(0, 1, (c, c, c))
    y = rng.standard_normal(g.p_shape, dtype=np.float32)
    sh, vx = _samples(g, 512, 24, 52, crop=c)
    e_p, e_a = _check(srt, orc, plan, o, f, y, sh, vx, 1e-5)
    print(f"PARITY srt512 fp32 (48^3 crop, 512 shells, 24 voxels): forward rel-L2 {e_p:.3e}, "
          f"adjoint rel-L2 {e_a:.3e}")
    fd, yd = to_dev(f), to_dev(y)
    af, aty = plan.forward(fd), plan.adjoint(yd)
    lhs, rhs = srt.dot_f64(af, yd), srt.dot_f64(fd, aty)
    assert abs(lhs - rhs) / math.sqrt(srt.dot_f64(af, af) * srt.dot_f64(yd, yd)) <= 1e-6
    plan.close()
