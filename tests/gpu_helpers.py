"""Shared helpers for the GPU parity tests (not a test module)."""
from __future__ import annotations

import math

import numpy as np


def geom_pair(orc, ms, mz, dxy, dz, radius, n_phi, n_zs, n_ell, phi0=0.0, zs=None, ell=None,
              weight_dtype="fp32", keep_f64=False, csr_only=False, a1_rotation=False,
              rho_linear=False, rowwise=False, a1_full=False, voxel_linear=False):
    """The same explicit geometry for the CUDA plan and for the oracle."""
    from paper_2402_15641_gb300.srt import Geometry
    h = mz * dz
    rxy = ms * dxy / math.sqrt(2.0)
    zs_lo, zs_hi = zs if zs is not None else (-0.5 * h, 0.5 * h)
    ell_lo, ell_hi = ell if ell is not None else (radius - rxy, radius + rxy)
    g = Geometry(ms, mz, float(dxy), float(dz), float(radius), n_phi, float(phi0), n_zs,
                 float(zs_lo), float(zs_hi), n_ell, float(ell_lo), float(ell_hi),
                 weight_dtype, keep_f64, csr_only, a1_rotation, rho_linear, rowwise,
                 a1_full=a1_full, voxel_linear=voxel_linear)
    o = orc.OracleGeometry(ms, mz, float(dxy), float(dz), float(radius), n_phi, float(phi0), n_zs,
                           float(zs_lo), float(zs_hi), n_ell, float(ell_lo), float(ell_hi),
                           bool(rho_linear), bool(voxel_linear))
    return g, o


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def to_np(t):
    return t.detach().double().cpu().numpy()


def bf16_is_rne_of(widened: np.ndarray, exact: np.ndarray) -> np.ndarray:
    """True where `widened` (float32 holding a BF16 value) is the round-to-
    nearest-even BF16 of `exact` (FP64): it is representable, no BF16
    neighbour is closer, and on a tie its last fraction bit is even."""
    w = np.asarray(widened, dtype=np.float32)
    bits = w.view(np.uint32)
    ok = (bits & 0xFFFF) == 0
    up = (bits + (1 << 16)).view(np.float32).astype(np.float64)
    dn = (bits - (1 << 16)).view(np.float32).astype(np.float64)
    d0 = np.abs(w.astype(np.float64) - exact)
    ok &= d0 <= np.abs(up - exact)
    ok &= d0 <= np.abs(dn - exact)
    tie = (d0 == np.abs(up - exact)) | (d0 == np.abs(dn - exact))
    ok &= ~tie | (((bits >> 16) & 1) == 0)
    return ok
