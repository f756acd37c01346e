"""FP64 CPU oracle for the discrete cylindrical-aperture SRT (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and does not import the product package.

The arithmetic lives in ``srt_oracle.c`` (per-shell direct quadrature of the
paper's discretisation, Sec. 2 and Sec. 3.1 / Algorithm 1 of the paper, without
forming the two CRT matrices).  This file builds it with gcc and marshals
numpy arrays.

Parity status: every exported function is pinned by ``tests/test_oracle_*.py``:
- the closed-form ball;
- brute-force shell sampling, with the in-plane radius snapped, interpolated
  and exact (the continuum limit);
- analytic arc lengths and first moments;
- coarea area sums;
- the adjoint identity;
- symmetries;
- a hand-computed one-voxel case;
- for the piecewise-linear voxels: partition of unity against the constant
  basis, dense sampling of the interpolated function along circles, the walk
  against the per-node box moments, and the adjoint identity.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, asdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsrt_oracle.so")


@dataclass(frozen=True)
class OracleGeometry:
    """Cylindrical-aperture geometry as the oracle reads it (all lengths mm)."""

    ms: int
    mz: int
    dxy: float
    dz: float
    radius: float
    n_phi: int
    phi0: float
    n_zs: int
    zs_lo: float
    zs_hi: float
    n_ell: int
    ell_lo: float
    ell_hi: float
    rho_linear: bool = False  # intermediate piecewise linear in rho (else constant on bins)
    voxel_linear: bool = False  # f bilinear in (x, y) between voxel centres (else constant)

    @staticmethod
    def default(ms, mz, dxy, dz, radius, n_phi, n_zs, n_ell, phi0=0.0, rho_linear=False,
                voxel_linear=False):
        """Default readings: rings at cell centres of the volume height and a
        radius grid covering [R - r_xy, R + r_xy], r_xy = ms*dxy/sqrt(2)."""
        h = mz * dz
        rxy = ms * dxy / math.sqrt(2.0)
        return OracleGeometry(ms, mz, float(dxy), float(dz), float(radius), n_phi, float(phi0),
                              n_zs, -0.5 * h, 0.5 * h, n_ell, radius - rxy, radius + rxy,
                              bool(rho_linear), bool(voxel_linear))

    @property
    def n_vox(self):
        return self.ms * self.ms * self.mz

    @property
    def p_shape(self):
        return (self.n_phi, self.n_zs, self.n_ell)

    @property
    def f_shape(self):
        return (self.ms, self.ms, self.mz)

    def as_dict(self):
        return asdict(self)


class _Geom(ctypes.Structure):
    _fields_ = [
        ("ms", ctypes.c_int32), ("mz", ctypes.c_int32),
        ("dxy", ctypes.c_double), ("dz", ctypes.c_double), ("radius", ctypes.c_double),
        ("n_phi", ctypes.c_int32), ("phi0", ctypes.c_double),
        ("n_zs", ctypes.c_int32), ("zs_lo", ctypes.c_double), ("zs_hi", ctypes.c_double),
        ("n_ell", ctypes.c_int32), ("ell_lo", ctypes.c_double), ("ell_hi", ctypes.c_double),
        ("rho_linear", ctypes.c_int32), ("voxel_linear", ctypes.c_int32),
    ]


def _cg(g: OracleGeometry) -> _Geom:
    return _Geom(g.ms, g.mz, g.dxy, g.dz, g.radius, g.n_phi, g.phi0, g.n_zs, g.zs_lo, g.zs_hi,
                 g.n_ell, g.ell_lo, g.ell_hi, int(g.rho_linear), int(g.voxel_linear))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, strict IEEE: no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lp = ctypes.POINTER(ctypes.c_long)
        G = ctypes.POINTER(_Geom)
        _lib.orc_forward.argtypes = [G, dp, dp, ctypes.c_int]
        _lib.orc_adjoint.argtypes = [G, dp, dp, ctypes.c_int]
        _lib.orc_forward_shells.argtypes = [G, dp, ip, ctypes.c_long, dp, ctypes.c_int]
        _lib.orc_adjoint_voxels.argtypes = [G, dp, ip, ctypes.c_long, dp, ctypes.c_int]
        _lib.orc_adjoint_shells.argtypes = [G, ip, dp, ctypes.c_long, dp, ctypes.c_int]
        _lib.orc_shell_contrib.argtypes = [G, ctypes.c_int, ctypes.c_int, ctypes.c_int, lp, dp,
                                           ctypes.c_long]
        _lib.orc_shell_contrib.restype = ctypes.c_long
        _lib.orc_circle_arcs.argtypes = [G, ctypes.c_int, ctypes.c_int, ip, dp, ctypes.c_int]
        _lib.orc_semicircle_arcs.argtypes = [G, ctypes.c_int, ctypes.c_int, ip, dp, ctypes.c_int]
        _lib.orc_point_weight.argtypes = [G] + [ctypes.c_int] * 6
        _lib.orc_point_weight.restype = ctypes.c_double
        _lib.orc_arc_in_box.argtypes = [ctypes.c_double] * 7
        _lib.orc_arc_in_box.restype = ctypes.c_double
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def forward(g: OracleGeometry, f, nthreads: int = 0) -> np.ndarray:
    """p[j, h, m] for a volume f[ix, iy, iz] (FP64)."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(g.f_shape)
    p = np.zeros(g.p_shape, dtype=np.float64)
    r = lib().orc_forward(ctypes.byref(_cg(g)), _dptr(f), _dptr(p), nthreads)
    if r:
        raise RuntimeError(f"orc_forward failed ({r})")
    return p


def adjoint(g: OracleGeometry, p, nthreads: int = 0) -> np.ndarray:
    """f'[ix, iy, iz] = A^T p, from the same shell weights as :func:`forward`."""
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(g.p_shape)
    f = np.zeros(g.f_shape, dtype=np.float64)
    r = lib().orc_adjoint(ctypes.byref(_cg(g)), _dptr(p), _dptr(f), nthreads)
    if r:
        raise RuntimeError(f"orc_adjoint failed ({r})")
    return f


def forward_shells(g: OracleGeometry, f, shells, nthreads: int = 0) -> np.ndarray:
    """Forward values at shells[i] = (j, h, m)."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(g.f_shape)
    sh = np.ascontiguousarray(shells, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(len(sh), dtype=np.float64)
    r = lib().orc_forward_shells(ctypes.byref(_cg(g)), _dptr(f), _iptr(sh), len(sh), _dptr(out),
                                 nthreads)
    if r:
        raise RuntimeError(f"orc_forward_shells failed ({r})")
    return out


def adjoint_voxels(g: OracleGeometry, p, voxels, nthreads: int = 0) -> np.ndarray:
    """Adjoint values at voxels[i] = (ix, iy, k), via per-voxel weights."""
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(g.p_shape)
    vx = np.ascontiguousarray(voxels, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(len(vx), dtype=np.float64)
    r = lib().orc_adjoint_voxels(ctypes.byref(_cg(g)), _dptr(p), _iptr(vx), len(vx), _dptr(out),
                                 nthreads)
    if r:
        raise RuntimeError(f"orc_adjoint_voxels failed ({r})")
    return out


def adjoint_shells(g: OracleGeometry, shells, vals, nthreads: int = 0) -> np.ndarray:
    """A^T applied to data that is zero except at shells[i] = (j, h, m), where
    it equals vals[i]; returns the full volume."""
    sh = np.ascontiguousarray(shells, dtype=np.int32).reshape(-1, 3)
    v = np.ascontiguousarray(vals, dtype=np.float64).reshape(-1)
    f = np.zeros(g.f_shape, dtype=np.float64)
    r = lib().orc_adjoint_shells(ctypes.byref(_cg(g)), _iptr(sh), _dptr(v), len(sh), _dptr(f),
                                 nthreads)
    if r:
        raise RuntimeError(f"orc_adjoint_shells failed ({r})")
    return f


def shell_weights(g: OracleGeometry, j: int, h: int, m: int) -> dict:
    """Per-voxel weights of one shell, {voxel index: weight}, from the walk."""
    cap = 1 << 16
    while True:
        vox = np.zeros(cap, dtype=np.int64)
        w = np.zeros(cap, dtype=np.float64)
        n = lib().orc_shell_contrib(ctypes.byref(_cg(g)), j, h, m,
                                    vox.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dptr(w),
                                    cap)
        if n == -3:
            cap *= 4
            continue
        if n < 0:
            raise RuntimeError(f"orc_shell_contrib failed ({n})")
        out: dict = {}
        for v, x in zip(vox[:n].tolist(), w[:n].tolist()):
            out[v] = out.get(v, 0.0) + x
        return out


def circle_arcs(g: OracleGeometry, j: int, l: int) -> dict:
    """In-plane circle (column j, bin-centre radius rho_l): {pixel: arc length},
    or with piecewise-linear voxels {node: integral of its basis}."""
    cap = 4 * (8 * g.ms + 8) if g.voxel_linear else 4 * (g.ms + 1) + 4
    pix = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap, dtype=np.float64)
    n = lib().orc_circle_arcs(ctypes.byref(_cg(g)), j, l, _iptr(pix), _dptr(ln), cap)
    if n < 0:
        raise RuntimeError(f"orc_circle_arcs failed ({n})")
    out: dict = {}
    for q, x in zip(pix[:n].tolist(), ln[:n].tolist()):
        out[q] = out.get(q, 0.0) + x
    return out


def semicircle_arcs(g: OracleGeometry, h: int, m: int) -> dict:
    """(z, rho) semicircle (ring h, radius l_m): {cell l*mz + k: weight}; the
    weight is the arc length in the cell (piecewise-constant intermediate) or
    the node's hat integrated along the arc in the slab (piecewise linear)."""
    cap = 2 * (2 * (g.mz + 1) + 2 * (g.n_ell + 2) + 4)
    cell = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap, dtype=np.float64)
    n = lib().orc_semicircle_arcs(ctypes.byref(_cg(g)), h, m, _iptr(cell), _dptr(ln), cap)
    if n < 0:
        raise RuntimeError(f"orc_semicircle_arcs failed ({n})")
    out: dict = {}
    for c, x in zip(cell[:n].tolist(), ln[:n].tolist()):
        out[c] = out.get(c, 0.0) + x
    return out


def point_weight(g: OracleGeometry, j, h, m, ix, iy, k) -> float:
    return float(lib().orc_point_weight(ctypes.byref(_cg(g)), j, h, m, ix, iy, k))


def arc_in_box(cx, cy, r, x0, x1, y0, y1) -> float:
    return float(lib().orc_arc_in_box(cx, cy, r, x0, x1, y0, y1))
