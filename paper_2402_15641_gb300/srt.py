"""Python binding of libsrt: geometry, plans and the transform on torch tensors.

Argument marshalling only: every step of the transform runs in the CUDA
kernels behind include/srt.h.  torch supplies device memory and streams.

Layouts (float32, contiguous, on the plan's device):
  volume       f: [B, ms, ms, mz]            (or [ms, ms, mz] for B = 1)
  measurements p: [B, n_phi, n_zs, n_ell]    (or [n_phi, n_zs, n_ell])
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, asdict, replace

import numpy as np
import torch

from . import _lib as L
from ._lib import check


@dataclass(frozen=True)
class Geometry:
    """Mirror of ``srt_geometry`` (lengths mm, angles rad)."""

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
    weight_dtype: str = "fp32"  # "fp32" | "bf16"
    keep_f64: bool = False
    csr_only: bool = False
    a1_rotation: bool = False
    rho_linear: bool = False  # intermediate piecewise linear in rho (else constant on bins)
    rowwise: bool = False  # every product a warp per output row (else register tiles of rows)
    n_phi_total: int = 0  # > 0: the plan holds columns phi_first .. + n_phi - 1 of this many
    phi_first: int = 0
    a1_full: bool = False  # store A1 for every column (else for the aperture's symmetry set)
    fuse_reshapes: bool = False  # P2 / P1^-1 folded into the A2 / A2^T tiles
    voxel_linear: bool = False  # f bilinear in (x, y) between voxel centres (else constant)

    @staticmethod
    def default(ms, mz, dxy, dz, radius, n_phi, n_zs, n_ell, **options) -> "Geometry":
        """Default readings, computed by the library (srt_geometry_default);
        options set weight_dtype / keep_f64 / csr_only / a1_rotation / rho_linear /
        rowwise / a1_full / fuse_reshapes / voxel_linear."""
        g = L.SrtGeometry()
        check(L.lib().srt_geometry_default(ctypes.byref(g), ms, mz, dxy, dz, radius, n_phi, n_zs,
                                           n_ell), "srt_geometry_default")
        return Geometry(g.ms, g.mz, g.dxy, g.dz, g.radius, g.n_phi, g.phi0, g.n_zs, g.zs_lo,
                        g.zs_hi, g.n_ell, g.ell_lo, g.ell_hi, **options)

    @staticmethod
    def from_sizes(d: dict, **kw) -> "Geometry":
        return Geometry.default(d["ms"], d["mz"], d["dxy"], d["dz"], d["radius"], d["n_phi"],
                                d["n_zs"], d["n_ell"], **kw)

    def with_(self, **kw) -> "Geometry":
        return replace(self, **kw)

    def column_block(self, j0: int, j1: int) -> "Geometry":
        """The plan geometry of sensor columns j0 .. j1-1 of this aperture."""
        if not 0 <= j0 < j1 <= self.n_phi or self.n_phi_total:
            raise ValueError(f"column block [{j0}, {j1}) of {self.n_phi} columns")
        return replace(self, n_phi=j1 - j0, n_phi_total=self.n_phi, phi_first=j0)

    def to_c(self) -> L.SrtGeometry:
        wd = {"fp32": L.SRT_FP32, "bf16": L.SRT_BF16}[self.weight_dtype]
        return L.SrtGeometry(self.ms, self.mz, self.dxy, self.dz, self.radius, self.n_phi,
                             self.phi0, self.n_zs, self.zs_lo, self.zs_hi, self.n_ell,
                             self.ell_lo, self.ell_hi, wd,
                             (L.SRT_KEEP_F64 if self.keep_f64 else 0)
                             | (L.SRT_CSR_ONLY if self.csr_only else 0)
                             | (L.SRT_A1_ROTATION if self.a1_rotation else 0)
                             | (L.SRT_RHO_LINEAR if self.rho_linear else 0)
                             | (L.SRT_ROWWISE if self.rowwise else 0)
                             | (L.SRT_A1_FULL if self.a1_full else 0)
                             | (L.SRT_FUSE_RESHAPES if self.fuse_reshapes else 0)
                             | (L.SRT_VOXEL_LINEAR if self.voxel_linear else 0),
                             self.n_phi_total, self.phi_first)

    @property
    def f_shape(self):
        return (self.ms, self.ms, self.mz)

    @property
    def p_shape(self):
        return (self.n_phi, self.n_zs, self.n_ell)

    def as_dict(self):
        return asdict(self)


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


_CPU = torch.device("cpu")


class Plan:
    """An assembled operator pair (A1, A2 and transposes) resident on one GPU."""

    def __init__(self, geom: Geometry, device=None, stream=None, lib=None):
        """lib: a loaded libsrt (_lib.load), e.g. the debug build with its
        gathered-row checks; default: the package's libsrt.so."""
        if not torch.cuda.is_available():
            raise RuntimeError("srt.Plan needs a CUDA device; there is no CPU path")
        self.geom = geom
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self._lib = L.lib() if lib is None else lib
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self._lib.srt_plan(ctypes.byref(geom.to_c()), ctypes.c_void_p(_stream_ptr(stream)),
                                     ctypes.byref(h)), "srt_plan")
        self._h = h
        self._ws = {}
        info = L.SrtPlanInfo()
        check(self._lib.srt_plan_info(self._h, ctypes.byref(info)), "srt_plan_info")
        self.info = {k: getattr(info, k) for k, _ in L.SrtPlanInfo._fields_}
        self.info["tile_records"] = list(info.tile_records)

    # -------------------------------------------------------------- memory
    def workspace_bytes(self, batch: int = 1) -> int:
        n = ctypes.c_size_t()
        check(self._lib.srt_workspace_bytes(self._h, batch, ctypes.byref(n)), "srt_workspace_bytes")
        return n.value

    def host_workspace_bytes(self, batch: int = 1) -> int:
        n = ctypes.c_size_t()
        check(self._lib.srt_host_workspace_bytes(self._h, batch, ctypes.byref(n)),
              "srt_host_workspace_bytes")
        return n.value

    def workspace(self, batch: int = 1, host: bool = False) -> torch.Tensor:
        """The plan's cached workspace for `batch` (shared by every call that
        passes no workspace: calls that may overlap on the device, e.g. on
        different streams or threads, need workspaces of their own)."""
        key = (batch, host)
        if key not in self._ws:
            nb = self.host_workspace_bytes(batch) if host else self.workspace_bytes(batch)
            self._ws[key] = torch.empty(nb, dtype=torch.uint8, device=self.device)
        return self._ws[key]

    # ---------------------------------------------------------- transforms
    def _batch(self, t: torch.Tensor, shape) -> int:
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("expected a contiguous float32 tensor")
        if tuple(t.shape) == tuple(shape):
            return 1
        if t.dim() == len(shape) + 1 and tuple(t.shape[1:]) == tuple(shape):
            return t.shape[0]
        raise ValueError(f"shape {tuple(t.shape)} does not match {tuple(shape)}")

    # The library takes raw pointers: a tensor on the wrong device or an output
    # that is too small would be read or written out of bounds, so both are
    # refused here, before any call.
    @staticmethod
    def _on(t: torch.Tensor, device: torch.device, what: str) -> None:
        if t.device != device:
            raise ValueError(f"{what} must be on {device}, not {t.device}")

    def _out(self, t: torch.Tensor, batch: int, shape, device: torch.device, what: str) -> None:
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{what}: expected a contiguous float32 tensor")
        self._on(t, device, what)
        if t.numel() != batch * int(np.prod(shape)):
            raise ValueError(f"{what}: shape {tuple(t.shape)} does not hold {batch} x "
                             f"{tuple(shape)}")

    def _workspace(self, ws: torch.Tensor) -> tuple[int, int]:
        """(pointer, size in bytes) of a caller's device workspace."""
        self._on(ws, self.device, "workspace")
        if not ws.is_contiguous():
            raise ValueError("workspace must be contiguous")
        return _ptr(ws), ws.numel() * ws.element_size()

    def forward(self, f: torch.Tensor, out: torch.Tensor | None = None, workspace=None,
                stream=None) -> torch.Tensor:
        """p = A f (Algorithm 1 on every sensor column)."""
        B = self._batch(f, self.geom.f_shape)
        self._on(f, self.device, "f")
        if out is None:
            shape = self.geom.p_shape if f.dim() == 3 else (B, *self.geom.p_shape)
            out = torch.empty(shape, dtype=torch.float32, device=f.device)
        else:
            self._out(out, B, self.geom.p_shape, self.device, "out")
        ws, nb = self._workspace(self.workspace(B) if workspace is None else workspace)
        check(self._lib.srt_forward(self._h, _ptr(f), _ptr(out), B, ws, nb,
                                    ctypes.c_void_p(_stream_ptr(stream))), "srt_forward")
        return out

    def adjoint(self, p: torch.Tensor, out: torch.Tensor | None = None, workspace=None,
                stream=None) -> torch.Tensor:
        """f' = A^T p (Algorithm 2, matched adjoint)."""
        B = self._batch(p, self.geom.p_shape)
        self._on(p, self.device, "p")
        if out is None:
            shape = self.geom.f_shape if p.dim() == 3 else (B, *self.geom.f_shape)
            out = torch.empty(shape, dtype=torch.float32, device=p.device)
        else:
            self._out(out, B, self.geom.f_shape, self.device, "out")
        ws, nb = self._workspace(self.workspace(B) if workspace is None else workspace)
        check(self._lib.srt_adjoint(self._h, _ptr(p), _ptr(out), B, ws, nb,
                                    ctypes.c_void_p(_stream_ptr(stream))), "srt_adjoint")
        return out

    def forward_host(self, f_host: torch.Tensor, out_host: torch.Tensor, stream=None):
        """End-to-end forward on host tensors (copies inside the call)."""
        B = self._batch(f_host, self.geom.f_shape)
        self._on(f_host, _CPU, "f_host")
        self._out(out_host, B, self.geom.p_shape, _CPU, "out_host")
        ws, nb = self._workspace(self.workspace(B, host=True))
        check(self._lib.srt_forward_host(self._h, _ptr(f_host), _ptr(out_host), B, ws, nb,
                                         ctypes.c_void_p(_stream_ptr(stream))),
              "srt_forward_host")
        return out_host

    def adjoint_host(self, p_host: torch.Tensor, out_host: torch.Tensor, stream=None):
        """End-to-end adjoint on host tensors (copies inside the call)."""
        B = self._batch(p_host, self.geom.p_shape)
        self._on(p_host, _CPU, "p_host")
        self._out(out_host, B, self.geom.f_shape, _CPU, "out_host")
        ws, nb = self._workspace(self.workspace(B, host=True))
        check(self._lib.srt_adjoint_host(self._h, _ptr(p_host), _ptr(out_host), B, ws, nb,
                                         ctypes.c_void_p(_stream_ptr(stream))),
              "srt_adjoint_host")
        return out_host

    # ------------------------------------------------------------- extras
    def export(self, which: int, f64: bool = False):
        """(rowptr, col, val32, val64|None) of A1 (1), A2 (2), A1^T (3), A2^T (4)."""
        rows = {1: self.info["rows1"], 2: self.info["rows2"], 3: self.info["cols1"],
                4: self.info["cols2"]}[which]
        nnz = self.info["nnz1"] if which in (1, 3) else self.info["nnz2"]
        rp = np.zeros(rows + 1, dtype=np.int32)
        col = np.zeros(max(nnz, 1), dtype=np.int32)
        v32 = np.zeros(max(nnz, 1), dtype=np.float32)
        v64 = np.zeros(max(nnz, 1), dtype=np.float64) if f64 else None
        check(self._lib.srt_plan_export(self._h, which, rp.ctypes.data, col.ctypes.data,
                                        v32.ctypes.data, v64.ctypes.data if f64 else None),
              "srt_plan_export")
        return rp, col[:nnz], v32[:nnz], (v64[:nnz] if f64 else None)

    def set_timing(self, enable: bool = True):
        check(self._lib.srt_plan_set_timing(self._h, 1 if enable else 0), "srt_plan_set_timing")

    def stage_times(self, direction: int):
        buf = (ctypes.c_float * 4)()
        check(self._lib.srt_stage_times(self._h, direction, buf, 4), "srt_stage_times")
        return list(buf)

    def launches_per_call(self, direction: int = 0, batch: int = 1) -> int:
        return int(self._lib.srt_launches_per_call(self._h, direction, batch))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.srt_plan_destroy(self._h)
            self._h = None
            self._ws.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pipeline:
    """Host-buffer calls with up to `slots` (2-4) in flight (srt_pipe_*): a
    call copies its input while earlier calls compute, and its result goes
    back while later calls compute.  submit() returns a ticket at once; the
    host tensors are held until wait(ticket)."""

    def __init__(self, plan: Plan, batch: int = 1, slots: int = 3):
        self.plan, self.batch, self.slots = plan, batch, slots
        self._lib = L.lib()
        h = ctypes.c_void_p()
        check(self._lib.srt_pipe_create(plan._h, batch, slots, ctypes.byref(h)),
              "srt_pipe_create")
        self._h = h
        self._held = {}

    def submit(self, direction: str, in_host: torch.Tensor, out_host: torch.Tensor) -> int:
        if not getattr(self, "_h", None) or not getattr(self.plan, "_h", None):
            raise RuntimeError("pipeline or its plan has been closed")
        g = self.plan.geom
        d = {"forward": 0, "adjoint": 1}[direction]
        shapes = (g.f_shape, g.p_shape) if d == 0 else (g.p_shape, g.f_shape)
        for t, shp in zip((in_host, out_host), shapes):
            if t.device.type != "cpu" or self.plan._batch(t, shp) != self.batch:
                raise ValueError(f"expected a host tensor of {self.batch} x {shp}")
        tk = ctypes.c_int64()
        check(self._lib.srt_pipe_submit(self._h, d, _ptr(in_host), _ptr(out_host),
                                        ctypes.byref(tk)), "srt_pipe_submit")
        self._held[tk.value] = (in_host, out_host)
        return tk.value

    def wait(self, ticket: int, timeout_s: float = 60.0) -> torch.Tensor:
        """Block until call `ticket`'s result is in its host tensor; returns it."""
        check(self._lib.srt_pipe_wait(self._h, ticket, timeout_s), "srt_pipe_wait")
        for t in [t for t in self._held if t <= ticket]:
            out = self._held.pop(t)[1]
            if t == ticket:
                return out
        return None

    def stage_times(self, ticket: int):
        """(input copy, transform, result copy, compute idle before it) in ms
        for a finished call among the last 8 submitted."""
        buf = (ctypes.c_float * 4)()
        check(self._lib.srt_pipe_stage_times(self._h, ticket, buf), "srt_pipe_stage_times")
        return tuple(buf)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.srt_pipe_destroy(self._h)
            self._h = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_dot_ws = {}


def dot_f64(a: torch.Tensor, b: torch.Tensor, stream=None) -> float:
    """FP64 inner product of two float32 device tensors (deterministic)."""
    if a.numel() != b.numel() or a.dtype != torch.float32 or b.dtype != torch.float32:
        raise ValueError("dot_f64 needs two float32 tensors of equal size")
    if a.device.type != "cuda" or b.device != a.device:
        raise ValueError(f"dot_f64 needs both tensors on one CUDA device, not {a.device}, "
                         f"{b.device}")
    a, b = a.contiguous(), b.contiguous()
    lib = L.lib()
    dev = a.device
    if dev not in _dot_ws:
        _dot_ws[dev] = torch.empty(lib.srt_dot_workspace_bytes() // 8 + 1, dtype=torch.float64,
                                   device=dev)
    ws = _dot_ws[dev]
    out = ws[-1:]
    check(lib.srt_dot_f64(_ptr(a), _ptr(b), a.numel(), _ptr(out), _ptr(ws),
                          (ws.numel() - 1) * 8, ctypes.c_void_p(_stream_ptr(stream))),
          "srt_dot_f64")
    return float(out.item())


def fp32_fma_peak(iters: int = 20000, stream=None) -> float:
    """Sustained FP32 FMA rate of the current GPU's CUDA cores, TFLOP/s."""
    out = ctypes.c_double()
    check(L.lib().srt_fp32_fma_peak(iters, ctypes.byref(out),
                                    ctypes.c_void_p(_stream_ptr(stream))), "srt_fp32_fma_peak")
    return out.value
