#!/usr/bin/env python
"""Throughput of the cylindrical-aperture SRT: forward + matched adjoint.

One step = srt_forward followed by srt_adjoint of one batch of volumes on the
256^3 workload (256^3 voxels @ 0.1 mm, R = 20 mm, 256 sensor columns, 256
rings, 768 radius bins; FP32 entries, batch 1) unless --workload/--weights
say otherwise.  Inputs are seeded synthetic phantoms (100 balls + 500-blob
vessel tree) and N(0, 1) measurement-shaped data, resident in HBM before the
timed region; L2 is flushed (256 MiB write) between timed steps.

Prints ONE JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle
(the only reference this method has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SRT fwd+adj ops/s & HBM GB/s vs peak at 256^3"
UNIT = "fwd+adj pairs/s"
FP32_LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="srt256")
    p.add_argument("--weights", choices=["fp32", "bf16"], default="fp32")
    p.add_argument("--batch", type=int, default=1)
    p.add_argument("--csr-only", action="store_true",
                   help="store A2, A2^T as CSR instead of applying them from the Toeplitz taps")
    p.add_argument("--a1-rotation", action="store_true",
                   help="store A1 for a quarter of the sensor columns (quarter turns only, no mirror)")
    p.add_argument("--rowwise", action="store_true",
                   help="every product a warp per output row (else register tiles of rows)")
    p.add_argument("--voxel-linear", action="store_true",
                   help="f bilinear in (x, y) between voxel centres (else constant on voxels)")
    p.add_argument("--fuse-reshapes", action="store_true",
                   help="P2 and P1^-1 folded into the A2 / A2^T tile products")
    p.add_argument("--a1-full", action="store_true",
                   help="store A1 for every sensor column (else for the aperture's symmetry set)")
    p.add_argument("--rho-linear", action="store_true",
                   help="piecewise-linear intermediate in rho (else constant on the radius bins)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=100)
    p.add_argument("--e2e-depth", type=int, default=3,
                   help="steps submitted ahead of the one whose result is read (1-3)")
    return p.parse_args()


def peaks(n_sm):
    """Roofline denominators: measured HBM copy bandwidth and SM clock, and
    the FP32 FMA peak derived from the device's SM count and that clock."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    d = {}
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
    hbm = d.get("hbm_gbs", 6800.0)
    sm_max = d.get("sm_max_mhz", 2070.0)
    src = "measured" if "hbm_gbs" in d else "fallback"
    # FP32 FMA peak from unit counts and the maximum SM clock: SMs x 128
    # FP32 lanes x 2 FLOP per FMA x clock.
    fp32 = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    return dict(hbm_gbs=hbm, fp32_tflops=fp32, sm_max_mhz=sm_max, src=src, n_sm=n_sm)


class Clocks:
    """nvidia-smi sampler for the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.file.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# Sources outside the timed transform (measurement helpers): not hashed.
NOT_ON_PATH = ("peak.cu",)


def csrc_digest():
    """Hash of the CUDA sources of the transform, to tie ncu counters to the
    kernels they were taken on."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2402_15641_gb300", "csrc")
    for n in sorted(os.listdir(d)):
        if n.endswith((".cu", ".cuh")) and n not in NOT_ON_PATH:
            with open(os.path.join(d, n), "rb") as fh:
                h.update(n.encode())
                h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_stage, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                rec[k.strip()] = v.strip()
    if rec.get("csrc_sha") != csrc_digest():
        return None
    v = rec.get(f"dram_bytes_per_launch.{kernel_stage}")
    return float(v) if v else None


def stage_model(geom, info, batch, weights, fused=False, fused_p1=False):
    """Algorithmic FLOPs and compulsory bytes per launch of each stage.
    fused: A2 writes p and A2^T writes F1 in the reshaped layouts (no P2 and
    P1^-1 kernels); fused_p1: A1 writes Y1' (no P1 kernel).  The fused
    reshapes' stages are dropped, the products' bytes unchanged."""
    vb = 2 if weights == "bf16" else 4
    pix, c1 = geom.ms * geom.ms, geom.n_ell * geom.mz
    r1, r2 = geom.n_phi * geom.n_ell, geom.n_zs * geom.n_ell
    nnz1, nnz2 = info["nnz1"], info["nnz2"]
    y1 = 4 * batch * r1 * geom.mz           # bytes of Y1 (= Y1')
    pp = 4 * batch * r2 * geom.n_phi        # bytes of P' (= p)
    fv = 4 * batch * pix * geom.mz          # bytes of f
    # A1 (and A1^T) stored for a fundamental set of columns: a quarter under
    # quarter turns, an eighth (n_phi/8 + 1 of n_phi columns) with the mirror
    frac = {1: 1 / 4, 2: (geom.n_phi // 8 + 1) / geom.n_phi}.get(info.get("a1_rot", 0), 1.0)
    a1b = int(nnz1 * frac) * (vb + 4) + 4 * (int(r1 * frac) + 1)
    a1tb = int(nnz1 * frac) * (vb + 4) + 4 * (pix + 1)
    spmm1 = dict(flop=2 * nnz1 * geom.mz * batch, bytes=a1b + fv + y1)
    if info.get("a2_taps"):  # A2 held by the taps of T: key + value per tap, sub-row pointers
        sub = 4 * (geom.n_ell * (2 * geom.mz - 1) + 1)
        a2b = a2tb = info["n_taps"] * (vb + 4) + sub
    else:
        a2b = nnz2 * (vb + 4) + 4 * (r2 + 1)
        a2tb = nnz2 * (vb + 4) + 4 * (c1 + 1)
    spmm2 = dict(flop=2 * nnz2 * geom.n_phi * batch, bytes=a2b + y1 + pp)
    spmm2t = dict(flop=spmm2["flop"], bytes=a2tb + pp + y1)
    spmm1t = dict(flop=spmm1["flop"], bytes=a1tb + y1 + fv)
    # useful FMAs per gathered dense operand: 1 for a row-per-warp product;
    # entries per record for the register tiles (A1^T: stored entries, the
    # symmetry passes repeat entries and records alike)
    # (A2: the records are per radius pair and key, each folding the taps of
    # two rings or slabs, so entries per record = 2 n_taps / records away
    # from the volume's ends)
    rec = info.get("tile_records") or [0, 0, 0]
    for st, n_ent, r in ((spmm2, 2 * info.get("n_taps", 0), rec[0]),
                         (spmm2t, 2 * info.get("n_taps", 0), rec[1]),
                         (spmm1t, int(nnz1 * frac), rec[2])):
        st["fma_per_gather"] = round(n_ent / r, 3) if r else 1.0
    spmm1["fma_per_gather"] = 1.0
    p1 = dict(flop=0, bytes=2 * y1)
    p2 = dict(flop=0, bytes=2 * pp)
    return {"fwd": [("spmm1", spmm1), None if fused_p1 else ("permute1", p1), ("spmm2", spmm2),
                    None if fused else ("permute2", p2)],
            "adj": [("permute2_inv", p2), ("spmm2t", spmm2t),
                    None if fused else ("permute1_inv", p1), ("spmm1t", spmm1t)]}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x, world):
    """Max of x over the ranks (NCCL on the GPUs, or gloo on the host)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, batch, total_ms):
    """Whole-job fwd+adj pairs per second: every rank (an independent
    replica) processes steps x batch pairs, and the job lasts as long as the
    slowest rank (total_ms, already the max over ranks)."""
    return world * steps * batch / (total_ms / 1e3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload_config(name, geom, batch, weights, extra=None):
    from paper_2402_15641_gb300 import inputs as I
    w = I.WORKLOADS[name]
    cfg = {"workload": f"{name}: {geom.ms}^2x{geom.mz} voxels @ {geom.dxy} mm, R={geom.radius} mm, "
                       f"n_phi={geom.n_phi}, n_zs={geom.n_zs}, n_ell={geom.n_ell}, "
                       f"{weights} entries, batch {batch}",
           "phantom": f"{w.get('n_balls', 0)} balls + {w.get('n_blobs', 0)}-blob vessel tree "
                      f"(seed 0); adjoint input N(0,1) (seed 1)",
           "batch": batch, "weights": weights}
    if extra:
        cfg.update(extra)
    return cfg


def cpu_oracle_rate(name, budget_s, seed=5, rho_linear=False, voxel_linear=False):
    """Oracle forward + adjoint on a seeded shell sample sized to budget_s;
    returns (pairs/s extrapolated to the full workload, threads, sample text)."""
    import numpy as np
    from oracle import oracle as O
    from paper_2402_15641_gb300 import inputs as I
    sz = I.sizes(name)
    g = O.OracleGeometry.default(**sz, rho_linear=rho_linear, voxel_linear=voxel_linear)
    f = I.phantom(name)
    y = I.probe(name)
    total = g.n_phi * g.n_zs * g.n_ell
    rng = np.random.default_rng(seed)

    def sample(n):
        return np.stack([rng.integers(0, g.n_phi, n), rng.integers(0, g.n_zs, n),
                         rng.integers(0, g.n_ell, n)], axis=1)

    def run(sh):
        t0 = time.perf_counter()
        O.forward_shells(g, f, sh)
        O.adjoint_shells(g, sh, y[sh[:, 0], sh[:, 1], sh[:, 2]])
        return time.perf_counter() - t0

    # calibrate on samples large enough that start-up costs (threads, page
    # faults) do not inflate the per-shell time, then take about budget_s
    n, t = 64, 0.0
    for _ in range(3):
        t = run(sample(n))
        if t >= 0.25 * budget_s:
            break
        n = max(n, int(n * 0.3 * budget_s / max(t, 1e-3)))
    n = max(n, int(n * budget_s / max(t, 1e-3)))
    t = run(sample(n))
    rate = (n / total) / t
    return rate, O.num_threads(), n, t


def run_reference(args):
    world, rank, _ = dist_init()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2402_15641_gb300 import inputs as I
    import numpy as np
    sz = I.sizes(args.workload)
    g = O.OracleGeometry.default(**sz, rho_linear=args.rho_linear,
                                 voxel_linear=args.voxel_linear)
    f = I.phantom(args.workload)
    y = I.probe(args.workload)
    total = g.n_phi * g.n_zs * g.n_ell
    rng = np.random.default_rng(11)
    # size each step so that warmup + steps take about 90 s of host time
    sh = np.stack([rng.integers(0, g.n_phi, 64), rng.integers(0, g.n_zs, 64),
                   rng.integers(0, g.n_ell, 64)], axis=1)
    t0 = time.perf_counter()
    O.forward_shells(g, f, sh)
    O.adjoint_shells(g, sh, y[sh[:, 0], sh[:, 1], sh[:, 2]])
    per_shell = (time.perf_counter() - t0) / 64
    per_step = 90.0 / max(1, args.steps + args.warmup)
    n = int(max(8, min(200000, per_step / per_shell)))
    times = []
    for it in range(args.warmup + args.steps):
        sh = np.stack([rng.integers(0, g.n_phi, n), rng.integers(0, g.n_zs, n),
                       rng.integers(0, g.n_ell, n)], axis=1)
        t0 = time.perf_counter()
        O.forward_shells(g, f, sh)
        O.adjoint_shells(g, sh, y[sh[:, 0], sh[:, 1], sh[:, 2]])
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    frac = n / total
    value = args.steps * frac / sum(times)
    sample = (f"{n} seeded shells (of {total}) per step, oracle forward + adjoint over them; "
              f"rate extrapolated to the full operator by shell count")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{args.workload} (FP64 CPU oracle, per-shell quadrature)",
                      "sample_shells_per_step": n},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2402_15641_gb300 import build, inputs as I
    from paper_2402_15641_gb300.srt import Geometry, Pipeline, Plan, fp32_fma_peak

    build.build()
    pk = peaks(torch.cuda.get_device_properties(local).multi_processor_count)
    sz = I.sizes(args.workload)
    geom = Geometry.from_sizes(sz, weight_dtype=args.weights, csr_only=args.csr_only,
                               a1_rotation=args.a1_rotation, rho_linear=args.rho_linear,
                               rowwise=args.rowwise, a1_full=args.a1_full,
                               fuse_reshapes=args.fuse_reshapes,
                               voxel_linear=args.voxel_linear)
    B = args.batch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = Plan(geom)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0

    f_np = I.phantom(args.workload).astype(np.float32)
    y_np = I.probe(args.workload).astype(np.float32)
    f = torch.from_numpy(np.broadcast_to(f_np, (B, *f_np.shape)).copy()).cuda()
    y = torch.from_numpy(np.broadcast_to(y_np, (B, *y_np.shape)).copy()).cuda()
    p_out = torch.empty((B, *geom.p_shape), device="cuda")
    f_out = torch.empty((B, *geom.f_shape), device="cuda")
    ws = plan.workspace(B)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        plan.forward(f, out=p_out, workspace=ws)
        plan.adjoint(y, out=f_out, workspace=ws)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    fma_meas = fp32_fma_peak(5000)  # CUDA-core FMA roof, measured here (untimed)
    plan.set_timing(True)
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stage = {"fwd": [], "adj": []}
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        plan.forward(f, out=p_out, workspace=ws)
        plan.adjoint(y, out=f_out, workspace=ws)
        ev[k][1].record(stream)
        stage["fwd"].append(plan.stage_times(0))  # both calls are queued: no sync inside a step
        stage["adj"].append(plan.stage_times(1))
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    plan.set_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = reduce_max(sum(step_ms), world)
    value = job_rate(world, args.steps, B, total_ms)

    # per-stage figures from the CUDA events recorded on the launch stream
    # reshapes fused into the products: the tile products' (P2, P1^-1) take
    # one launch off each direction, A1's (P1) one more off the forward
    n_fwd, n_adj = plan.launches_per_call(0, B), plan.launches_per_call(1, B)
    fused, fused_p1 = n_adj == 3, n_fwd == n_adj - 1
    model = stage_model(geom, plan.info, B, args.weights, fused, fused_p1)
    stages = {}
    for d in ("fwd", "adj"):
        mean = np.mean(np.array(stage[d]), axis=0)
        for sm, ms in zip(model[d], mean):
            if sm is None:  # a reshape fused into its product
                continue
            name, m = sm
            s = {"ms": round(float(ms), 5), "gb_s": round(m["bytes"] / (ms * 1e6), 1),
                 "hbm_frac": round(m["bytes"] / (ms * 1e6) / pk["hbm_gbs"], 4)}
            if m["flop"]:
                s["tflop_s"] = round(m["flop"] / (ms * 1e9), 3)
                s["fp32_frac"] = round(m["flop"] / (ms * 1e9) / pk["fp32_tflops"], 4)
            s["flop"], s["bytes"] = m["flop"], m["bytes"]
            if "fma_per_gather" in m:
                s["fma_per_gather"] = m["fma_per_gather"]
            stages[f"{d}.{name}"] = s
    dom = max(stages, key=lambda k: stages[k]["ms"])
    ds = stages[dom]
    # L1 returns 128 B (32 FP32 operands) per clock per SM; a product whose
    # gathered operands each feed u useful FMAs cannot pass 32 u FMAs per
    # clock per SM (u = 1 for a row per warp, entries per record for tiles)
    delivery = pk["n_sm"] * 32 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12 * ds.get("fma_per_gather", 1.0)
    if "tflop_s" in ds:
        roof = {"bound": "alu", "achieved": ds["tflop_s"], "peak": round(pk["fp32_tflops"], 2),
                "unit": "TFLOP/s", "frac": ds["fp32_frac"],
                "traffic": ncu_traffic(dom, args.workload), "kernel": dom,
                "peak_source": f"derived: {pk['n_sm']} SMs x 128 FP32 lanes x 2 x max SM clock "
                               f"{pk['sm_max_mhz']:.0f} MHz",
                "fma_measured_tflops": round(fma_meas, 2),
                "frac_of_measured_fma": round(ds["tflop_s"] / fma_meas, 4),
                "fma_per_gather": ds.get("fma_per_gather", 1.0),
                "delivery_roof_tflops": round(delivery, 2),
                "frac_of_delivery_roof": round(ds["tflop_s"] / delivery, 4)}
    else:
        roof = {"bound": "hbm", "achieved": ds["gb_s"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ds["hbm_frac"], "traffic": ncu_traffic(dom, args.workload),
                "kernel": dom, "peak_source": f"{pk['src']} (MEASURED_PEAKS.json hbm_gbs)"}
    step_bytes = sum(s["bytes"] for s in stages.values())
    hbm = {"algorithmic_gb_per_step": round(step_bytes / 1e9, 4),
           "gb_s": round(step_bytes / (total_ms / args.steps * 1e6), 1)}
    hbm["frac_of_peak"] = round(hbm["gb_s"] / pk["hbm_gbs"], 4)

    # end to end through the public host-buffer entry points
    e2e = None
    if args.e2e_steps > 0:
        f_h = torch.from_numpy(np.broadcast_to(f_np, (B, *f_np.shape)).copy()).pin_memory()
        y_h = torch.from_numpy(np.broadcast_to(y_np, (B, *y_np.shape)).copy()).pin_memory()
        p_h = torch.empty((B, *geom.p_shape), dtype=torch.float32).pin_memory()
        a_h = torch.empty((B, *geom.f_shape), dtype=torch.float32).pin_memory()
        for _ in range(2):
            plan.forward_host(f_h, p_h)
            plan.adjoint_host(y_h, a_h)
        torch.cuda.synchronize()
        barrier(world)
        # one call at a time (srt_forward_host / srt_adjoint_host)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            plan.forward_host(f_h, p_h)
            plan.adjoint_host(y_h, a_h)
            _ = float(p_h[0, 0, 0, 0]) + float(a_h[0, 0, 0, 0])
        serial_s = reduce_max(time.perf_counter() - t0, world)
        # pipelined (srt_pipe_*): a call's input copy overlaps the earlier
        # calls' computation; every step's result is read on the host, `depth`
        # steps after it was submitted
        depth = min(3, max(1, args.e2e_depth))  # the pipe keeps the last 8 calls' events
        pipe = Pipeline(plan, B, slots=3)
        nbuf = depth + 1
        p2 = [p_h] + [torch.empty_like(p_h).pin_memory() for _ in range(depth)]
        a2 = [a_h] + [torch.empty_like(a_h).pin_memory() for _ in range(depth)]
        times = []  # each call's copies, transform and compute-stream idle time

        def submit(k):
            return (pipe.submit("forward", f_h, p2[k % nbuf]),
                    pipe.submit("adjoint", y_h, a2[k % nbuf]))

        def read(k, tickets):
            for t in tickets:
                pipe.wait(t)
            v = float(p2[k % nbuf][0, 0, 0, 0]) + float(a2[k % nbuf][0, 0, 0, 0])
            times.extend(pipe.stage_times(t) for t in tickets)
            return v

        read(1, submit(1))
        read(0, submit(0))
        times.clear()
        barrier(world)
        t0 = time.perf_counter()
        queue = []
        for k in range(args.e2e_steps):
            queue.append((k, submit(k)))
            if len(queue) > depth:
                read(*queue.pop(0))
        while queue:
            read(*queue.pop(0))
        e2e_s = reduce_max(time.perf_counter() - t0, world)
        names = ("h2d", "transform", "d2h", "compute_idle")
        # the pipe's own events: copies, transform, and the compute stream's
        # idle time before each transform, over the last 8 calls and all
        pipe_ms = {k: round(float(np.mean([x[i] for x in times[-8:]])), 3)
                   for i, k in enumerate(names)}
        pipe_all = {k: round(float(np.mean([x[i] for x in times])), 3)
                    for i, k in enumerate(names)}
        pipe_all["compute_idle_total_ms"] = round(float(np.sum([x[3] for x in times])), 2)
        pipe.close()
        e2e = {"value": world * args.e2e_steps * B / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": f_h.numel() * 4 + y_h.numel() * 4,
               "d2h_bytes_per_step": p_h.numel() * 4 + a_h.numel() * 4,
               "steps": args.e2e_steps,
               "api": "srt_pipe_submit / srt_pipe_wait, 3 slots (calls in flight)",
               "depth": depth,
               "pipe_ms_per_call_last8": pipe_ms,
               "pipe_ms_per_call_all": pipe_all,
               "one_call_at_a_time": world * args.e2e_steps * B / serial_s}

    launches = args.steps * (plan.launches_per_call(0, B) + plan.launches_per_call(1, B))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded phantoms and N(0,1) data, no dataset)",
           "config": workload_config(args.workload, geom, B, args.weights,
                                     {"l2": "flushed between steps (256 MiB write, untimed)",
                                      "parallelism": "replicas" if world > 1 else "single GPU",
                                      "plan_build_s": round(plan_s, 3),
                                      "nnz1": plan.info["nnz1"], "nnz2": plan.info["nnz2"],
                                      "a2_form": (f"Toeplitz taps ({plan.info['n_taps']} taps of T), "
                                                  + ("a warp per row" if args.rowwise
                                                     else "2 x 2 row tiles")
                                                  if plan.info["a2_taps"] else "CSR"),
                                      "a1_form": {0: "every column", 1: "the first n_phi/4 "
                                                  "columns, the rest by quarter turns",
                                                  2: "the first n_phi/8 + 1 columns, the rest by "
                                                  "quarter turns and the diagonal mirror"}[
                                                      plan.info["a1_rot"]]
                                                  + ("; a warp per row" if args.rowwise
                                                     else "; A1 a warp per row, A1^T 2 x 2-pixel "
                                                          "register tiles"),
                                      "reshapes": ", ".join(
                                          (["P1 fused into the A1 epilogue"] if fused_p1 else [])
                                          + (["P2 and P1^-1 fused into the A2 / A2^T epilogues"]
                                             if fused else []))
                                      or "four reshape kernels",
                                      "plan_device_gb": round(plan.info["device_bytes"] / 1e9, 3),
                                      "intermediate": ("piecewise linear in rho" if args.rho_linear
                                                       else "piecewise constant on radius bins"),
                                      "voxels": ("bilinear in (x, y) between voxel centres"
                                                 if args.voxel_linear
                                                 else "piecewise constant")}),
           "roofline": roof, "hbm": hbm, "stages": stages, "clocks": clk, "e2e": e2e,
           "gpu_launches": launches}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, n, t = cpu_oracle_rate(args.workload, 15.0, rho_linear=args.rho_linear,
                                            voxel_linear=args.voxel_linear)
        out["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle forward + adjoint over {n} seeded shells of "
                      f"{geom.n_phi * geom.n_zs * geom.n_ell} ({t:.1f} s); rate extrapolated "
                      f"to the full operator by shell count"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
