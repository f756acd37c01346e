"""Seeded synthetic inputs: workload presets, phantoms and probe data.

This module holds no arithmetic of the transform itself.  It only builds the
numbers fed to the transform (geometry sizes, voxel volumes, measurement-shaped
noise), so that the CUDA path and the FP64 oracle can be driven with identical
inputs.  Everything is deterministic given the seed (numpy PCG64).

Volume layout: ``f[ix, iy, iz]`` with voxel centres ``(i - (M-1)/2) * spacing``
(box centred at the origin, z fastest in memory).
"""
from __future__ import annotations

import math

import numpy as np

# Seeds used across tests, bench and serving.
SEED_PHANTOM = 0
SEED_PROBE = 1
SEED_FD = 2
SEED_SERVE = 3

# Workload presets: the sizes of the paper's problem statement (Algorithm 1
# inputs) for the five workloads this library is exercised on.  Only sizes;
# both the oracle and the CUDA plan derive radius/ring grids themselves.
WORKLOADS = {
    # 32^3 @ 0.5 mm, R = 12 mm, 64 columns, 32 rings, 96 radius bins; 5 balls.
    "srt32": dict(ms=32, mz=32, dxy=0.5, dz=0.5, radius=12.0, n_phi=64, n_zs=32, n_ell=96,
                  n_balls=5, n_blobs=0),
    # 128^3 @ 0.2 mm, R = 20 mm, 256/128/512; 40 balls + 200-blob vessel tree.
    "srt128": dict(ms=128, mz=128, dxy=0.2, dz=0.2, radius=20.0, n_phi=256, n_zs=128, n_ell=512,
                   n_balls=40, n_blobs=200),
    # 256^3 @ 0.1 mm, R = 20 mm, 256/256/768; 100 balls + 500-blob vessel tree.
    "srt256": dict(ms=256, mz=256, dxy=0.1, dz=0.1, radius=20.0, n_phi=256, n_zs=256, n_ell=768,
                   n_balls=100, n_blobs=500),
    # 16^3 finite-difference gradient-check geometry (0.5 mm, R = 12 mm).
    "srt16fd": dict(ms=16, mz=16, dxy=0.5, dz=0.5, radius=12.0, n_phi=32, n_zs=16, n_ell=48,
                    n_balls=3, n_blobs=0),
}


def serving_geometry(edge: int, n_phi: int) -> dict:
    """Serving mix geometry: 25.6 mm field of view, R = 20 mm, rings = edge,
    radius bins = 4 * edge."""
    d = 25.6 / edge
    return dict(ms=edge, mz=edge, dxy=d, dz=d, radius=20.0, n_phi=n_phi, n_zs=edge,
                n_ell=4 * edge, n_balls=8, n_blobs=0)


def sizes(name_or_dict) -> dict:
    w = WORKLOADS[name_or_dict] if isinstance(name_or_dict, str) else name_or_dict
    return {k: w[k] for k in ("ms", "mz", "dxy", "dz", "radius", "n_phi", "n_zs", "n_ell")}


def _axis(m: int, d: float) -> np.ndarray:
    return (np.arange(m) - (m - 1) / 2.0) * d


def add_ball(f: np.ndarray, dxy: float, dz: float, centre, a: float, amp: float,
             sub: int = 4) -> None:
    """Add amp * (fraction of each voxel inside the ball) to f, in place.
    Voxels cut by the sphere are sub-sampled sub^3 times."""
    ms, _, mz = f.shape
    cx, cy, cz = centre
    xs, zs = _axis(ms, dxy), _axis(mz, dz)
    ix = np.nonzero(np.abs(xs - cx) <= a + dxy)[0]
    iy = np.nonzero(np.abs(xs - cy) <= a + dxy)[0]
    iz = np.nonzero(np.abs(zs - cz) <= a + dz)[0]
    if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
        return
    X = xs[ix][:, None, None] - cx
    Y = xs[iy][None, :, None] - cy
    Z = zs[iz][None, None, :] - cz
    r = np.sqrt(X * X + Y * Y + Z * Z)
    half = 0.5 * math.sqrt(2 * dxy * dxy + dz * dz)
    frac = (r <= a - half).astype(np.float64)
    cut = np.nonzero((r > a - half) & (r < a + half))
    if len(cut[0]):
        o = (np.arange(sub) + 0.5) / sub - 0.5
        ox = o[:, None, None] * dxy
        oy = o[None, :, None] * dxy
        oz = o[None, None, :] * dz
        bx = X[cut[0], 0, 0]
        by = Y[0, cut[1], 0]
        bz = Z[0, 0, cut[2]]
        inside = ((bx[:, None, None, None] + ox) ** 2 + (by[:, None, None, None] + oy) ** 2
                  + (bz[:, None, None, None] + oz) ** 2) <= a * a
        frac[cut] = inside.reshape(len(bx), -1).mean(axis=1)
    f[np.ix_(ix, iy, iz)] += amp * frac


def balls(ms, mz, dxy, dz, n, rng, r_lo=1.0, r_hi=4.0, a_lo=0.2, a_hi=1.0, sub=4):
    """n uniform balls, radii U[r_lo, r_hi] mm, amplitudes U[a_lo, a_hi],
    centres drawn so that each ball lies fully inside the box."""
    f = np.zeros((ms, ms, mz), dtype=np.float64)
    hx, hz = 0.5 * ms * dxy, 0.5 * mz * dz
    out = []
    for _ in range(n):
        a = rng.uniform(r_lo, min(r_hi, 0.95 * min(hx, hz)))
        amp = rng.uniform(a_lo, a_hi)
        c = (rng.uniform(-hx + a, hx - a), rng.uniform(-hx + a, hx - a), rng.uniform(-hz + a, hz - a))
        add_ball(f, dxy, dz, c, a, amp, sub)
        out.append((c, a, amp))
    return f, out


def vessel_tree(ms, mz, dxy, dz, n_blobs, rng, s_lo=0.2, s_hi=0.8, a_lo=0.2, a_hi=1.0,
                p_branch=0.05, jitter=0.35):
    """Gaussian-blob vessel tree: a seeded branching random walk of blob
    centres (step = mean sigma, angular jitter, branch probability p_branch),
    isotropic Gaussians sampled at voxel centres."""
    f = np.zeros((ms, ms, mz), dtype=np.float64)
    if n_blobs <= 0:
        return f
    hx, hz = 0.5 * ms * dxy, 0.5 * mz * dz
    xs, zs = _axis(ms, dxy), _axis(mz, dz)
    step = 0.5 * (s_lo + s_hi)

    def unit(v):
        return v / max(np.linalg.norm(v), 1e-12)

    heads = [(np.array([rng.uniform(-0.6, 0.6) * hx, rng.uniform(-0.6, 0.6) * hx,
                        rng.uniform(-0.6, 0.6) * hz]), unit(rng.standard_normal(3)))]
    placed = 0
    while placed < n_blobs:
        if not heads:
            heads.append((np.array([rng.uniform(-0.6, 0.6) * hx, rng.uniform(-0.6, 0.6) * hx,
                                    rng.uniform(-0.6, 0.6) * hz]), unit(rng.standard_normal(3))))
        pos, d = heads.pop(0)
        s = rng.uniform(s_lo, s_hi)
        amp = rng.uniform(a_lo, a_hi)
        w = 4.0 * s
        gx = np.exp(-0.5 * ((xs - pos[0]) / s) ** 2) * (np.abs(xs - pos[0]) <= w)
        gy = np.exp(-0.5 * ((xs - pos[1]) / s) ** 2) * (np.abs(xs - pos[1]) <= w)
        gz = np.exp(-0.5 * ((zs - pos[2]) / s) ** 2) * (np.abs(zs - pos[2]) <= w)
        ix, iy, iz = np.nonzero(gx)[0], np.nonzero(gy)[0], np.nonzero(gz)[0]
        if len(ix) and len(iy) and len(iz):
            f[np.ix_(ix, iy, iz)] += amp * (gx[ix][:, None, None] * gy[iy][None, :, None]
                                            * gz[iz][None, None, :])
        placed += 1
        nd = unit(d + jitter * rng.standard_normal(3))
        npos = pos + step * nd
        lim = np.array([hx, hx, hz]) * 0.9
        bounce = np.abs(npos) > lim
        nd[bounce] *= -1.0
        npos = np.clip(npos, -lim, lim)
        heads.append((npos, nd))
        if rng.random() < p_branch:
            heads.append((npos.copy(), unit(np.cross(nd, rng.standard_normal(3)))))
    return f


def phantom(name_or_dict, seed: int = SEED_PHANTOM, sub: int = 4) -> np.ndarray:
    """Ball phantom (+ vessel tree when the workload has blobs), FP64."""
    w = WORKLOADS[name_or_dict] if isinstance(name_or_dict, str) else name_or_dict
    rng = np.random.default_rng(seed)
    f, _ = balls(w["ms"], w["mz"], w["dxy"], w["dz"], w.get("n_balls", 5), rng, sub=sub)
    if w.get("n_blobs", 0):
        f += vessel_tree(w["ms"], w["mz"], w["dxy"], w["dz"], w["n_blobs"], rng)
    return f


def probe(name_or_dict, seed: int = SEED_PROBE) -> np.ndarray:
    """N(0, 1) data of measurement shape (n_phi, n_zs, n_ell), FP64."""
    w = WORKLOADS[name_or_dict] if isinstance(name_or_dict, str) else name_or_dict
    rng = np.random.default_rng(seed)
    return rng.standard_normal((w["n_phi"], w["n_zs"], w["n_ell"]))


def crop_phantom(name_or_dict, crop: int, seed: int = SEED_PHANTOM) -> np.ndarray:
    """Phantom that is zero outside the central crop^3 voxels."""
    f = phantom(name_or_dict, seed)
    ms, _, mz = f.shape
    a, b = (ms - crop) // 2, (mz - crop) // 2
    out = np.zeros_like(f)
    out[a:a + crop, a:a + crop, b:b + crop] = f[a:a + crop, a:a + crop, b:b + crop]
    return out
