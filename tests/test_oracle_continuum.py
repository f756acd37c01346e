"""Pins of the oracle against the continuous transform and brute-force sampling.

* Closed-form ball (Sec. 2, SRT definition): the SRT of a uniform ball is the
  area of the shell's cap inside the ball.  The oracle on a partial-volume
  voxelised ball must approach it as the voxel size and the radius step are
  halved (discretisation error of piecewise-constant voxels and of the
  radius-snapped intermediate of Algorithm 1).
* Brute-force shell sampling (Sec. 2 spherical parametrisation, with the
  in-plane radius snapped to the shared radius grid as Algorithm 1 does):
  midpoint sampling of t and a with no knowledge of grid crossings converges
  to the oracle's exact segment sums as the sample count grows.
"""
import math

import numpy as np

from paper_2402_15641_gb300 import inputs as I
from tests.closed_forms import ball_srt


def test_ball_convergence_ladder(orc):
    c, a, amp = (1.3, -0.7, 0.9), 3.0, 1.0
    js, n_zs = [0, 5, 11], 8
    errs = []
    for lev in range(3):
        s = 2 ** lev
        ms, d = 32 * s, 0.5 / s
        g = orc.OracleGeometry.default(ms, ms, d, d, 12.0, 64, n_zs, 96 * s)
        f = np.zeros(g.f_shape)
        I.add_ball(f, d, d, c, a, amp, sub=8 if lev < 2 else 4)
        sh = np.array([[j, h, m] for j in js for h in range(n_zs) for m in range(g.n_ell)])
        p = orc.forward_shells(g, f, sh)
        ell = g.ell_lo + (np.arange(g.n_ell) + 0.5) * (g.ell_hi - g.ell_lo) / g.n_ell
        zh = g.zs_lo + (np.arange(n_zs) + 0.5) * (g.zs_hi - g.zs_lo) / n_zs
        want = np.concatenate([
            ball_srt((12 * math.cos(2 * math.pi * j / 64), 12 * math.sin(2 * math.pi * j / 64),
                      zh[h]), c, a, amp, ell)
            for j in js for h in range(n_zs)])
        errs.append(np.linalg.norm(p - want) / np.linalg.norm(want))
    assert errs[0] < 0.03, errs
    assert errs[1] < 0.5 * errs[0], errs
    assert errs[2] < 0.5 * errs[1], errs


def _brute(g, f, n_t, n_a):
    """Snapped shell integral by midpoint sampling: for each t-sample the
    in-plane radius is the centre of the bin holding l_m sin t; the in-plane
    circle integral is sampled at n_a angles with nearest-voxel lookup."""
    L, H = g.ms * g.dxy, g.mz * g.dz
    dl = (g.ell_hi - g.ell_lo) / g.n_ell
    ell = g.ell_lo + (np.arange(g.n_ell) + 0.5) * dl
    zh = g.zs_lo + (np.arange(g.n_zs) + 0.5) * (g.zs_hi - g.zs_lo) / g.n_zs
    phi = g.phi0 + 2 * math.pi * np.arange(g.n_phi) / g.n_phi
    a = (np.arange(n_a) + 0.5) * (2 * math.pi / n_a)
    ff = f.reshape(g.ms * g.ms, g.mz)
    circ = np.zeros((g.n_phi, g.n_ell, g.mz))   # sampled circle integrals
    for j in range(g.n_phi):
        sx, sy = g.radius * math.cos(phi[j]), g.radius * math.sin(phi[j])
        for l in range(g.n_ell):
            x = sx + ell[l] * np.cos(a)
            y = sy + ell[l] * np.sin(a)
            ix = np.floor((x + L / 2) / g.dxy).astype(np.int64)
            iy = np.floor((y + L / 2) / g.dxy).astype(np.int64)
            ok = (ix >= 0) & (ix < g.ms) & (iy >= 0) & (iy < g.ms)
            circ[j, l] = ell[l] * (2 * math.pi / n_a) * ff[ix[ok] * g.ms + iy[ok]].sum(axis=0)
    t = (np.arange(n_t) + 0.5) * (math.pi / n_t)
    p = np.zeros(g.p_shape)
    for h in range(g.n_zs):
        for m in range(g.n_ell):
            z = zh[h] + ell[m] * np.cos(t)
            rho = ell[m] * np.sin(t)
            k = np.floor((z + H / 2) / g.dz).astype(np.int64)
            l = np.floor((rho - g.ell_lo) / dl).astype(np.int64)
            ok = (k >= 0) & (k < g.mz) & (l >= 0) & (l < g.n_ell)
            p[:, h, m] = ell[m] * (math.pi / n_t) * circ[:, l[ok], k[ok]].sum(axis=1)
    return p


def test_bruteforce_sampling_converges_to_oracle(orc):
    rxy = 6 * 0.55 / math.sqrt(2)
    g = orc.OracleGeometry(6, 5, 0.55, 0.4, 3.5, 5, 0.21, 4, -0.9, 0.8, 14, 3.5 - rxy, 3.5 + rxy)
    rng = np.random.default_rng(21)
    f = rng.uniform(0.0, 1.0, g.f_shape)
    p = orc.forward(g, f)
    errs = []
    for n in (4000, 32000, 256000):
        pb = _brute(g, f, n, n)
        errs.append(np.linalg.norm(pb - p) / np.linalg.norm(p))
    assert errs[0] < 2e-3, errs
    assert errs[1] < 0.25 * errs[0], errs
    assert errs[2] < 0.25 * errs[1], errs
    assert errs[2] < 5e-5, errs
