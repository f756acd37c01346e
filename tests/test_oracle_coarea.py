"""Coarea pins of the oracle's matrix entries (CPU only).

The distance from a point has gradient of length one, so by the coarea
formula the area of a region equals the integral over rho of the length of
the circle of radius rho inside it.  The oracle's entries are such lengths
sampled at the radius nodes of Sec. 3.1 (exact arc lengths on the shared
radius grid), so dl times a sum of entries over the radius index is a
midpoint rule for an area that is known independently:
  * A1 (in-plane circles, Sec. 3.1): dl * sum_l A1[(j, l), pixel] -> dxy^2,
    every pixel lying inside the annulus [lo, hi] around every sensor;
  * A2 ((z, rho) semicircles): dl * sum_m of the entries of shell row
    (h, m) in slab k and a band of radius bins -> the area of slab x band
    inside the disk of radius hi around the ring (the rows' radii fill
    [lo, hi]; distances below lo cannot occur in the band rho >= lo).
In the piecewise-linear mode the hats of one slab add up to the arc length
inside [lo, hi], so the same area holds for the whole band.
The lengths have square-root behaviour where a circle touches a cell edge,
so the rule converges at order about 1.5 in the worst cell, not 2; the
gates ask for steady decrease and better than first order overall.
"""
import math

import numpy as np
import pytest
from scipy import integrate


def _geom(orc, n_ell, rho_linear=False):
    ms, dxy, R = 5, 0.6, 3.0
    rxy = ms * dxy / math.sqrt(2)
    return orc.OracleGeometry(ms, 4, dxy, 0.45, R, 6, 0.37, 3, -0.7, 1.1, n_ell, R - rxy,
                              R + rxy, rho_linear)


LADDER = (24, 48, 96, 192, 384)


def _gate(errs, ratio, total, finest):
    for a, b in zip(errs, errs[1:]):
        assert b < ratio * a, errs
    assert errs[0] / errs[-1] >= total, errs
    assert errs[-1] < finest, errs


def test_a1_columns_sum_to_the_pixel_area(orc):
    errs = []
    for n in LADDER:
        g = _geom(orc, n)
        dl = (g.ell_hi - g.ell_lo) / n
        worst = 0.0
        for j in range(g.n_phi):
            col = np.zeros(g.ms * g.ms)
            for l in range(n):
                for pix, x in orc.circle_arcs(g, j, l).items():
                    col[pix] += x
            worst = max(worst, np.abs(dl * col - g.dxy ** 2).max() / g.dxy ** 2)
        errs.append(worst)
    # measured: 0.18, 0.081, 0.033, 0.011, 0.0053
    _gate(errs, ratio=0.6, total=16.0, finest=1e-2)


def _band_area(u0, u1, ra, rb, hi):
    """Area of {u in [u0, u1], rho in [ra, rb], u^2 + rho^2 <= hi^2}."""
    def width(u):
        top = min(rb, math.sqrt(max(hi * hi - u * u, 0.0)))
        return max(0.0, top - ra)
    kinks = [s * math.sqrt(max(hi * hi - r * r, 0.0)) for r in (ra, rb) for s in (-1.0, 1.0)]
    pts = [p for p in kinks if u0 < p < u1]
    return integrate.quad(width, u0, u1, points=pts or None, epsabs=1e-14, epsrel=1e-13,
                          limit=200)[0]


@pytest.mark.parametrize("rho_linear", [False, True])
def test_a2_slab_band_sums_give_the_area(orc, rho_linear):
    nb = 1 if rho_linear else 4        # bands of radius bins (the hats spill across bands)
    errs = []
    for n in LADDER:
        g = _geom(orc, n, rho_linear)
        lo, hi = g.ell_lo, g.ell_hi
        dl = (hi - lo) / n
        H = g.mz * g.dz
        zb = -H / 2 + np.arange(g.mz + 1) * g.dz
        zh = g.zs_lo + (np.arange(g.n_zs) + 0.5) * (g.zs_hi - g.zs_lo) / g.n_zs
        worst = 0.0
        for h in range(g.n_zs):
            acc = np.zeros((nb, g.mz))
            for m in range(n):
                for cell, x in orc.semicircle_arcs(g, h, m).items():
                    l, k = divmod(cell, g.mz)
                    acc[l * nb // n, k] += x
            for b in range(nb):
                ra, rb = lo + b * (hi - lo) / nb, lo + (b + 1) * (hi - lo) / nb
                for k in range(g.mz):
                    area = _band_area(zb[k] - zh[h], zb[k + 1] - zh[h], ra, rb, hi)
                    worst = max(worst, abs(dl * acc[b, k] - area) / (g.dz * (rb - ra)))
        errs.append(worst)
    # measured: constant 0.048 -> 0.0011, linear 0.0066 -> 0.00013
    _gate(errs, ratio=0.65, total=16.0, finest=3e-3 if not rho_linear else 1e-3)
