"""Closed forms used to pin the oracle (test helpers, independent of it).

The arc of a circle inside an axis-parallel rectangle is computed here by the
quadrant-interval method: in each quarter of the circle both cos and sin are
monotone, so the angles whose x (resp. y) coordinate lies in the rectangle
form one interval per quarter, given by acos/asin of the edge offsets.  The
oracle instead sorts grid-line crossings and tests segment midpoints.
"""
from __future__ import annotations

import math

import numpy as np

PI = math.pi


def _acos_r(u: float, r: float) -> float:
    """Angle in [0, pi] whose cosine is u/r (clamped)."""
    if u >= r:
        return 0.0
    if u <= -r:
        return PI
    return math.atan2(math.sqrt((r - u) * (r + u)), u)


def _asin_r(u: float, r: float) -> float:
    """Angle in [-pi/2, pi/2] whose sine is u/r (clamped)."""
    if u >= r:
        return 0.5 * PI
    if u <= -r:
        return -0.5 * PI
    return math.atan2(u, math.sqrt((r - u) * (r + u)))


def _ov(*iv):
    lo = max(a for a, _ in iv)
    hi = min(b for _, b in iv)
    return max(0.0, hi - lo)


def arc_circle_rect(cx, cy, r, x0, x1, y0, y1) -> float:
    """Length of the circle (cx, cy, r) inside [x0, x1] x [y0, y1]."""
    a1, a0 = _acos_r(x1 - cx, r), _acos_r(x0 - cx, r)
    s0, s1 = _asin_r(y0 - cy, r), _asin_r(y1 - cy, r)
    t = 0.0
    t += _ov((0.0, 0.5 * PI), (a1, a0), (s0, s1))                    # first quarter
    t += _ov((0.5 * PI, PI), (a1, a0), (PI - s1, PI - s0))            # second
    t += _ov((-PI, -0.5 * PI), (-a0, -a1), (-PI - s1, -PI - s0))      # third
    t += _ov((-0.5 * PI, 0.0), (-a0, -a1), (s0, s1))                  # fourth
    return r * t


def arc_circle_rect_v(cx, cy, r, x0, x1, y0, y1) -> np.ndarray:
    """arc_circle_rect over numpy arrays (broadcast).  The clamps of the
    scalar version come from sqrt(max((r - u)(r + u), 0)) being 0 beyond the
    circle: atan2 then gives 0 / pi resp. +-pi/2 there."""
    def acos_r(u):
        return np.arctan2(np.sqrt(np.maximum((r - u) * (r + u), 0.0)), u)

    def asin_r(u):
        return np.arctan2(u, np.sqrt(np.maximum((r - u) * (r + u), 0.0)))

    def ov(lo, hi):
        return np.maximum(0.0, hi - lo)

    a1, a0 = acos_r(np.asarray(x1) - cx), acos_r(np.asarray(x0) - cx)
    s0, s1 = asin_r(np.asarray(y0) - cy), asin_r(np.asarray(y1) - cy)
    hp = 0.5 * PI
    t = ov(np.maximum(0.0, np.maximum(a1, s0)), np.minimum(hp, np.minimum(a0, s1)))
    t = t + ov(np.maximum(hp, np.maximum(a1, PI - s1)), np.minimum(PI, np.minimum(a0, PI - s0)))
    t = t + ov(np.maximum(-PI, np.maximum(-a0, -PI - s1)), np.minimum(-hp, np.minimum(-a1, -PI - s0)))
    t = t + ov(np.maximum(-hp, np.maximum(-a0, s0)), np.minimum(0.0, np.minimum(-a1, s1)))
    return r * t


def _ov_iv(*iv):
    lo = max(a for a, _ in iv)
    hi = min(b for _, b in iv)
    return (lo, hi) if hi > lo else None


def moment_circle_rect(cx, cy, r, x0, x1, y0, y1) -> float:
    """int y ds over the part of the circle (cx, cy, r) inside [x0, x1] x
    [y0, y1]: on each quarter interval [t0, t1] of t (x = cx + r cos t,
    y = cy + r sin t), r cy (t1 - t0) + r^2 (cos t0 - cos t1)."""
    a1, a0 = _acos_r(x1 - cx, r), _acos_r(x0 - cx, r)
    s0, s1 = _asin_r(y0 - cy, r), _asin_r(y1 - cy, r)
    ivs = [_ov_iv((0.0, 0.5 * PI), (a1, a0), (s0, s1)),
           _ov_iv((0.5 * PI, PI), (a1, a0), (PI - s1, PI - s0)),
           _ov_iv((-PI, -0.5 * PI), (-a0, -a1), (-PI - s1, -PI - s0)),
           _ov_iv((-0.5 * PI, 0.0), (-a0, -a1), (s0, s1))]
    m = 0.0
    for iv in ivs:
        if iv is not None:
            t0, t1 = iv
            m += r * cy * (t1 - t0) + r * r * (math.cos(t0) - math.cos(t1))
    return m


def hat_weight_semicircle(zh, ell, z0, z1, nodes, lo, hi, l) -> float:
    """The hat of radius node l (piecewise-linear interpolation between the
    nodes, constant below the first and above the last, zero outside
    [lo, hi]) integrated along the (z, rho) semicircle of ring zh and radius
    ell inside the slab [z0, z1]."""
    n, dl = len(nodes), nodes[1] - nodes[0] if len(nodes) > 1 else hi - lo
    rl = nodes[l]
    acc = 0.0
    if l == 0:
        acc += arc_circle_rect(zh, 0.0, ell, z0, z1, lo, rl)
    else:
        ra = nodes[l - 1]
        L = arc_circle_rect(zh, 0.0, ell, z0, z1, ra, rl)
        M = moment_circle_rect(zh, 0.0, ell, z0, z1, ra, rl)
        acc += (M - ra * L) / dl
    if l == n - 1:
        acc += arc_circle_rect(zh, 0.0, ell, z0, z1, rl, hi)
    else:
        rb = nodes[l + 1]
        L = arc_circle_rect(zh, 0.0, ell, z0, z1, rl, rb)
        M = moment_circle_rect(zh, 0.0, ell, z0, z1, rl, rb)
        acc += (rb * L - M) / dl
    return acc


def ball_srt(sensor, centre, a, amp, ell) -> np.ndarray:
    """Closed-form SRT of a uniform ball: area of the spherical cap of the shell
    |x - sensor| = ell inside the ball, times amp.  Cap area 2*pi*ell*h with
    h = ell - (d^2 + ell^2 - a^2) / (2 d) = (a^2 - (d - ell)^2) / (2 d)."""
    d = float(np.linalg.norm(np.asarray(sensor) - np.asarray(centre)))
    ell = np.asarray(ell, dtype=np.float64)
    val = amp * PI * ell * (a * a - (d - ell) ** 2) / d
    return np.where(np.abs(d - ell) <= a, val, 0.0)


def geometry_numbers(ms, mz, dxy, dz, radius, n_phi, n_zs, n_ell, phi0=0.0):
    """Grid positions under the stated readings (cell-centred radii and rings,
    centred voxel box)."""
    H, L = mz * dz, ms * dxy
    rxy = L / math.sqrt(2.0)
    lo, hi = radius - rxy, radius + rxy
    dl = (hi - lo) / n_ell
    return dict(
        L=L, H=H, lo=lo, hi=hi, dl=dl,
        ell=lo + (np.arange(n_ell) + 0.5) * dl,
        edges=lo + np.arange(n_ell + 1) * dl,
        zh=-0.5 * H + (np.arange(n_zs) + 0.5) * H / n_zs,
        zb=-0.5 * H + np.arange(mz + 1) * dz,
        xb=-0.5 * L + np.arange(ms + 1) * dxy,
        phi=phi0 + 2 * PI * np.arange(n_phi) / n_phi,
    )
