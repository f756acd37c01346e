"""Pins of the oracle's piecewise-linear intermediate (CPU only).

The paper discretises the intermediate f^{1,2} with piecewise-constant cells
and notes that its algorithms carry over to other bases, naming
piecewise-linear ones (Sec. 3.1).  With rho_linear, f^{1,2} is interpolated
linearly in rho between the radius-bin centres (held constant from lo to the
first centre and from the last centre to hi).  Each part of that mode is fixed
by a fact independent of the oracle's code:
  * semicircle weights = the node's hat integrated along the arc in the slab,
    from the quadrant-interval closed forms of the arc length and of
    int rho ds (tests/closed_forms.py);
  * the hats sum to one on [lo, hi], so per slab the weights add up to the
    piecewise-constant ones (the arc length inside the slab and [lo, hi]);
  * a separable volume reproduced from closed forms (composition);
  * per-voxel weights by the second, box-by-box route; the adjoint identity;
  * brute-force midpoint sampling of the interpolated shell integral;
  * the closed-form SRT of a uniform ball, approached as the grid is refined.
"""
import math

import numpy as np
import pytest

from paper_2402_15641_gb300 import inputs as I
from tests.closed_forms import arc_circle_rect, ball_srt, hat_weight_semicircle


def _tiny(O, **kw):
    d = dict(ms=5, mz=4, dxy=0.6, dz=0.45, radius=3.0, n_phi=6, phi0=0.37, n_zs=3,
             zs_lo=-0.7, zs_hi=1.1, n_ell=12)
    d.update(kw)
    rxy = d["ms"] * d["dxy"] / math.sqrt(2)
    return O.OracleGeometry(d["ms"], d["mz"], d["dxy"], d["dz"], d["radius"], d["n_phi"],
                            d["phi0"], d["n_zs"], d["zs_lo"], d["zs_hi"], d["n_ell"],
                            d["radius"] - rxy, d["radius"] + rxy, True)


def _grid(g):
    L, H = g.ms * g.dxy, g.mz * g.dz
    dl = (g.ell_hi - g.ell_lo) / g.n_ell
    return dict(
        xb=-0.5 * L + np.arange(g.ms + 1) * g.dxy,
        zb=-0.5 * H + np.arange(g.mz + 1) * g.dz,
        ell=g.ell_lo + (np.arange(g.n_ell) + 0.5) * dl,
        zh=g.zs_lo + (np.arange(g.n_zs) + 0.5) * (g.zs_hi - g.zs_lo) / g.n_zs,
        phi=g.phi0 + 2 * math.pi * np.arange(g.n_phi) / g.n_phi,
    )


def test_semicircle_hat_weights_closed_form(orc):
    """Includes rings at the slab centres (n_zs = mz over the volume height):
    there every semicircle's slab breaks are symmetric about its top, where it
    touches its own radius node, the case a t-midpoint test misplaces."""
    for g in (_tiny(orc), _tiny(orc, n_ell=1), _tiny(orc, n_ell=2, zs_lo=-0.9, zs_hi=0.9),
              _tiny(orc, n_zs=4, zs_lo=-0.9, zs_hi=0.9),
              _tiny(orc, mz=5, n_zs=5, zs_lo=-1.125, zs_hi=1.125, n_ell=7)):
        G = _grid(g)
        checked = 0
        for h in range(g.n_zs):
            for m in range(g.n_ell):
                got = orc.semicircle_arcs(g, h, m)
                for l in range(g.n_ell):
                    for k in range(g.mz):
                        want = hat_weight_semicircle(G["zh"][h], G["ell"][m], G["zb"][k],
                                                     G["zb"][k + 1], G["ell"], g.ell_lo,
                                                     g.ell_hi, l)
                        have = got.get(l * g.mz + k, 0.0)
                        assert abs(have - want) <= 1e-12 * G["ell"][m], (h, m, l, k, have, want)
                        checked += want > 0
        assert checked > 0


def test_hats_partition_unity_per_slab(orc):
    """Per slab the hat weights add up to the arc length inside the slab and
    [lo, hi], i.e. to the piecewise-constant weights' sum."""
    g = _tiny(orc, n_ell=9)
    gc = orc.OracleGeometry(*[getattr(g, k) for k in (
        "ms", "mz", "dxy", "dz", "radius", "n_phi", "phi0", "n_zs", "zs_lo", "zs_hi", "n_ell",
        "ell_lo", "ell_hi")])
    G = _grid(g)
    for h in range(g.n_zs):
        for m in range(g.n_ell):
            lin, con = orc.semicircle_arcs(g, h, m), orc.semicircle_arcs(gc, h, m)
            for k in range(g.mz):
                sl = sum(v for c, v in lin.items() if c % g.mz == k)
                sc = sum(v for c, v in con.items() if c % g.mz == k)
                band = arc_circle_rect(G["zh"][h], 0.0, G["ell"][m], G["zb"][k], G["zb"][k + 1],
                                       g.ell_lo, g.ell_hi)
                assert abs(sl - sc) <= 1e-12 * G["ell"][m]
                assert abs(sl - band) <= 1e-12 * G["ell"][m]


def test_separable_volume_closed_form(orc):
    """f[ix, iy, k] = q[ix, iy] s[k]: p[j,h,m] = sum_{k,l} s[k] hat2(h,m; k,l)
    sum_pix q[pix] arc1(j,l; pix), every factor in closed form."""
    g = _tiny(orc)
    G = _grid(g)
    rng = np.random.default_rng(5)
    q = rng.uniform(0.1, 1.0, (g.ms, g.ms))
    s = rng.uniform(0.1, 1.0, g.mz)
    p = orc.forward(g, q[:, :, None] * s[None, None, :])
    c1 = np.zeros((g.n_phi, g.n_ell))
    for j in range(g.n_phi):
        sx, sy = g.radius * math.cos(G["phi"][j]), g.radius * math.sin(G["phi"][j])
        for l in range(g.n_ell):
            c1[j, l] = sum(q[ix, iy] * arc_circle_rect(sx, sy, G["ell"][l], G["xb"][ix],
                                                       G["xb"][ix + 1], G["xb"][iy],
                                                       G["xb"][iy + 1])
                           for ix in range(g.ms) for iy in range(g.ms))
    want = np.zeros(g.p_shape)
    for h in range(g.n_zs):
        for m in range(g.n_ell):
            a2 = np.array([[hat_weight_semicircle(G["zh"][h], G["ell"][m], G["zb"][k],
                                                  G["zb"][k + 1], G["ell"], g.ell_lo, g.ell_hi, l)
                            for k in range(g.mz)] for l in range(g.n_ell)])
            want[:, h, m] = c1 @ (a2 @ s)
    assert np.max(np.abs(p - want)) <= 1e-12 * np.max(np.abs(want))
    assert np.count_nonzero(want) > 0.3 * want.size


@pytest.mark.parametrize("centred", [False, True])
def test_point_weights_adjoint_identity(orc, centred):
    g = _tiny(orc, ms=6, mz=5, n_ell=14, **(dict(n_zs=5, zs_lo=-1.125, zs_hi=1.125)
                                           if centred else {}))
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(8):
        j, h, m = int(rng.integers(g.n_phi)), int(rng.integers(g.n_zs)), int(rng.integers(g.n_ell))
        w = orc.shell_weights(g, j, h, m)
        for ix in range(g.ms):
            for iy in range(g.ms):
                for k in range(g.mz):
                    pw = orc.point_weight(g, j, h, m, ix, iy, k)
                    assert abs(pw - w.get((ix * g.ms + iy) * g.mz + k, 0.0)) <= 1e-12
                    checked += pw != 0.0
    assert checked > 20
    f = rng.standard_normal(g.f_shape)
    y = rng.standard_normal(g.p_shape)
    af, aty = orc.forward(g, f), orc.adjoint(g, y)
    lhs, rhs = float(np.sum(af * y)), float(np.sum(f * aty))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(af) * np.linalg.norm(y)
    vox = np.array([[1, 2, 3], [4, 0, 1], [5, 5, 4], [2, 3, 0]])
    got = orc.adjoint_voxels(g, y, vox)
    assert np.max(np.abs(got - aty[vox[:, 0], vox[:, 1], vox[:, 2]])) <= 1e-11 * np.max(np.abs(aty))


def _brute_linear(g, f, n_t, n_a):
    """The interpolated shell integral by midpoint sampling: in-plane circle
    integrals sampled at the node radii (n_a angles, nearest voxel), then, per
    t-sample, linear interpolation in rho = l sin t between nodes (constant
    below the first and above the last node, zero outside [lo, hi])."""
    L, H = g.ms * g.dxy, g.mz * g.dz
    dl = (g.ell_hi - g.ell_lo) / g.n_ell
    ell = g.ell_lo + (np.arange(g.n_ell) + 0.5) * dl
    zh = g.zs_lo + (np.arange(g.n_zs) + 0.5) * (g.zs_hi - g.zs_lo) / g.n_zs
    phi = g.phi0 + 2 * math.pi * np.arange(g.n_phi) / g.n_phi
    a = (np.arange(n_a) + 0.5) * (2 * math.pi / n_a)
    ff = f.reshape(g.ms * g.ms, g.mz)
    circ = np.zeros((g.n_phi, g.n_ell, g.mz))
    for j in range(g.n_phi):
        sx, sy = g.radius * math.cos(phi[j]), g.radius * math.sin(phi[j])
        for l in range(g.n_ell):
            x, y = sx + ell[l] * np.cos(a), sy + ell[l] * np.sin(a)
            ix = np.floor((x + L / 2) / g.dxy).astype(np.int64)
            iy = np.floor((y + L / 2) / g.dxy).astype(np.int64)
            ok = (ix >= 0) & (ix < g.ms) & (iy >= 0) & (iy < g.ms)
            circ[j, l] = ell[l] * (2 * math.pi / n_a) * ff[ix[ok] * g.ms + iy[ok]].sum(axis=0)
    t = (np.arange(n_t) + 0.5) * (math.pi / n_t)
    p = np.zeros(g.p_shape)
    for h in range(g.n_zs):
        for m in range(g.n_ell):
            z, rho = zh[h] + ell[m] * np.cos(t), ell[m] * np.sin(t)
            k = np.floor((z + H / 2) / g.dz).astype(np.int64)
            ok = (k >= 0) & (k < g.mz) & (rho > g.ell_lo) & (rho < g.ell_hi)
            u = np.clip((rho[ok] - ell[0]) / dl, 0.0, g.n_ell - 1)
            l0 = np.minimum(np.floor(u).astype(np.int64), max(g.n_ell - 2, 0))
            fr = u - l0
            l1 = np.minimum(l0 + 1, g.n_ell - 1)
            vals = (1 - fr) * circ[:, l0, k[ok]] + fr * circ[:, l1, k[ok]]
            p[:, h, m] = ell[m] * (math.pi / n_t) * vals.sum(axis=1)
    return p


def test_bruteforce_sampling_converges_to_oracle(orc):
    rxy = 6 * 0.55 / math.sqrt(2)
    g = orc.OracleGeometry(6, 5, 0.55, 0.4, 3.5, 5, 0.21, 4, -0.9, 0.8, 14, 3.5 - rxy, 3.5 + rxy,
                           True)
    f = np.random.default_rng(21).uniform(0.0, 1.0, g.f_shape)
    p = orc.forward(g, f)
    errs = []
    for n in (4000, 32000, 256000):
        pb = _brute_linear(g, f, n, n)
        errs.append(np.linalg.norm(pb - p) / np.linalg.norm(p))
    assert errs[0] < 2e-3, errs
    assert errs[1] < 0.25 * errs[0], errs
    assert errs[2] < 0.25 * errs[1], errs
    assert errs[2] < 5e-5, errs


def test_ball_convergence_ladder(orc):
    c, a, amp = (1.3, -0.7, 0.9), 3.0, 1.0
    js, n_zs = [0, 5, 11], 8
    errs = []
    for lev in range(3):
        s = 2 ** lev
        ms, d = 32 * s, 0.5 / s
        g = orc.OracleGeometry.default(ms, ms, d, d, 12.0, 64, n_zs, 96 * s, rho_linear=True)
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
