"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test fixes a part of the oracle by an independent fact:
  * analytic arc lengths (quadrant-interval closed form, tests/closed_forms.py)
    for every in-plane circle / (z, rho) semicircle cell entry and for a
    separable volume, which pins the composition of the two integrals
    (Sec. 2: outer measure l dt, inner measure (l sin t) da, snapped to the
    shared radius grid of Algorithm 1);
  * a hand-derived one-voxel case;
  * per-voxel weights computed by a second, box-by-box route;
  * the adjoint identity <A f, g> = <f, A^T g> (Algorithm 2 is the exact
    transpose of Algorithm 1);
  * exact symmetries of the cylindrical geometry.
"""
import math

import numpy as np
import pytest

from tests.closed_forms import arc_circle_rect


def _tiny(O, **kw):
    d = dict(ms=5, mz=4, dxy=0.6, dz=0.45, radius=3.0, n_phi=6, phi0=0.37, n_zs=3,
             zs_lo=-0.7, zs_hi=1.1, n_ell=12)
    d.update(kw)
    rxy = d["ms"] * d["dxy"] / math.sqrt(2)
    return O.OracleGeometry(d["ms"], d["mz"], d["dxy"], d["dz"], d["radius"], d["n_phi"],
                            d["phi0"], d["n_zs"], d["zs_lo"], d["zs_hi"], d["n_ell"],
                            d["radius"] - rxy, d["radius"] + rxy)


def _grid(g):
    L, H = g.ms * g.dxy, g.mz * g.dz
    dl = (g.ell_hi - g.ell_lo) / g.n_ell
    return dict(
        xb=-0.5 * L + np.arange(g.ms + 1) * g.dxy,
        zb=-0.5 * H + np.arange(g.mz + 1) * g.dz,
        ell=g.ell_lo + (np.arange(g.n_ell) + 0.5) * dl,
        edges=g.ell_lo + np.arange(g.n_ell + 1) * dl,
        zh=g.zs_lo + (np.arange(g.n_zs) + 0.5) * (g.zs_hi - g.zs_lo) / g.n_zs,
        phi=g.phi0 + 2 * math.pi * np.arange(g.n_phi) / g.n_phi,
    )


# --------------------------------------------------------------- helper sanity
def test_closed_form_helper_sanity():
    # whole circle inside
    assert arc_circle_rect(0, 0, 1, -2, 2, -2, 2) == pytest.approx(2 * math.pi, rel=1e-15)
    # centre on an edge: half the circle
    assert arc_circle_rect(0, 0, 1, 0, 5, -5, 5) == pytest.approx(math.pi, rel=1e-15)
    # centre on a corner: a quarter
    assert arc_circle_rect(0, 0, 1, 0, 5, 0, 5) == pytest.approx(0.5 * math.pi, rel=1e-15)
    # disjoint
    assert arc_circle_rect(0, 0, 1, 2, 3, -1, 1) == 0.0
    # chord: circle r=2 cut by the strip x in [1, 5]: angle 2*acos(1/2)
    assert arc_circle_rect(0, 0, 2, 1, 5, -5, 5) == pytest.approx(2 * 2 * math.acos(0.5), rel=1e-14)


def test_oracle_arc_in_box_matches_closed_form(orc):
    rng = np.random.default_rng(11)
    for _ in range(2000):
        cx, cy = rng.uniform(-3, 3, 2)
        r = rng.uniform(0.05, 4)
        x0, y0 = rng.uniform(-3, 2, 2)
        x1, y1 = x0 + rng.uniform(0.01, 2), y0 + rng.uniform(0.01, 2)
        a = orc.arc_in_box(cx, cy, r, x0, x1, y0, y1)
        b = arc_circle_rect(cx, cy, r, x0, x1, y0, y1)
        assert abs(a - b) <= 1e-12 * max(1.0, r), (cx, cy, r, x0, x1, y0, y1, a, b)



def test_oracle_arc_in_box_at_degenerate_positions(orc):
    """Circles tangent to an edge from inside or outside, through a corner,
    centred on an edge or a corner: the cases random boxes never hit
    (boundary ties have measure zero, so the length is still exact)."""
    x0, x1, y0, y1 = -1.0, 1.0, -0.5, 0.5
    n = 0
    for cx, cy in [(0.0, 0.0), (0.3, -0.2), (1.0, 1.0), (0.5, 0.0), (1.0, 0.5)]:
        radii = [x1 - cx, cx - x0, y1 - cy, cy - y0, math.hypot(x1 - cx, y1 - cy),
                 math.hypot(x0 - cx, y0 - cy), abs(x1 - cx) + 1.0, 0.25]
        for r in [r for r in radii if r > 0]:
            a = orc.arc_in_box(cx, cy, r, x0, x1, y0, y1)
            b = arc_circle_rect(cx, cy, r, x0, x1, y0, y1)
            assert abs(a - b) <= 1e-12 * max(1.0, r), (cx, cy, r, a, b)
            n += 1
    assert n >= 30

# ----------------------------------------------------- per-entry arc lengths
# A 3 x 3 grid of unit pixels (lines at -1.5, -0.5, 0.5, 1.5) seen from four
# sensors at distance 3 on the axes, with radius-bin centres 1.5, 2.5, 3.5 and
# 4.5: every circle of columns 0 and 2 touches an x-line at its nearest or
# farthest point, every circle of columns 1 and 3 a y-line.  From the low
# side (column 2: the rightmost point on a line; column 3: the topmost) and
# from the high side (columns 0, 1); radius 1.5 touches the box boundary from
# outside (no arc lies in the box), radius 4.5 touches it from inside.
TANGENT = dict(ms=3, mz=2, dxy=1.0, dz=1.0, radius=3.0, n_phi=4, phi0=0.0, n_zs=1, zs=(-1.0, 1.0),
               n_ell=4, ell=(1.0, 5.0))


def tangent_geometry(O, rho_linear=False):
    t = TANGENT
    return O.OracleGeometry(t["ms"], t["mz"], t["dxy"], t["dz"], t["radius"], t["n_phi"],
                            t["phi0"], t["n_zs"], t["zs"][0], t["zs"][1], t["n_ell"],
                            t["ell"][0], t["ell"][1], rho_linear)


def _sampled_arcs(sx, sy, rho, ms, dxy, n=400_000):
    """Arc per pixel by dense midpoint sampling of the angle: each sample
    carries rho * 2 pi / n and goes to the pixel it falls in.  Independent of
    both breakpoint walks and closed forms; exact to O(rho / n) per crossing."""
    a = (np.arange(n) + 0.5) * (2 * math.pi / n)
    hx = 0.5 * ms * dxy
    ix = np.floor((sx + rho * np.cos(a) + hx) / dxy).astype(np.int64)
    iy = np.floor((sy + rho * np.sin(a) + hx) / dxy).astype(np.int64)
    ok = (ix >= 0) & (ix < ms) & (iy >= 0) & (iy < ms)
    return np.bincount(ix[ok] * ms + iy[ok], minlength=ms * ms) * (rho * 2 * math.pi / n)


def test_circle_walk_at_tangent_positions(orc):
    """A circle that touches a pixel line must not move the arc around the
    point of contact into the pixel across that line (the arc's midpoint lies
    on the line); one that touches the box from outside has no arc inside."""
    g = tangent_geometry(orc)
    G = _grid(g)
    touched = 0
    for j in range(g.n_phi):
        sx, sy = g.radius * math.cos(G["phi"][j]), g.radius * math.sin(G["phi"][j])
        for l in range(g.n_ell):
            rho = G["ell"][l]
            near = abs(sx) - rho if j % 2 == 0 else abs(sy) - rho
            assert any(abs(abs(near) - abs(b)) < 1e-15 for b in G["xb"])  # really tangent
            touched += 1
            got = orc.circle_arcs(g, j, l)
            samp = _sampled_arcs(sx, sy, rho, g.ms, g.dxy)
            for ix in range(g.ms):
                for iy in range(g.ms):
                    want = arc_circle_rect(sx, sy, rho, G["xb"][ix], G["xb"][ix + 1],
                                           G["xb"][iy], G["xb"][iy + 1])
                    have = got.get(ix * g.ms + iy, 0.0)
                    assert abs(have - want) <= 1e-12 * rho, (j, l, ix, iy, have, want)
                    assert abs(have - samp[ix * g.ms + iy]) <= 1e-4, (j, l, ix, iy, have)
            if l == 0:  # radius 1.5 touches the box from outside
                assert got == {}, (j, got)
    assert touched == 16
    # the case that first showed the fault: sensor (-3, 0), radius 2.5, its
    # rightmost point on x = -0.5; the arc around it belongs to pixel (0, 1)
    got = orc.circle_arcs(g, 2, 1)
    want = arc_circle_rect(-3.0, 0.0, 2.5, -1.5, -0.5, -0.5, 0.5)
    assert want > 1.0 and abs(got.get(0 * 3 + 1, 0.0) - want) <= 1e-12
    assert 1 * 3 + 1 not in got


def test_forward_at_tangent_positions_matches_closed_forms(orc):
    """The whole shell walk at the tangent geometry, for the separable
    volume f = q[ix, iy] s[k]: p[j,h,m] = sum_{k,l} s[k] arc2(h,m;k,l)
    sum_pix q[pix] arc1(j,l;pix) with every arc from the closed form."""
    g = tangent_geometry(orc)
    G = _grid(g)
    rng = np.random.default_rng(21)
    q = rng.uniform(0.1, 1.0, (g.ms, g.ms))
    s = rng.uniform(0.1, 1.0, g.mz)
    f = q[:, :, None] * s[None, None, :]
    p = orc.forward(g, f)
    for j in range(g.n_phi):
        sx, sy = g.radius * math.cos(G["phi"][j]), g.radius * math.sin(G["phi"][j])
        inner = [sum(q[ix, iy] * arc_circle_rect(sx, sy, G["ell"][l], G["xb"][ix],
                                                  G["xb"][ix + 1], G["xb"][iy], G["xb"][iy + 1])
                     for ix in range(g.ms) for iy in range(g.ms)) for l in range(g.n_ell)]
        for h in range(g.n_zs):
            for m in range(g.n_ell):
                want = sum(s[k] * arc_circle_rect(G["zh"][h], 0.0, G["ell"][m], G["zb"][k],
                                                  G["zb"][k + 1], G["edges"][l],
                                                  G["edges"][l + 1]) * inner[l]
                           for k in range(g.mz) for l in range(g.n_ell))
                assert abs(p[j, h, m] - want) <= 1e-12 * max(1.0, abs(want)), (j, h, m)


def test_circle_arcs_match_closed_form(orc):
    g = _tiny(orc)
    G = _grid(g)
    L = g.ms * g.dxy
    for j in range(g.n_phi):
        sx, sy = g.radius * math.cos(G["phi"][j]), g.radius * math.sin(G["phi"][j])
        for l in range(g.n_ell):
            rho = G["ell"][l]
            got = orc.circle_arcs(g, j, l)
            tot = 0.0
            for ix in range(g.ms):
                for iy in range(g.ms):
                    want = arc_circle_rect(sx, sy, rho, G["xb"][ix], G["xb"][ix + 1],
                                           G["xb"][iy], G["xb"][iy + 1])
                    have = got.get(ix * g.ms + iy, 0.0)
                    assert abs(have - want) <= 1e-12 * rho, (j, l, ix, iy, have, want)
                    tot += have
            # row sum = arc of the circle inside the whole square
            sq = arc_circle_rect(sx, sy, rho, -L / 2, L / 2, -L / 2, L / 2)
            assert abs(tot - sq) <= 1e-12 * rho


def test_semicircle_arcs_match_closed_form(orc):
    g = _tiny(orc)
    G = _grid(g)
    H = g.mz * g.dz
    for h in range(g.n_zs):
        for m in range(g.n_ell):
            ell = G["ell"][m]
            got = orc.semicircle_arcs(g, h, m)
            tot = 0.0
            for l in range(g.n_ell):
                for k in range(g.mz):
                    want = arc_circle_rect(G["zh"][h], 0.0, ell, G["zb"][k], G["zb"][k + 1],
                                           G["edges"][l], G["edges"][l + 1])
                    have = got.get(l * g.mz + k, 0.0)
                    assert abs(have - want) <= 1e-12 * ell, (h, m, l, k, have, want)
                    tot += have
            band = arc_circle_rect(G["zh"][h], 0.0, ell, -H / 2, H / 2, g.ell_lo, g.ell_hi)
            assert abs(tot - band) <= 1e-12 * ell


# ------------------------------------------- composition, separable volume
def test_separable_volume_closed_form(orc):
    """f[ix, iy, k] = q[ix, iy] * s[k]:  p[j,h,m] = sum_{k,l} s[k] *
    arc2(h,m; k,l) * sum_pix q[pix] * arc1(j,l; pix), every arc closed-form."""
    g = _tiny(orc)
    G = _grid(g)
    rng = np.random.default_rng(5)
    q = rng.uniform(0.1, 1.0, (g.ms, g.ms))
    s = rng.uniform(0.1, 1.0, g.mz)
    f = q[:, :, None] * s[None, None, :]
    p = orc.forward(g, f)
    c1 = np.zeros((g.n_phi, g.n_ell))  # in-plane circle integral of q
    for j in range(g.n_phi):
        sx, sy = g.radius * math.cos(G["phi"][j]), g.radius * math.sin(G["phi"][j])
        for l in range(g.n_ell):
            acc = 0.0
            for ix in range(g.ms):
                for iy in range(g.ms):
                    acc += q[ix, iy] * arc_circle_rect(sx, sy, G["ell"][l], G["xb"][ix],
                                                       G["xb"][ix + 1], G["xb"][iy], G["xb"][iy + 1])
            c1[j, l] = acc
    want = np.zeros(g.p_shape)
    for h in range(g.n_zs):
        for m in range(g.n_ell):
            a2 = np.array([[arc_circle_rect(G["zh"][h], 0.0, G["ell"][m], G["zb"][k], G["zb"][k + 1],
                                            G["edges"][l], G["edges"][l + 1])
                            for k in range(g.mz)] for l in range(g.n_ell)])  # [l, k]
            want[:, h, m] = c1 @ (a2 @ s)
    assert np.max(np.abs(p - want)) <= 1e-12 * np.max(np.abs(want))
    assert np.count_nonzero(want) > 0.3 * want.size


# ----------------------------------------------------------- hand case
def test_one_voxel_hand_case(orc):
    """Unit voxel [-1/2, 1/2]^3, sensor (2, 0, 0), two radius bins over
    [2 - 1/sqrt2, 2 + 1/sqrt2].  Derived by hand:
      bin 0: l0 = 2 - 1/(2 sqrt2); the (z, rho) arc inside the slab is
             l0 * (pi - 2 acos(1/(2 l0))) and lies above rho = 2 - 1/sqrt2 and
             below rho = 2; the in-plane circle of radius l0 enters the pixel
             through y = -1/2 and leaves through y = +1/2: 2 l0 asin(1/(2 l0)).
      bin 1: l1 = 2 + 1/(2 sqrt2); the slab part of the (z, rho) arc has
             rho >= l1 sin(acos(1/(2 l1))) > 2, i.e. lies in bin 1 only; the
             in-plane arc is again 2 l1 asin(1/(2 l1))."""
    g = orc.OracleGeometry(1, 1, 1.0, 1.0, 2.0, 1, 0.0, 1, -0.5, 0.5, 2,
                           2 - 1 / math.sqrt(2), 2 + 1 / math.sqrt(2))
    l0 = 2 - 1 / (2 * math.sqrt(2))
    l1 = 2 + 1 / (2 * math.sqrt(2))
    # conditions under which the hand formulas hold
    assert l0 * math.sin(math.acos(0.5 / l0)) >= 2 - 1 / math.sqrt(2)
    assert l0 < 2.0
    assert l1 * math.sin(math.acos(0.5 / l1)) > 2.0
    assert 2 - math.sqrt(l0 ** 2 - 0.25) > -0.5 and l0 ** 2 - 2.25 > 0.25
    assert 2 - math.sqrt(l1 ** 2 - 0.25) > -0.5 and l1 ** 2 - 2.25 > 0.25
    p0 = l0 * (math.pi - 2 * math.acos(0.5 / l0)) * 2 * l0 * math.asin(0.5 / l0)
    p1 = l1 * (math.pi - 2 * math.acos(0.5 / l1)) * 2 * l1 * math.asin(0.5 / l1)
    p = orc.forward(g, np.ones((1, 1, 1)))
    assert p.shape == (1, 1, 2)
    assert p[0, 0, 0] == pytest.approx(p0, rel=1e-13)
    assert p[0, 0, 1] == pytest.approx(p1, rel=1e-13)
    f = orc.adjoint(g, np.array([[[0.3, -1.7]]]))
    assert f[0, 0, 0] == pytest.approx(0.3 * p0 - 1.7 * p1, rel=1e-13)


# --------------------------------------------- second route: point weights
def test_point_weights_match_shell_walk(orc):
    g = _tiny(orc, ms=6, mz=5, n_ell=14)
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(12):
        j, h, m = int(rng.integers(g.n_phi)), int(rng.integers(g.n_zs)), int(rng.integers(g.n_ell))
        w = orc.shell_weights(g, j, h, m)
        for ix in range(g.ms):
            for iy in range(g.ms):
                for k in range(g.mz):
                    v = (ix * g.ms + iy) * g.mz + k
                    pw = orc.point_weight(g, j, h, m, ix, iy, k)
                    assert abs(pw - w.get(v, 0.0)) <= 1e-12, (j, h, m, ix, iy, k)
                    checked += pw != 0.0
    assert checked > 20


# ------------------------------------------------------- adjoint identity
def test_adjoint_identity_and_voxel_route(orc):
    g = _tiny(orc, ms=7, mz=6, n_ell=16, n_phi=8, n_zs=5)
    rng = np.random.default_rng(4)
    f = rng.standard_normal(g.f_shape)
    y = rng.standard_normal(g.p_shape)
    af = orc.forward(g, f)
    aty = orc.adjoint(g, y)
    lhs, rhs = float(np.sum(af * y)), float(np.sum(f * aty))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(af) * np.linalg.norm(y)
    vox = np.array([[ix, iy, k] for ix in range(g.ms) for iy in range(g.ms) for k in range(g.mz)])
    sel = vox[rng.choice(len(vox), 40, replace=False)]
    got = orc.adjoint_voxels(g, y, sel)
    want = aty[sel[:, 0], sel[:, 1], sel[:, 2]]
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(aty))
    sel_sh = np.array([[j, h, m] for j in range(g.n_phi) for h in range(g.n_zs)
                       for m in range(g.n_ell)])[::7]
    got = orc.forward_shells(g, f, sel_sh)
    assert np.array_equal(got, af[sel_sh[:, 0], sel_sh[:, 1], sel_sh[:, 2]])
    # adjoint over a shell subset = full adjoint of data masked to that subset
    y_mask = np.zeros_like(y)
    y_mask[sel_sh[:, 0], sel_sh[:, 1], sel_sh[:, 2]] = y[sel_sh[:, 0], sel_sh[:, 1], sel_sh[:, 2]]
    sub = orc.adjoint_shells(g, sel_sh, y[sel_sh[:, 0], sel_sh[:, 1], sel_sh[:, 2]], nthreads=3)
    np.testing.assert_allclose(sub, orc.adjoint(g, y_mask), rtol=0,
                               atol=1e-12 * np.max(np.abs(sub)))


# ------------------------------------------------------------- symmetries
@pytest.fixture(scope="module")
def sym_setup(orc):
    g = orc.OracleGeometry.default(8, 6, 0.5, 0.4, 5.0, 8, 6, 20)
    rng = np.random.default_rng(9)
    f = rng.uniform(0, 1, g.f_shape)
    return g, f, orc.forward(g, f)


def test_rotation_by_quarter_turn(orc, sym_setup):
    g, f, p = sym_setup
    f_rot = f[:, ::-1, :].transpose(1, 0, 2)  # f_rot(x, y) = f(y, -x): object turned +90 deg
    p_rot = orc.forward(g, np.ascontiguousarray(f_rot))
    np.testing.assert_allclose(p_rot, np.roll(p, g.n_phi // 4, axis=0), rtol=0,
                               atol=1e-12 * np.max(p))


def test_mirror_y(orc, sym_setup):
    g, f, p = sym_setup
    p_m = orc.forward(g, np.ascontiguousarray(f[:, ::-1, :]))
    idx = (-np.arange(g.n_phi)) % g.n_phi
    np.testing.assert_allclose(p_m, p[idx], rtol=0, atol=1e-12 * np.max(p))


def test_mirror_z(orc, sym_setup):
    g, f, p = sym_setup
    p_m = orc.forward(g, np.ascontiguousarray(f[:, :, ::-1]))
    np.testing.assert_allclose(p_m, p[:, ::-1, :], rtol=0, atol=1e-12 * np.max(p))


def test_z_translation_shifts_rings(orc, sym_setup):
    g, f, _ = sym_setup
    f0 = f.copy()
    f0[:, :, -1] = 0.0
    f_t = np.zeros_like(f0)
    f_t[:, :, 1:] = f0[:, :, :-1]
    p0 = orc.forward(g, f0)
    pt = orc.forward(g, f_t)
    np.testing.assert_allclose(pt[:, 1:, :], p0[:, :-1, :], rtol=0, atol=1e-12 * np.max(p0))
