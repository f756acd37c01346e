"""Pins of the oracle's piecewise-linear voxels (voxel_linear; the paper notes
the algorithms carry over to piecewise-linear bases, Sec. 3.1) against facts
other than its own code (CPU only):
  * partition of unity: a node's bases sum to one inside the volume, so the
    node weights of a circle sum to its arc length inside the volume, which
    the constant basis's walk gives;
  * quadrature: the weights applied to any node field equal the line
    integral of that field's clamped bilinear interpolation, evaluated by
    numpy's Gauss-Legendre rule on the sub-arcs between the angles where the
    circle crosses a pixel or node line;
  * the walk against a second route (per-node box moments);
  * the adjoint identity and the quarter-turn and mirror symmetries.
A dropped term, a sign, a swapped axis or a wrong margin in the closed-form
arc integrals fails the quadrature pin."""
import math

import numpy as np
import pytest


def _geom(O, ms=6, mz=4, dxy=0.5, dz=0.45, radius=4.0, n_phi=8, phi0=0.37, n_zs=3, n_ell=14,
          voxel_linear=True):
    rxy = ms * dxy / math.sqrt(2)
    h = mz * dz
    return O.OracleGeometry(ms, mz, dxy, dz, radius, n_phi, phi0, n_zs, -0.5 * h, 0.5 * h,
                            n_ell, radius - rxy, radius + rxy, False, voxel_linear)


def _sensor(g, j):
    phi = g.phi0 + 2 * math.pi * j / g.n_phi
    return g.radius * math.cos(phi), g.radius * math.sin(phi)


def _rho(g, l):
    return g.ell_lo + (l + 0.5) * (g.ell_hi - g.ell_lo) / g.n_ell


def _interp(g, F, x, y):
    """Clamped bilinear interpolation of node values F[ix, iy] (nodes at the
    voxel centres), written independently of the oracle."""
    hx = 0.5 * g.ms * g.dxy
    sx = np.clip((x + hx) / g.dxy - 0.5, 0.0, g.ms - 1)
    sy = np.clip((y + hx) / g.dxy - 0.5, 0.0, g.ms - 1)
    i0 = np.minimum(np.floor(sx).astype(int), max(g.ms - 2, 0))
    k0 = np.minimum(np.floor(sy).astype(int), max(g.ms - 2, 0))
    u, v = sx - i0, sy - k0
    i1, k1 = np.minimum(i0 + 1, g.ms - 1), np.minimum(k0 + 1, g.ms - 1)
    return ((1 - u) * (1 - v) * F[i0, k0] + u * (1 - v) * F[i1, k0]
            + (1 - u) * v * F[i0, k1] + u * v * F[i1, k1])


def _sampled(g, F, j, l, order=8):
    """Line integral of the interpolated field along the circle: Gauss-Legendre
    (numpy's nodes) on every sub-arc between the angles where the circle
    crosses a pixel line or a node line, where the integrand is smooth."""
    cx, cy = _sensor(g, j)
    r = _rho(g, l)
    hx = 0.5 * g.ms * g.dxy
    lines = -hx + np.arange(2 * g.ms + 1) * 0.5 * g.dxy
    angles = [0.0, 2 * math.pi]
    for c, off in ((cx, 0.0), (cy, 0.5 * math.pi)):
        u = lines - c
        ok = np.abs(u) <= r
        base = np.arccos(np.clip(u[ok] / r, -1.0, 1.0))
        for a in np.concatenate([base, -base]):  # x = c + r cos(a), or y = c + r sin(a)
            angles.append((a + off) % (2 * math.pi))
    angles = np.unique(np.array(angles))
    t, wq = np.polynomial.legendre.leggauss(order)
    total = 0.0
    for a0, a1 in zip(angles[:-1], angles[1:]):
        am, ah = 0.5 * (a0 + a1), 0.5 * (a1 - a0)
        a = am + ah * t
        x, y = cx + r * np.cos(a), cy + r * np.sin(a)
        xm, ym = cx + r * math.cos(am), cy + r * math.sin(am)
        if abs(xm) < hx and abs(ym) < hx:
            total += float(np.sum(wq * _interp(g, F, x, y))) * ah * r
    return total


GEOMS = [dict(), dict(ms=7, dxy=0.4, phi0=0.0, n_phi=8), dict(ms=5, dxy=0.7, radius=3.1, n_ell=11),
         dict(ms=2, dxy=1.0, radius=2.5, n_ell=9), dict(ms=1, dxy=1.2, radius=2.0, n_ell=7)]


@pytest.mark.parametrize("kw", GEOMS)
def test_partition_of_unity(orc, kw):
    g = _geom(orc, **kw)
    gc = _geom(orc, voxel_linear=False, **kw)
    seen = 0
    for j in range(g.n_phi):
        for l in range(g.n_ell):
            w = orc.circle_arcs(g, j, l)
            a = orc.circle_arcs(gc, j, l)
            total = sum(a.values())
            assert abs(sum(w.values()) - total) <= 1e-13 * max(total, g.dxy)
            assert all(0 <= q < g.ms * g.ms for q in w)
            assert min(w.values(), default=0.0) >= -1e-15 * g.dxy
            seen += total > 0
    assert seen > g.n_phi


@pytest.mark.parametrize("kw", GEOMS[:4])
def test_weights_integrate_the_interpolated_field(orc, kw):
    g = _geom(orc, **kw)
    rng = np.random.default_rng(5)
    F = rng.uniform(-1.0, 2.0, (g.ms, g.ms))
    checked = 0
    for j in range(0, g.n_phi, 3):
        for l in range(0, g.n_ell, 2):
            w = orc.circle_arcs(g, j, l)
            if not w:
                continue
            got = sum(v * F[q // g.ms, q % g.ms] for q, v in w.items())
            want = _sampled(g, F, j, l)
            scale = sum(abs(v) for v in w.values()) * np.max(np.abs(F))
            assert abs(got - want) <= 1e-12 * scale, (j, l, got, want)
            checked += 1
    assert checked >= 6


def test_a_planted_sign_error_is_caught(orc):
    """The quadrature pin sees a wrong basis: node weights for the x-mirrored
    field differ from the field's own integral unless the circle is
    symmetric."""
    g = _geom(orc)
    rng = np.random.default_rng(6)
    F = rng.uniform(0.0, 1.0, (g.ms, g.ms))
    j, l = 1, 7
    w = orc.circle_arcs(g, j, l)
    wrong = sum(v * F[g.ms - 1 - q // g.ms, q % g.ms] for q, v in w.items())
    assert abs(wrong - _sampled(g, F, j, l)) > 1e-4 * _sampled(g, np.ones_like(F), j, l)


def test_walk_matches_box_moments(orc):
    """The shell walk's per-node weights against the per-node route: node
    weights from box moments of the circle over the node's four support
    boxes, times the (z, rho) semicircle weights."""
    g = _geom(orc, ms=6, mz=5, n_ell=14)
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(10):
        j, h, m = int(rng.integers(g.n_phi)), int(rng.integers(g.n_zs)), int(rng.integers(g.n_ell))
        w = orc.shell_weights(g, j, h, m)
        scale = max(abs(v) for v in w.values()) if w else 1.0
        for ix in range(g.ms):
            for iy in range(g.ms):
                for k in range(g.mz):
                    v = (ix * g.ms + iy) * g.mz + k
                    pw = orc.point_weight(g, j, h, m, ix, iy, k)
                    assert abs(pw - w.get(v, 0.0)) <= 1e-11 * scale, (j, h, m, ix, iy, k)
                    checked += pw != 0.0
    assert checked > 20


def test_constant_field_matches_constant_basis(orc):
    g = _geom(orc, ms=5, mz=4, n_ell=12)
    gc = _geom(orc, ms=5, mz=4, n_ell=12, voxel_linear=False)
    f = np.ones(g.f_shape)
    f[:, :, 1] = 2.5  # constant in x, y; any profile in z
    np.testing.assert_allclose(orc.forward(g, f), orc.forward(gc, f), rtol=0,
                               atol=1e-12 * np.max(orc.forward(gc, f)))


def test_adjoint_identity_and_voxel_route(orc):
    g = _geom(orc, ms=6, mz=5, n_ell=13, n_phi=8, n_zs=4)
    rng = np.random.default_rng(4)
    f = rng.standard_normal(g.f_shape)
    y = rng.standard_normal(g.p_shape)
    af, aty = orc.forward(g, f), orc.adjoint(g, y)
    assert abs(float(np.sum(af * y)) - float(np.sum(f * aty))) <= \
        1e-12 * np.linalg.norm(af) * np.linalg.norm(y)
    vox = np.array([[ix, iy, k] for ix in range(g.ms) for iy in range(g.ms) for k in range(g.mz)])
    sel = vox[rng.choice(len(vox), 30, replace=False)]
    got = orc.adjoint_voxels(g, y, sel)
    want = aty[sel[:, 0], sel[:, 1], sel[:, 2]]
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(aty))


def test_quarter_turn_and_mirror(orc):
    g = orc.OracleGeometry.default(8, 6, 0.5, 0.4, 5.0, 8, 6, 20, voxel_linear=True)
    rng = np.random.default_rng(9)
    f = rng.uniform(0, 1, g.f_shape)
    p = orc.forward(g, f)
    f_rot = f[:, ::-1, :].transpose(1, 0, 2)  # object turned +90 deg
    np.testing.assert_allclose(orc.forward(g, np.ascontiguousarray(f_rot)),
                               np.roll(p, g.n_phi // 4, axis=0), rtol=0, atol=1e-12 * np.max(p))
    idx = (-np.arange(g.n_phi)) % g.n_phi
    np.testing.assert_allclose(orc.forward(g, np.ascontiguousarray(f[:, ::-1, :])), p[idx],
                               rtol=0, atol=1e-12 * np.max(p))


def _gauss_srt(c, sig, s, ell):
    """Continuous SRT (Sec. 2: the integral over the sphere of radius ell
    about s) of exp(-|x - c|^2 / (2 sig^2)) in free space:
    2 pi ell sig^2 / d (exp(-(d - ell)^2 / 2 sig^2) - exp(-(d + ell)^2 / 2 sig^2)),
    d = |c - s|."""
    d = float(np.linalg.norm(c - s))
    return 2 * math.pi * ell * sig ** 2 / d * (np.exp(-(d - ell) ** 2 / (2 * sig ** 2))
                                              - np.exp(-(d + ell) ** 2 / (2 * sig ** 2)))


def test_linear_bases_approach_the_continuous_transform(orc):
    """A Gaussian narrow enough to vanish at the volume's edge, sampled on
    grids of 8^3 to 64^3 voxels (radius bins 3x the edge): every basis
    approaches its closed-form SRT at about second order, and the bilinear
    voxels with the linear intermediate are the closest at the finer levels
    (measured 1.56x closer than both constant at 64^3)."""
    R, L, sig = 6.0, 4.0, 0.45
    c = np.array([0.31, -0.22, 0.17])
    sub = 6
    o = (np.arange(sub) + 0.5) / sub - 0.5
    err = {}
    for ms in (8, 16, 32, 64):
        d = L / ms
        xc = (np.arange(ms) - (ms - 1) / 2) * d
        X, Y, Z = np.meshgrid(xc, xc, xc, indexing="ij")

        def g(dx, dy, dz):
            return np.exp(-((X + dx - c[0]) ** 2 + (Y + dy - c[1]) ** 2 + (Z + dz - c[2]) ** 2)
                          / (2 * sig ** 2))
        f_avg = sum(g(a * d, b * d, e * d) for a in o for b in o for e in o) / sub ** 3
        f_node = sum(g(0.0, 0.0, e * d) for e in o) / sub  # values at the centres, slab means in z
        n_ell, n_zs = 3 * ms, 4
        g0 = orc.OracleGeometry.default(ms, ms, d, d, R, 16, n_zs, n_ell)
        ell = g0.ell_lo + (np.arange(n_ell) + 0.5) * (g0.ell_hi - g0.ell_lo) / n_ell
        zh = g0.zs_lo + (np.arange(n_zs) + 0.5) * (g0.zs_hi - g0.zs_lo) / n_zs
        sh = np.array([[j, h, m] for j in (0, 3, 6) for h in range(n_zs) for m in range(n_ell)])
        want = np.array([_gauss_srt(c, sig, np.array([R * math.cos(2 * math.pi * j / 16),
                                                      R * math.sin(2 * math.pi * j / 16), zh[h]]),
                                    ell[m]) for j, h, m in sh])
        for vl in (False, True):
            for rl in (False, True):
                geo = orc.OracleGeometry.default(ms, ms, d, d, R, 16, n_zs, n_ell, rho_linear=rl,
                                                 voxel_linear=vl)
                p = orc.forward_shells(geo, f_node if vl else f_avg, sh)
                err.setdefault((vl, rl), []).append(np.linalg.norm(p - want) / np.linalg.norm(want))
    for key, e in err.items():
        assert all(b < 0.4 * a for a, b in zip(e, e[1:])), (key, e)
        assert e[-1] < 3e-3, (key, e)
    assert err[(True, True)][-1] < 0.75 * err[(False, False)][-1], err
    assert err[(True, True)][-2] < 0.75 * err[(False, False)][-2], err
