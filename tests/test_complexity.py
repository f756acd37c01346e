"""The complexity claim of Sec. 3.1: with N_l = O(M^{1/3}) radii, the two-CRT
factorisation costs O(M^{4/3}) against O(M^{5/3}) for quadrature over every
shell.  On a family of geometries with every axis count proportional to
s = M^{1/3} (ms = mz = n_zs = s, n_phi = 2s, n_ell = 3s, fixed field of
view), the oracle's own weights give
  * entries per A1 row (in-plane circle) and per A2 row ((z, rho)
    semicircle) proportional to s, so each product costs rows (s^2) x
    entries (s) x dense width (s) = s^4 = M^{4/3};
  * voxels per shell proportional to s^2, so the direct sum over s^3 shells
    costs s^5 = M^{5/3}.
Slopes are fitted over s = 8, 16, 32 on seeded samples of rows and shells."""

import numpy as np


def _geom(orc, s):
    fov, R = 12.8, 12.0
    return orc.OracleGeometry.default(s, s, fov / s, fov / s, R, 2 * s, s, 3 * s)


def _slope(xs, ys):
    return float(np.polyfit(np.log(xs), np.log(ys), 1)[0])


def test_entries_per_row_and_voxels_per_shell_scale_as_claimed(orc):
    sizes = [8, 16, 32]
    a1, a2, shell = [], [], []
    for s in sizes:
        g = _geom(orc, s)
        rng = np.random.default_rng(100 + s)
        rows1 = [(int(rng.integers(g.n_phi)), int(rng.integers(g.n_ell))) for _ in range(400)]
        rows2 = [(int(rng.integers(g.n_zs)), int(rng.integers(g.n_ell))) for _ in range(400)]
        shells = [(int(rng.integers(g.n_phi)), int(rng.integers(g.n_zs)), int(rng.integers(g.n_ell)))
                  for _ in range(60)]
        a1.append(np.mean([len(orc.circle_arcs(g, j, l)) for j, l in rows1]))
        a2.append(np.mean([len(orc.semicircle_arcs(g, h, m)) for h, m in rows2]))
        shell.append(np.mean([len(orc.shell_weights(g, j, h, m)) for j, h, m in shells]))
    k1, k2, ks = _slope(sizes, a1), _slope(sizes, a2), _slope(sizes, shell)
    assert abs(k1 - 1.0) < 0.15, (k1, a1)
    assert abs(k2 - 1.0) < 0.15, (k2, a2)
    assert abs(ks - 2.0) < 0.2, (ks, shell)
    # work exponents in M = s^3: rows s^2, dense width s
    factorised = (2 + k1 + 1) / 3, (2 + k2 + 1) / 3
    direct = (3 + ks) / 3
    assert all(abs(e - 4 / 3) < 0.06 for e in factorised), factorised
    assert abs(direct - 5 / 3) < 0.07, direct
    # and the factorisation wins by a growing factor: direct / factorised ~ s
    s = sizes[-1]
    ratio = (s ** 3 * shell[-1]) / (2 * s * s * a1[-1] * s + s * 3 * s * a2[-1] * 2 * s)
    assert ratio > 1.0
