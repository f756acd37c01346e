"""The seeded input recipe (CPU only): workload sizes, phantoms, probe data.

These generators feed both the CUDA path and the oracle, so what they promise
is checked here: the sizes of each workload, balls lying fully inside the
box, partial-volume ball masses close to the ball's volume, crops that are
zero outside the central voxels, N(0, 1) probe data, and the same numbers
for the same seed.
"""
import math

import numpy as np
import pytest

from paper_2402_15641_gb300 import inputs as I


def test_workload_sizes():
    want = {"srt32": (32, 0.5, 12.0, 64, 32, 96), "srt128": (128, 0.2, 20.0, 256, 128, 512),
            "srt256": (256, 0.1, 20.0, 256, 256, 768), "srt16fd": (16, 0.5, 12.0, 32, 16, 48)}
    for name, (m, d, R, nphi, nzs, nell) in want.items():
        s = I.sizes(name)
        assert (s["ms"], s["mz"], s["dxy"], s["dz"], s["radius"], s["n_phi"], s["n_zs"],
                s["n_ell"]) == (m, m, d, d, R, nphi, nzs, nell)
        # sensors outside the volume's in-plane half-diagonal
        assert s["radius"] > s["ms"] * s["dxy"] / math.sqrt(2)
    for edge in (64, 96, 128, 192):
        for nphi in (128, 256):
            g = I.serving_geometry(edge, nphi)
            assert g["ms"] * g["dxy"] == pytest.approx(25.6)
            assert (g["n_zs"], g["n_ell"], g["radius"], g["n_phi"]) == (edge, 4 * edge, 20.0, nphi)


@pytest.mark.parametrize("a", [0.9, 1.7, 2.6])
def test_partial_volume_ball_mass(a):
    dxy, dz, ms, mz = 0.25, 0.3, 32, 28
    f = np.zeros((ms, ms, mz))
    I.add_ball(f, dxy, dz, (0.31, -0.17, 0.08), a, 0.7, sub=8)
    assert f.min() >= 0 and f.max() <= 0.7 + 1e-12
    mass = f.sum() * dxy * dxy * dz / 0.7
    assert mass == pytest.approx(4.0 / 3.0 * math.pi * a ** 3, rel=5e-3)
    # voxels wholly inside hold the amplitude, voxels wholly outside nothing
    x = (np.arange(ms) - (ms - 1) / 2) * dxy - 0.31
    y = (np.arange(ms) - (ms - 1) / 2) * dxy + 0.17
    z = (np.arange(mz) - (mz - 1) / 2) * dz - 0.08
    r = np.sqrt(x[:, None, None] ** 2 + y[None, :, None] ** 2 + z[None, None, :] ** 2)
    half = 0.5 * math.sqrt(2 * dxy * dxy + dz * dz)
    assert np.all(f[r <= a - half] == 0.7)
    assert np.all(f[r >= a + half] == 0.0)


def test_balls_lie_inside_the_box():
    rng = np.random.default_rng(7)
    ms, mz, dxy, dz = 32, 24, 0.5, 0.5
    f, bl = I.balls(ms, mz, dxy, dz, 40, rng)
    hx, hz = ms * dxy / 2, mz * dz / 2
    for (cx, cy, cz), a, amp in bl:
        assert 1.0 <= a <= 4.0 and 0.2 <= amp <= 1.0
        assert abs(cx) + a <= hx and abs(cy) + a <= hx and abs(cz) + a <= hz
    # the voxels' mass is the balls' (none is cut by the box)
    mass = f.sum() * dxy * dxy * dz
    want = sum(amp * 4.0 / 3.0 * math.pi * a ** 3 for _, a, amp in bl)
    assert mass == pytest.approx(want, rel=1e-2)


def test_phantoms_are_seeded_and_cropped():
    w = dict(I.WORKLOADS["srt32"], n_blobs=60)
    a, b = I.phantom(w), I.phantom(w)
    assert np.array_equal(a, b) and a.shape == (32, 32, 32)
    assert np.isfinite(a).all() and a.min() >= 0 and a.max() > 0
    assert not np.array_equal(a, I.phantom(w, seed=5))
    # the vessel tree adds mass on top of the balls
    assert a.sum() > I.phantom(I.WORKLOADS["srt32"]).sum()
    c = I.crop_phantom(w, 12)
    inner = (slice(10, 22),) * 3
    assert np.array_equal(c[inner], a[inner])
    c[inner] = 0
    assert not c.any()


def test_probe_data():
    p = I.probe("srt32")
    assert p.shape == (64, 32, 96)
    assert np.array_equal(p, I.probe("srt32"))
    assert abs(p.mean()) < 0.01 and abs(p.std() - 1) < 0.01
