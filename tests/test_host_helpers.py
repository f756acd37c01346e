"""The library's own FP64 geometry and BF16 rounding helpers, run on the host
(CPU only).  srt_arc_in_rect, srt_arc_in_rect_m and srt_f64_to_bf16 are
host-device functions of csrc/common.cuh; tests/host_helpers.cu compiles them
for the host with nvcc and runs them on inputs given here.  The results must
match:
  * the arc length and first moment int y ds of a circle inside a box, from
    the closed forms of tests/closed_forms.py (Python, written apart from
    the CUDA sources), on random and on tangent, edge and corner cases;
  * the round-to-nearest-even BF16 code of each FP64 value, rounded once,
    from exact rational arithmetic; values below the BF16 normal range flush
    to signed zero and values past its largest finite value round to
    infinity, as the function documents.
These are the helpers the assembly kernels compute every entry with; the GPU
parity tests check the device build of the same code against the oracle."""
import math
import os
import subprocess

import numpy as np
import pytest

from tests.closed_forms import arc_circle_rect, moment_circle_rect
from tests.test_bf16_helper import _rne_bf16

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def run():
    from paper_2402_15641_gb300 import build as B
    out = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out, exist_ok=True)
    exe = os.path.join(out, "host_helpers")
    subprocess.run([B.nvcc(), "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2402_15641_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_helpers.cu"), "-o", exe],
                   check=True, capture_output=True)

    def call(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                           check=True, timeout=120)
        return r.stdout.split()
    return call


def _bf16_code(x: float) -> int:
    """The expected code: exact RNE in the normal range, flush below it,
    infinity past the largest finite BF16 value."""
    sign = 0x8000 if math.copysign(1.0, x) < 0 else 0
    a = abs(x)
    if a < 2.0 ** -126:
        return sign
    v = _rne_bf16(a)
    if v >= 2.0 ** 128:
        return sign | 0x7F80
    return sign | int(np.array([v], dtype=np.float32).view(np.uint32)[0] >> 16)


def test_bf16_rounding(run):
    rng = np.random.default_rng(11)
    xs = list(np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 6000)) * rng.choice([-1, 1], 6000))
    for m in (128, 129, 200, 254, 255):        # ties between codes, even and odd
        xs += [(m + 0.5) / 128.0, -(m + 0.5) / 128.0, (m + 0.5) / 128.0 * 2.0 ** 40]
    xs += [130.5 / 128.0 + 2.0 ** -30]         # just above a tie (FP32 would round onto it)
    xs += [1.0, 2.0 ** -126, 2.0 ** -127, 1e-40, -1e-45, 0.0, -0.0]
    big = (2.0 - 2.0 ** -7) * 2.0 ** 127       # largest finite BF16
    xs += [big, big * (1 + 2.0 ** -10), big * (1 + 2.0 ** -8), 3.0e38, 1e300]
    got = run([f"bf16 {float(x).hex()}" for x in xs])
    assert [int(g) for g in got] == [_bf16_code(float(x)) for x in xs]


def _arc_cases(rng, n):
    cases = []
    for _ in range(n):
        cx, cy = rng.uniform(-3, 3, 2)
        r = rng.uniform(0.05, 4)
        x0, y0 = rng.uniform(-3, 2, 2)
        cases.append((cx, cy, r, x0, x0 + rng.uniform(0.01, 2), y0, y0 + rng.uniform(0.01, 2)))
    # tangent boxes, centre on an edge or a corner, the whole circle, none of it
    cases += [(0.0, 0.0, 1.0, 1.0, 2.0, -1.0, 1.0), (0.0, 0.0, 1.0, -1.0, 1.0, 1.0, 2.0),
              (0.0, 0.0, 1.0, 0.0, 5.0, -5.0, 5.0), (0.0, 0.0, 1.0, 0.0, 5.0, 0.0, 5.0),
              (0.3, -0.2, 1.5, -5.0, 5.0, -5.0, 5.0), (0.0, 0.0, 1.0, 2.0, 3.0, -1.0, 1.0),
              (0.0, 0.0, 2.0, 1.0, 5.0, -5.0, 5.0), (0.0, 5.0, 1.0, -1.0, 1.0, 4.0, 6.0),
              (0.0, 5.0, 1.0, -0.5, 0.5, 5.5, 6.0)]
    # tangent to each edge from inside and outside, through corners
    x0, x1, y0, y1 = -1.0, 1.0, -0.5, 0.5
    for cx, cy in [(0.0, 0.0), (0.3, -0.2), (1.0, 1.0), (0.5, 0.0), (1.0, 0.5)]:
        for r in [x1 - cx, cx - x0, y1 - cy, cy - y0, math.hypot(x1 - cx, y1 - cy),
                  math.hypot(x0 - cx, y0 - cy), abs(x1 - cx) + 1.0]:
            if r > 0:
                cases.append((cx, cy, r, x0, x1, y0, y1))
    return cases


def test_arc_length_and_moment(run):
    rng = np.random.default_rng(12)
    cases = _arc_cases(rng, 3000)
    got = run([" ".join(["arc"] + [float(v).hex() for v in c]) for c in cases])
    vals = np.array([float.fromhex(g) for g in got]).reshape(-1, 3)
    for c, (length, length_m, my) in zip(cases, vals):
        want = arc_circle_rect(*c)
        want_m = moment_circle_rect(*c)
        r, cy = c[2], c[1]
        assert abs(length - want) <= 1e-12 * max(1.0, r), (c, length, want)
        assert abs(length_m - length) <= 1e-13 * max(1.0, r), (c, length_m, length)
        assert abs(my - want_m) <= 1e-12 * max(1.0, r * (r + abs(cy))), (c, my, want_m)


def test_arc_length_against_oracle_walk_at_degenerate_positions(run, orc):
    """The tangent, corner and edge-centred cases once more, now against the
    oracle's arc_in_box: sorted breakpoints and an open-box midpoint test, a
    method unlike the quarter intervals that both the library helper and
    the closed form use, so an error shared by those two still shows here."""
    cases = _arc_cases(np.random.default_rng(13), 0)
    got = run([" ".join(["arc"] + [float(v).hex() for v in c]) for c in cases])
    vals = np.array([float.fromhex(g) for g in got]).reshape(-1, 3)
    assert len(cases) >= 35
    for c, (length, _, _) in zip(cases, vals):
        want = orc.arc_in_box(*c)
        assert abs(length - want) <= 1e-12 * max(1.0, c[2]), (c, length, want)


def _bilinear_quadrature(cx, cy, r, x0, x1, y0, y1, bx, by, order=10):
    """int (1 + bx x)(1 + by y) ds along the circle inside the box: numpy's
    Gauss-Legendre rule on the sub-arcs between the angles where the circle
    meets a box line (the integrand is smooth on each)."""
    ang = [0.0, 2 * math.pi]
    for c, lines, off in ((cx, (x0, x1), 0.0), (cy, (y0, y1), 0.5 * math.pi)):
        for v in lines:
            u = v - c
            if abs(u) <= r:
                b = math.acos(max(-1.0, min(1.0, u / r)))
                ang += [(b + off) % (2 * math.pi), (-b + off) % (2 * math.pi)]
    ang = np.unique(np.array(ang))
    t, w = np.polynomial.legendre.leggauss(order)
    total = 0.0
    for a0, a1 in zip(ang[:-1], ang[1:]):
        am, ah = 0.5 * (a0 + a1), 0.5 * (a1 - a0)
        xm, ym = cx + r * math.cos(am), cy + r * math.sin(am)
        if not (x0 < xm < x1 and y0 < ym < y1):
            continue
        a = am + ah * t
        x, y = cx + r * np.cos(a), cy + r * np.sin(a)
        total += float(np.sum(w * (1 + bx * x) * (1 + by * y))) * ah * r
    return total


def test_arc_bilinear_against_quadrature(run):
    """srt_arc_bilinear (the piecewise-linear voxels' entries, node-centred
    coordinates) against Gauss-Legendre quadrature: random circles through
    the four boxes of a node's support and its half-width margin boxes, with
    the slopes those boxes use (+-1/d, 0), short arcs where the series
    apply, and random boxes and slopes."""
    rng = np.random.default_rng(21)
    cases = []
    for _ in range(1500):
        d = float(rng.choice([0.1, 0.5, 1.3]))
        r = float(rng.uniform(0.5, 40.0))
        ang = rng.uniform(0, 2 * math.pi)
        dist = r + rng.uniform(-1.5, 1.5) * d  # the circle passes near the node
        cx, cy = -dist * math.cos(ang), -dist * math.sin(ang)
        sx, sy = int(rng.integers(2)), int(rng.integers(2))
        half_x, half_y = rng.random() < 0.2, rng.random() < 0.2
        wx = 0.5 * d if half_x else d
        wy = 0.5 * d if half_y else d
        x0, x1 = (-wx, 0.0) if sx == 0 else (0.0, wx)
        y0, y1 = (-wy, 0.0) if sy == 0 else (0.0, wy)
        bx = 0.0 if half_x else (1.0 / d if sx == 0 else -1.0 / d)
        by = 0.0 if half_y else (1.0 / d if sy == 0 else -1.0 / d)
        cases.append((cx, cy, r, x0, x1, y0, y1, bx, by))
    for _ in range(300):
        r = float(rng.uniform(0.2, 5.0))
        cx, cy = rng.uniform(-3, 3, 2)
        x0, y0 = rng.uniform(-4, 3, 2)
        x1, y1 = x0 + rng.uniform(0.01, 3), y0 + rng.uniform(0.01, 3)
        cases.append((cx, cy, r, x0, x1, y0, y1, *rng.uniform(-2, 2, 2)))
    # a circle tangent to a box line, and one through a corner
    cases += [(0.0, -2.0, 2.0, -0.1, 0.1, 0.0, 0.1, 10.0, -10.0),
              (-3.0, -4.0, 5.0, -0.1, 0.0, 0.0, 0.1, 10.0, -10.0)]
    got = run([" ".join(["bil"] + [float(v).hex() for v in c]) for c in cases])
    hits = 0
    for c, g in zip(cases, got):
        val = float.fromhex(g)
        want = _bilinear_quadrature(*c)
        scale = (c[4] - c[3]) + (c[6] - c[5])  # a bound on the arc length in the box
        scale *= (1 + abs(c[7]) * max(abs(c[3]), abs(c[4]))) * \
            (1 + abs(c[8]) * max(abs(c[5]), abs(c[6])))
        assert abs(val - want) <= 1e-12 * scale, (c, val, want)
        hits += want > 0
    assert hits > 500
