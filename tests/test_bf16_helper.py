"""The check that the GPU tests apply to BF16-stored entries, pinned on the
CPU: bf16_is_rne_of(w, x) must accept exactly the round-to-nearest-even BF16
of the FP64 value x, rounded once (BF16 entries are rounded directly from
the FP64 lengths, never through FP32).  The expected codes come from exact
rational arithmetic on the BF16 grid."""
import math
from fractions import Fraction

import numpy as np

from tests.gpu_helpers import bf16_is_rne_of


def _rne_bf16(x: float) -> float:
    """Round a positive FP64 value to BF16 (8 significant bits), ties to even,
    exactly."""
    e = math.frexp(x)[1] - 1                   # 2^e <= x < 2^(e+1)
    ulp = Fraction(2) ** (e - 7)
    q = Fraction(x) / ulp
    lo = math.floor(q)
    r = q - lo
    n = lo + 1 if r > Fraction(1, 2) or (r == Fraction(1, 2) and lo % 2 == 1) else lo
    return float(n * ulp)


def _neighbours(w: float):
    b = np.array([w], dtype=np.float32).view(np.uint32)[0]
    up = np.array([b + (1 << 16)], dtype=np.uint32).view(np.float32)[0]
    dn = np.array([b - (1 << 16)], dtype=np.uint32).view(np.float32)[0]
    return float(up), float(dn)


def test_accepts_the_rounding_and_rejects_its_neighbours():
    rng = np.random.default_rng(3)
    xs = np.exp(rng.uniform(np.log(1e-6), np.log(1e6), 2000))
    want = np.array([_rne_bf16(float(x)) for x in xs])
    assert np.all(bf16_is_rne_of(want.astype(np.float32), xs))
    for x, w in zip(xs[:300], want[:300]):
        for other in _neighbours(w):
            assert not bf16_is_rne_of(np.array([other], dtype=np.float32), np.array([x]))[0]
    # not a BF16 value at all: the FP32 rounding of x, where it differs
    f32 = xs.astype(np.float32)
    differs = f32.astype(np.float64) != want
    assert differs.any() and not bf16_is_rne_of(f32[differs], xs[differs]).any()


def test_ties_go_to_even():
    for m in (129, 130, 200, 255):             # BF16 significands m / 128 (m = 128..255)
        x = (m + 0.5) / 128.0                  # exactly halfway to the next code
        even = (m if m % 2 == 0 else m + 1) / 128.0
        odd = (m + 1 if m % 2 == 0 else m) / 128.0
        assert bf16_is_rne_of(np.array([even], dtype=np.float32), np.array([x]))[0]
        assert not bf16_is_rne_of(np.array([odd], dtype=np.float32), np.array([x]))[0]


def test_double_rounding_through_fp32_is_refused():
    """x lies just above a BF16 tie, closer to it than FP32 resolves: FP32
    rounds x onto the tie, and the tie then goes to the even code below,
    while the single rounding of x goes up."""
    a = 130 / 128.0                            # even BF16 code
    tie = (130.5) / 128.0
    x = tie + 2.0 ** -30                       # FP32 spacing here is 2^-23
    assert float(np.float32(x)) == tie
    once = _rne_bf16(x)
    assert once == 131 / 128.0
    twice = _rne_bf16(float(np.float32(x)))
    assert twice == a
    assert bf16_is_rne_of(np.array([once], dtype=np.float32), np.array([x]))[0]
    assert not bf16_is_rne_of(np.array([twice], dtype=np.float32), np.array([x]))[0]
