"""The index algebra of the Toeplitz form of A2 (CPU only).

With the rings spaced like the slabs (spacing dz, n_zs rings, range starting
s dz + eps above the volume's bottom), A2[(h,m),(l,k)] = T[m, d, l] with
d = k - h - s, and T is stored over D = mz + n_zs - 1 columns q = d + n_zs - 1
+ s = k - h + n_zs - 1 per radius bin.  The product kernels walk, for output
row (h, m) of A2, the sub-rows (m, q) for q = n_zs-1-h .. n_zs-2-h+mz and
gather slab k = h + q - (n_zs - 1); for row (l, k) of A2^T, the sub-rows
(l, e = D - 1 - q) for e = mz-1-k .. mz-2-k+n_zs and gather ring
h = k + e - (mz - 1).  Here that walk is restated and checked, on random
sparse T and random geometries, against A2 built from its definition: every
index in range, every entry once, and the entry count the plan reports.
The master tensor's ring position is checked too: the ring of the one-ring
slab grid must sit relative to slab q as ring h sits relative to slab k."""
import math

import numpy as np
import pytest


def _random_taps(rng, mz, nz, n_ell, density=0.15):
    D = mz + nz - 1
    T = {}
    for m in range(n_ell):
        for q in range(D):
            ls = [l for l in range(n_ell) if rng.random() < density]
            if ls:
                T[(m, q)] = [(l, float(rng.standard_normal())) for l in ls]
    return T


def _definition(T, mz, nz, n_ell):
    """{(row (h, m), column (l, k)): value} from A2 = T[m, k - h + nz - 1, l]."""
    D = mz + nz - 1
    A = {}
    for h in range(nz):
        for k in range(mz):
            q = k - h + nz - 1
            assert 0 <= q < D
            for m in range(n_ell):
                for l, w in T.get((m, q), []):
                    A[((h, m), (l, k))] = w
    return A


def _forward_walk(T, mz, nz, n_ell):
    D = mz + nz - 1
    A = {}
    for h in range(nz):
        for m in range(n_ell):
            s0 = m * D + (nz - 1 - h)
            assert m * D <= s0 and s0 + mz <= (m + 1) * D     # pointer reads in range
            for sub in range(s0, s0 + mz):
                q = sub - m * D
                for l, w in T.get((m, q), []):
                    k = h + q - (nz - 1)
                    assert 0 <= k < mz and 0 <= l * mz + k < n_ell * mz
                    key = ((h, m), (l, k))
                    assert key not in A
                    A[key] = w
    return A


def _adjoint_walk(T, mz, nz, n_ell):
    D = mz + nz - 1
    Ta = {}
    for (m, q), lst in T.items():
        for l, w in lst:
            Ta.setdefault((l, D - 1 - q), []).append((m, w))
    A = {}
    for l in range(n_ell):
        for k in range(mz):
            s0 = l * D + (mz - 1 - k)
            assert l * D <= s0 and s0 + nz <= (l + 1) * D
            hs = []
            for sub in range(s0, s0 + nz):
                e = sub - l * D
                h = k + e - (mz - 1)
                assert 0 <= h < nz
                hs.append(h)
                for m, w in Ta.get((l, e), []):
                    assert 0 <= h * n_ell + m < nz * n_ell
                    key = ((h, m), (l, k))
                    assert key not in A
                    A[key] = w
            assert hs == sorted(hs)                            # rings ascending
    return A


def _count(T, mz, nz):
    """The plan's entry count: the tap in column q serves rings h < nz with
    slab k = h + q - (nz - 1) in the volume."""
    n = 0
    for (m, q), lst in T.items():
        u = q - (nz - 1)
        h0, h1 = max(0, -u), min(nz - 1, mz - 1 - u)
        n += len(lst) * max(0, h1 - h0 + 1)
    return n


@pytest.mark.parametrize("seed", range(12))
def test_walks_reproduce_the_definition(seed):
    rng = np.random.default_rng(seed)
    mz, nz, n_ell = int(rng.integers(1, 9)), int(rng.integers(1, 12)), int(rng.integers(1, 7))
    T = _random_taps(rng, mz, nz, n_ell)
    A = _definition(T, mz, nz, n_ell)
    assert _forward_walk(T, mz, nz, n_ell) == A
    assert _adjoint_walk(T, mz, nz, n_ell) == A
    assert _count(T, mz, nz) == len(A)


@pytest.mark.parametrize("seed", range(20))
def test_master_tensor_ring_position(seed):
    """Ring h at z_lo + (h + 1/2) dz, slab k centred at -H/2 + (k + 1/2) dz;
    the one-ring grid has D slabs centred about 0 and its ring at
    eps - dmin dz - D dz / 2 + dz / 2 with delta = z_lo + H/2 = s dz + eps,
    dmin = -(nz - 1) - s.  Then ring - slab offsets agree for q = k - h +
    nz - 1."""
    rng = np.random.default_rng(100 + seed)
    mz, nz = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    dz = float(rng.uniform(0.05, 2.0))
    H = mz * dz
    z_lo = -H / 2 + float(rng.uniform(-30, 30)) * dz
    delta = z_lo + H / 2
    s = round(delta / dz)
    eps = delta - s * dz
    D = mz + nz - 1
    dmin = -(nz - 1) - s
    zr = eps - dmin * dz - D * dz / 2 + dz / 2
    assert abs(eps) <= 0.5 * dz + 1e-12
    for h in range(nz):
        for k in range(mz):
            q = k - h + nz - 1
            ring = z_lo + (h + 0.5) * dz
            slab = -H / 2 + (k + 0.5) * dz
            slab_t = -D * dz / 2 + (q + 0.5) * dz
            assert math.isclose(ring - slab, zr - slab_t, rel_tol=0, abs_tol=1e-9 * dz * (1 + abs(s)))
