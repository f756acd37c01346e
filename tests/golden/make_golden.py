"""Write the oracle regression fixtures of this directory.

The paper reports no numerical values for a worked example, so the stored
values here are not the paper's: this script computes them with the FP64
oracle (oracle/) only, on seeded inputs from paper_2402_15641_gb300.inputs,
and tests/test_golden.py recomputes them.  A change to the oracle's
arithmetic that moves them must regenerate them (python
tests/golden/make_golden.py) in a commit that names the passage of the paper,
or the reading of it, that justifies the change.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2402_15641_gb300 import inputs as I  # noqa: E402

CASES = [("srt16fd", False, False), ("srt16fd", True, False), ("srt16fd", False, True)]


def compute(name, rho_linear, voxel_linear=False, n=48, seed=2024):
    sz = I.sizes(name)
    g = O.OracleGeometry.default(**sz, rho_linear=rho_linear, voxel_linear=voxel_linear)
    f = I.phantom(name)
    y = I.probe(name)
    rng = np.random.default_rng(seed)
    sh = np.stack([rng.integers(0, g.n_phi, n), rng.integers(0, g.n_zs, n),
                   rng.integers(0, g.n_ell, n)], axis=1)
    vx = np.stack([rng.integers(0, g.ms, n), rng.integers(0, g.ms, n),
                   rng.integers(0, g.mz, n)], axis=1)
    return sh, O.forward_shells(g, f, sh), vx, O.adjoint_voxels(g, y, vx)


def path(name, rho_linear, voxel_linear=False):
    return os.path.join(HERE, f"oracle_{name}{'_rho_linear' if rho_linear else ''}"
                              f"{'_voxel_linear' if voxel_linear else ''}.txt")


def main():
    for name, lin, vox in CASES:
        sh, p, vx, a = compute(name, lin, vox)
        with open(path(name, lin, vox), "w") as fh:
            fh.write(f"# FP64 oracle regression values, workload {name}, intermediate "
                     f"{'piecewise linear in rho' if lin else 'piecewise constant'}"
                     f"{', voxels bilinear between centres' if vox else ''}; written by\n"
                     "# tests/golden/make_golden.py (oracle/ only; the paper prints no worked example)\n")
            fh.write("# kind i0 i1 i2 value: fwd = p[j][h][m] of the seeded phantom; "
                     "adj = (A^T g)[ix][iy][k] of the seeded probe\n")
            for (j, h, m), v in zip(sh.tolist(), p.tolist()):
                fh.write(f"fwd {j} {h} {m} {v!r}\n")
            for (ix, iy, k), v in zip(vx.tolist(), a.tolist()):
                fh.write(f"adj {ix} {iy} {k} {v!r}\n")


if __name__ == "__main__":
    main()
