"""Oracle regression fixtures (tests/golden/, written by make_golden.py from
the oracle alone; the paper prints no worked example): recomputing them must
give the stored FP64 values, so any change to the oracle's arithmetic shows
up here and has to be justified when the fixtures are regenerated."""
import numpy as np
import pytest

from tests.golden import make_golden as M


@pytest.mark.parametrize("name,rho_linear,voxel_linear", M.CASES)
def test_oracle_reproduces_stored_values(orc, name, rho_linear, voxel_linear):
    rows = [ln.split() for ln in open(M.path(name, rho_linear, voxel_linear))
            if not ln.startswith("#")]
    fwd = [(tuple(map(int, r[1:4])), float(r[4])) for r in rows if r[0] == "fwd"]
    adj = [(tuple(map(int, r[1:4])), float(r[4])) for r in rows if r[0] == "adj"]
    assert len(fwd) == len(adj) == 48
    sh, p, vx, a = M.compute(name, rho_linear, voxel_linear)
    assert [t for t, _ in fwd] == [tuple(x) for x in sh.tolist()]
    assert [t for t, _ in adj] == [tuple(x) for x in vx.tolist()]
    want_p = np.array([v for _, v in fwd])
    want_a = np.array([v for _, v in adj])
    assert np.max(np.abs(p - want_p)) <= 1e-12 * np.max(np.abs(want_p))
    assert np.max(np.abs(a - want_a)) <= 1e-12 * np.max(np.abs(want_a))
    assert np.count_nonzero(want_p) > 24
