"""The debug build (libsrt_checks.so, -DSRT_CHECKS): every product kernel
checks each gathered row index against its operand's row count before the
access, counts an index outside it and reads row 0 instead (no fault).

On geometries whose operators were checked on the CPU (exports against the
oracle and exact transposes in the other GPU tests), the checked build finds
no bad index and gives the release build's results bitwise, for every kernel
family (CSR rows, A2 taps, A2 and A1^T tiles, the symmetric A1 forms).  With
the operand row count capped below the true count (srt_checks_cap), in-range
indices trip the check: the call returns SRT_ERR_CUDA and srt_checks_read
reports them, and no access leaves an operand, since the kernels read row 0
in their place."""
import numpy as np
import pytest

from paper_2402_15641_gb300 import inputs as I
from tests.gpu_helpers import geom_pair, to_dev
from tests.test_oracle_pins import TANGENT

pytestmark = pytest.mark.gpu

GEOMS = [dict(I.sizes("srt16fd")), dict(I.sizes("srt32")), TANGENT,
         dict(ms=7, mz=5, dxy=0.5, dz=0.37, radius=6.0, n_phi=6, n_zs=3, n_ell=13, phi0=0.2),
         dict(ms=10, mz=8, dxy=0.5, dz=0.5, radius=6.0, n_phi=16, n_zs=8, n_ell=13,
              zs=(-2.0 + 0.15, 2.0 + 0.15))]
FORMS = [{}, dict(rowwise=True), dict(a1_full=True), dict(csr_only=True), dict(rho_linear=True)]


@pytest.fixture(scope="module")
def libs():
    import torch
    from paper_2402_15641_gb300 import build, _lib
    assert torch.cuda.is_available()
    build.build()
    checked = _lib.load(build.build(checks=True))
    return _lib.lib(), checked


def test_release_build_has_no_checks(libs):
    import ctypes
    from paper_2402_15641_gb300._lib import SRT_ERR_ARG
    release, _ = libs
    n = ctypes.c_int64(-1)
    assert release.srt_checks_read(ctypes.byref(n)) == SRT_ERR_ARG
    assert release.srt_checks_cap(5) == SRT_ERR_ARG


@pytest.mark.parametrize("sz", GEOMS)
@pytest.mark.parametrize("form", FORMS)
def test_checked_build_finds_nothing_and_matches_release(libs, orc, sz, form):
    import ctypes
    import torch
    from paper_2402_15641_gb300.srt import Plan
    release, checked = libs
    g, _ = geom_pair(orc, **sz, **form)
    a, b = Plan(g, lib=release), Plan(g, lib=checked)
    rng = np.random.default_rng(61)
    f = to_dev(rng.uniform(0, 1, (2, *g.f_shape)))
    y = to_dev(rng.standard_normal((2, *g.p_shape)))
    assert torch.equal(a.forward(f), b.forward(f))
    assert torch.equal(a.adjoint(y), b.adjoint(y))
    n = ctypes.c_int64(-1)
    assert checked.srt_checks_read(ctypes.byref(n)) == 0 and n.value == 0


@pytest.mark.parametrize("form", FORMS)
def test_capped_rows_trip_the_checks(libs, orc, form):
    import ctypes
    from paper_2402_15641_gb300._lib import SrtError, SRT_ERR_CUDA
    from paper_2402_15641_gb300.srt import Plan
    _, checked = libs
    g, _ = geom_pair(orc, **dict(I.sizes("srt16fd")), **form)
    plan = Plan(g, lib=checked)
    f = to_dev(np.random.default_rng(62).uniform(0, 1, g.f_shape))
    y = to_dev(np.random.default_rng(63).standard_normal(g.p_shape))
    n = ctypes.c_int64(-1)
    try:
        assert checked.srt_checks_cap(7) == 0
        for call, x in ((plan.forward, f), (plan.adjoint, y)):
            with pytest.raises(SrtError) as e:
                call(x)
            assert e.value.code == SRT_ERR_CUDA
            assert checked.srt_checks_read(ctypes.byref(n)) == 0 and n.value > 0
    finally:
        assert checked.srt_checks_cap(0) == 0
    plan.forward(f)
    plan.adjoint(y)
    assert checked.srt_checks_read(ctypes.byref(n)) == 0 and n.value == 0
