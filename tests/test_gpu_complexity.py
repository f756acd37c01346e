"""The complexity claim of Sec. 3.1 on the assembled operators: over the
family ms = mz = n_zs = s, n_phi = 2s, n_ell = 3s (fixed field of view),
nnz1 and nnz2 grow as s^3 = M, so the forward's FLOPs 2 (nnz1 mz + nnz2
n_phi) grow as s^4 = M^{4/3} (exact counts from the plans' count pass)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_plan_sizes_scale_as_m_to_the_four_thirds():
    import torch
    from paper_2402_15641_gb300 import build
    from paper_2402_15641_gb300.srt import Geometry, Plan
    assert torch.cuda.is_available()
    build.build()
    sizes, n1, n2, fl = [32, 64, 128, 256], [], [], []
    for s in sizes:
        plan = Plan(Geometry.default(s, s, 12.8 / s, 12.8 / s, 12.0, 2 * s, s, 3 * s))
        i = plan.info
        n1.append(i["nnz1"])
        n2.append(i["nnz2"])
        fl.append(2 * (i["nnz1"] * s + i["nnz2"] * 2 * s))
        plan.close()
    k1 = np.polyfit(np.log(sizes), np.log(n1), 1)[0]
    k2 = np.polyfit(np.log(sizes), np.log(n2), 1)[0]
    kf = np.polyfit(np.log(sizes), np.log(fl), 1)[0]
    print(f"COMPLEXITY nnz1 ~ s^{k1:.3f}, nnz2 ~ s^{k2:.3f}, forward FLOPs ~ s^{kf:.3f} "
          f"= M^{kf / 3:.3f} (nnz1 {n1}, nnz2 {n2})")
    assert abs(k1 - 3) < 0.1 and abs(k2 - 3) < 0.1
    assert abs(kf / 3 - 4 / 3) < 0.03
