"""The algorithmic work bench.py divides by (the roofline numerator), pinned
to hand-counted figures for the 256^3 workload: FLOPs = 2 per stored entry
per dense column; bytes = entries x (value + index) + row pointers + dense
input + dense output, with FP32 dense operands."""
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

G = SimpleNamespace(ms=256, mz=256, n_phi=256, n_zs=256, n_ell=768)
NNZ1, NNZ2, TAPS = 45_314_304, 82_815_806, 678_652
F = 4 * 256 * 256 * 256                 # f: 67,108,864 B
Y1 = 4 * 256 * 768 * 256                # Y1 (= Y1'), and P' (= p): 201,326,592 B


def _stages(**info):
    m = bench.stage_model(G, dict(nnz1=NNZ1, nnz2=NNZ2, **info), 1, "fp32")
    return {name: d for part in m.values() for name, d in part}


def test_fp32_taps_model():
    s = _stages(a2_taps=1, n_taps=TAPS)
    assert s["spmm1"]["flop"] == 23_200_923_648                  # 2 x 45.3 M x 256
    assert s["spmm2"]["flop"] == s["spmm2t"]["flop"] == 42_401_692_672
    # A1: 8 B per entry, 196,609 row pointers, f in, Y1 out
    assert s["spmm1"]["bytes"] == 362_514_432 + 786_436 + F + Y1 == 631_736_324
    # A1^T: same entries, 65,537 row pointers
    assert s["spmm1t"]["bytes"] == 362_514_432 + 262_148 + Y1 + F
    # A2 from the taps: 8 B per tap, 768 x 511 + 1 sub-row pointers, Y1' in, P' out
    assert s["spmm2"]["bytes"] == s["spmm2t"]["bytes"] == 5_429_216 + 1_569_796 + 2 * Y1
    for k in ("permute1", "permute2", "permute2_inv", "permute1_inv"):
        assert s[k] == {"flop": 0, "bytes": 2 * Y1}


def test_csr_bf16_and_rotation_models():
    s = bench.stage_model(G, dict(nnz1=NNZ1, nnz2=NNZ2), 1, "bf16")
    s = {n: d for part in s.values() for n, d in part}
    # BF16 entries: 6 B per entry; A2 as CSR with 196,609 / 196,609 pointers
    assert s["spmm2"]["bytes"] == NNZ2 * 6 + 4 * 196_609 + 2 * Y1
    assert s["spmm2t"]["bytes"] == NNZ2 * 6 + 4 * 196_609 + 2 * Y1
    s = bench.stage_model(G, dict(nnz1=NNZ1, nnz2=NNZ2, a1_rot=1), 1, "fp32")
    s = {n: d for part in s.values() for n, d in part}
    # A1 by rotation: a quarter of the entries and of the row pointers stored
    assert s["spmm1"]["bytes"] == NNZ1 // 4 * 8 + 4 * (196_608 // 4 + 1) + F + Y1
    assert s["spmm1"]["flop"] == 23_200_923_648                  # work is unchanged


def test_batch_scales_dense_bytes_and_flops():
    one = {n: d for p in bench.stage_model(G, dict(nnz1=NNZ1, nnz2=NNZ2), 1, "fp32").values()
           for n, d in p}
    four = {n: d for p in bench.stage_model(G, dict(nnz1=NNZ1, nnz2=NNZ2), 4, "fp32").values()
            for n, d in p}
    assert four["spmm2"]["flop"] == 4 * one["spmm2"]["flop"]
    entries = NNZ2 * 8 + 4 * 196_609
    assert four["spmm2"]["bytes"] - entries == 4 * (one["spmm2"]["bytes"] - entries)


def test_fused_reshapes_model():
    """With P2 and P1^-1 in the products' epilogues their stages drop out; the
    products read and write the same compulsory bytes (the layout changes,
    not the amount)."""
    info = dict(nnz1=NNZ1, nnz2=NNZ2, a2_taps=1, n_taps=TAPS)
    fused = bench.stage_model(G, info, 1, "fp32", fused=True)
    plain = bench.stage_model(G, info, 1, "fp32")
    assert [s and s[0] for s in fused["fwd"]] == ["spmm1", "permute1", "spmm2", None]
    assert [s and s[0] for s in fused["adj"]] == ["permute2_inv", "spmm2t", None, "spmm1t"]
    for d in ("fwd", "adj"):
        for a, b in zip(fused[d], plain[d]):
            if a is not None:
                assert a == b


def test_fused_p1_model():
    """With P1 in the A1 epilogue as well, the forward keeps two stages."""
    info = dict(nnz1=NNZ1, nnz2=NNZ2, a2_taps=1, n_taps=TAPS, a1_rot=2)
    both = bench.stage_model(G, info, 1, "fp32", fused=True, fused_p1=True)
    plain = bench.stage_model(G, info, 1, "fp32")
    assert [s and s[0] for s in both["fwd"]] == ["spmm1", None, "spmm2", None]
    assert both["adj"] == bench.stage_model(G, info, 1, "fp32", fused=True)["adj"]
    assert both["fwd"][0] == plain["fwd"][0] and both["fwd"][2] == plain["fwd"][2]
    only = bench.stage_model(G, info, 1, "fp32", fused_p1=True)
    assert [s and s[0] for s in only["fwd"]] == ["spmm1", None, "spmm2", "permute2"]
    assert only["adj"] == plain["adj"]
