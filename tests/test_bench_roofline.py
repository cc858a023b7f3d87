"""bench.py's roofline object: the CUDA-core TTM-chain against the measured HBM
copy bandwidth, the all-tensor-core chain against the TF32 rate derived from
the measured sustained BF16 rate."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402

PK = dict(hbm_gbs=6784.8, bf16=1950.8, bf16_sustained=1715.6, sm_max_mhz=2070.0, source="measured")
FP32 = 152 * 128 * 2 * 2070e6 / 1e12


def test_cuda_core_chain_is_reported_against_hbm():
    r = bench.ttm_roofline("k_ttmc_fwd", 2.0e9, 2.0e10, 1.0e-3, PK, FP32, 2_672_255_424)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(2000.0)
    assert r["frac"] == pytest.approx(2000.0 / 6784.8, abs=1e-4)
    assert r["traffic"] == 2_672_255_424
    assert r["alu_tflops"] == pytest.approx(20.0)


def test_tensor_core_chain_is_reported_against_the_tf32_rate():
    r = bench.ttm_roofline("k_ttmc_tc", 1.1e10, 1.0e12, 0.0673, PK, FP32, 123)
    peak = 1715.6 * 1.1 / 2.25
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(peak, abs=0.05)
    assert r["achieved"] == pytest.approx(1.0e12 / 0.0673 / 1e12, abs=0.005)
    assert r["frac"] == pytest.approx(r["achieved"] / peak, abs=1e-4)
    assert r["traffic"] is None  # no DRAM capture describes this kernel's full-size launch
    assert r["hbm_gbs"] == pytest.approx(1.1e10 / 0.0673 / 1e9, abs=0.05)


def test_mixed_chains_stay_on_the_hbm_roofline():
    r = bench.ttm_roofline("k_ttmc_fwd + k_ttmc_tc", 2.0e9, 2.0e10, 1.0e-3, PK, FP32, None)
    assert r["bound"] == "hbm"
