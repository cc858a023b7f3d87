"""bench.py reports the TTM-chain's DRAM traffic from the committed ncu
summary only while the counters still describe the code: the full-size
workload, the same kernel file and the same choice of the core's chain."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _args(**kw):
    a = dict(workload=bench.WORKLOAD, nnz=None)
    a.update(kw)
    return argparse.Namespace(**a)


def test_traffic_is_reported_for_the_captured_code():
    v = bench.ttm_traffic_per_launch(_args())
    assert isinstance(v, int) and v > 1_000_000_000


def test_traffic_is_null_for_other_sizes_and_workloads():
    assert bench.ttm_traffic_per_launch(_args(nnz=20_000_000)) is None
    assert bench.ttm_traffic_per_launch(_args(workload="uniform-200x150x100-nnz20k-k8")) is None


def test_traffic_is_null_once_a_fingerprinted_source_changes(monkeypatch):
    real = bench.source_fingerprints()
    for name in real:
        changed = dict(real)
        changed[name] = "0" * 64
        monkeypatch.setattr(bench, "source_fingerprints", lambda c=changed: c)
        assert bench.ttm_traffic_per_launch(_args()) is None


def test_core_mode_fingerprint_covers_only_the_choice_function():
    fp = bench.source_fingerprints()
    assert set(fp) == {"tk_ttmc.cu", "tk_core_mode"}
    assert all(len(h) == 64 for h in fp.values())
