"""Host-side checks of bench.py's committed measurement records (no GPU).

The DRAM traffic the bench reports for the FP32 GMM kernels comes from a
committed ncu summary keyed by a digest of the kernels' sources; a source
change without a new capture turns the reported traffic into null. These
tests fail on the CPU when that happens, before a GPU run does."""
import importlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_traffic_records_match_the_current_sources():
    bench = _bench()
    for kernel in ("gmm_fwd", "gmm_bwd"):
        value, note = bench.traffic_record(kernel)
        assert value is not None, (kernel, note)
        assert value > 0


def test_traffic_record_reports_a_stale_digest(monkeypatch):
    bench = _bench()
    monkeypatch.setattr(bench, "source_digest", lambda kernel: "ffffffffffffffff")
    value, note = bench.traffic_record("gmm_bwd")
    assert value is None and "changed" in note
