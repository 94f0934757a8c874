"""The DRAM traffic figures bench.py reports come from ncu captures of the
current traversal kernel source: every stored entry is keyed by workload and
kernel option set, carries the SHA-256 of trace_kernel.cuh it was measured
on, names a profile summary under profiles/ that quotes that hash and the
command that made it, and measured_traffic() returns the figure exactly when
the hash matches (and nothing for a kernel source or option set the counters
were not taken on)."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

KERNEL = os.path.join(ROOT, "paper_2305_08343_gb300", "csrc", "cuda", "trace_kernel.cuh")


def test_traffic_entries_match_the_kernel_source_and_profiles():
    sha = hashlib.sha256(open(KERNEL, "rb").read()).hexdigest()
    assert bench.MEASURED_TRAFFIC, "no measured traffic"
    for (workload, variant), (traffic, src_sha, profile) in bench.MEASURED_TRAFFIC.items():
        assert workload in bench.WORKLOADS
        text = open(os.path.join(ROOT, profile)).read()
        assert src_sha[:8] in text and "ncu " in text and "--clock-control none" in text
        if variant:
            assert f"--variant {variant}" in text, "the capture command names the option set"
        got, where = bench.measured_traffic(workload, variant)
        if src_sha == sha:
            assert got == traffic and where == profile
        else:  # measured on another kernel source: not reported
            assert got is None and where is None
        assert 1e8 < traffic < 1e11  # bytes per launch


def test_unmeasured_workload_reports_no_traffic():
    assert bench.measured_traffic("soup4m") == (None, None)
    assert bench.measured_traffic("hair12m", 2) == (None, None)


def test_traffic_bound_cases(monkeypatch):
    """traffic_bound: the chosen option set's capture decides; without one,
    the captured option sets of the same source decide when all are on chip;
    otherwise, and outside the default configuration, the bound is HBM."""
    sha = hashlib.sha256(open(KERNEL, "rb").read()).hexdigest()
    table = {("w", 0): (1e9, sha, "p"), ("w", 128): (2e9, sha, "p"),
             ("x", 0): (30e9, sha, "p")}
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", table)
    big = 50e9  # algorithmic bytes per launch
    t, src, on_chip, why = bench.traffic_bound("w", 0, big, True)
    assert (t, src, on_chip) == (1e9, "p", True) and "2.0%" in why
    t, src, on_chip, why = bench.traffic_bound("w", 1024, big, True)
    assert (t, src, on_chip) == (None, None, True) and "option set 1024" in why
    t, src, on_chip, why = bench.traffic_bound("w", 0, big, False)
    assert (t, on_chip) == (None, False)
    t, src, on_chip, why = bench.traffic_bound("x", 0, big, True)
    assert (t, on_chip) == (30e9, False)
    t, src, on_chip, why = bench.traffic_bound("x", 5, big, True)
    assert (t, on_chip) == (None, False)  # its only capture is off chip
    t, src, on_chip, why = bench.traffic_bound("soup4m", 0, big, True)
    assert (t, on_chip) == (None, False) and "no DRAM capture" in why
    # a capture of another kernel source counts for nothing
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", {("w", 0): (1e9, "0" * 64, "p")})
    assert bench.traffic_bound("w", 128, big, True)[2] is False
