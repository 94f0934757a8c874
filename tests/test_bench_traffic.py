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
