"""Host logic of bench.py on the CPU: the DRAM-traffic figure of the roofline
comes from the committed ncu summary of the contraction kernel, one line per
captured layout, and only while the kernel source has the hash recorded there."""
import hashlib
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_gemm_traffic_follows_the_committed_summary():
    txt = open(bench.GEMM_PROFILE).read()
    lines = re.findall(r"traffic_bytes_per_launch\[launches_per_step=(\d+)\]:\s*([0-9.eE+]+)", txt)
    assert lines, "the summary records traffic per layout"
    recorded = re.search(r"kernel_source_sha1:\s*([0-9a-f]+)", txt).group(1)
    current = hashlib.sha1(open(bench.GEMM_SOURCE, "rb").read()).hexdigest()
    for k, val in lines:
        got = bench.gemm_traffic(int(k))
        assert got == (float(val) if current == recorded else None)
    assert bench.gemm_traffic(97) is None  # no line for that layout
