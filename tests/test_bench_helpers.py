"""Host-side helpers of bench.py (no GPU): the kernel-source hash that matches a committed ncu
summary to the code it was taken on, and the summary's traffic figure."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_0907_4027_gb300" / "csrc"
    csrc.mkdir(parents=True)
    f = csrc / "gsw_kernels.cuh"
    f.write_text("int a = 1;  // one\n/* block\n comment */ int b = 2;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    f.write_text("// header\nint a = 1;   // changed comment\n\n int b = 2;\n")
    assert bench.kernel_source_hash() == h0
    f.write_text("int a = 1;\nint b = 3;\n")
    assert bench.kernel_source_hash() != h0


def test_committed_summaries_name_their_traffic():
    # every committed kernel summary carries a hash and a DRAM figure that bench.py can parse
    for kernel, workload in (("step", "rand100_512"), ("sep", "rand100_512"), ("tc", "rand1000_1920")):
        path = os.path.join(ROOT, "profiles", f"gsw_{kernel}_{workload}.md")
        txt = open(path).read()
        assert "kernel_source_sha256_16:" in txt and "dram_bytes_per_launch:" in txt
        t = bench.profiled_traffic(workload, kernel)
        assert t is None or t > 0
