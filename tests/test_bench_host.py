"""Host logic of bench.py that needs no GPU: the k_push source hash that gates
the recorded DRAM traffic covers the kernel source only, and the roofline
arithmetic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_source_text_drops_host_only_sections():
    text = ("// preamble\nconstexpr int A = 1;\n"
            "// --------------------------------------------------------------------------- handle\n"
            "struct pic_t { int host_only; };\n"
            "// --------------------------------------------------------------------------- device helpers\n"
            "__device__ inline int f() { return 1; }\n"
            "// --------------------------------------------------------------------------- host entry points\n"
            "int host_function(pic_t *h);\n")
    kept = bench.kernel_source_text(text)
    assert "constexpr int A = 1;" in kept and "__device__ inline int f()" in kept
    assert "host_only" not in kept and "host_function" not in kept


def test_source_hash_is_stable_and_covers_the_header_sections():
    h = bench.push_source_sha()
    assert len(h) == 16 and h == bench.push_source_sha()
    with open(os.path.join(ROOT, "paper_1308_2590_gb300/csrc/pic_internal.cuh")) as f:
        text = f.read()
    kept = bench.kernel_source_text(text)
    assert "__device__ inline void particle_moments_k" in kept      # device helpers are hashed
    assert "struct pic_t {" not in kept                              # the handle is not
    assert "int push_work_list(pic_t *h);" not in kept               # nor the host entry points
