"""bench.py reads DRAM traffic and FP64-pipe utilisation from committed ncu
summaries only when they were taken on the current kernel code: the match is
by the sha1 of the source with comments and blank space removed, so edits to
comments keep a summary valid and any code change invalidates it."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SRC = """// header comment
__global__ void k(double *x)   // trailing comment
{
    /* block
       comment */
    x[0] = 1.0;

}
"""


def test_code_sha1_ignores_comments_and_blank_space():
    h = bench._code_sha1(SRC)
    edited = SRC.replace("header comment", "another header").replace("trailing comment", "")
    edited = edited.replace("    x[0] = 1.0;", "        x[0] = 1.0;\n\n")
    assert bench._code_sha1(edited) == h


def test_code_sha1_sees_code_changes():
    h = bench._code_sha1(SRC)
    assert bench._code_sha1(SRC.replace("1.0", "2.0")) != h
    assert bench._code_sha1(SRC.replace("x[0]", "x[1]")) != h


def test_fmm_summary_has_the_fields_bench_reads():
    txt = open(os.path.join(ROOT, "profiles", "fmm_secular_batched4096_dram.md")).read()
    assert "code sha1: " in txt
    for key in ("traffic_bytes: ", "fp64_pipe_pct: "):
        assert key in txt
