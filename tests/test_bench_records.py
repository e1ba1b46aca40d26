"""bench.py's bookkeeping, on the CPU: the recorded DRAM traffic of a stage is
reported only while the code of that stage's kernels is unchanged, and a
comment does not count as a change."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_comments_and_blank_lines_do_not_count():
    code = 'int a = 1; // one\n\n/* two\n   lines */ int b = 2;\nconst char* s = "// kept";\n'
    other = 'int a = 1; // uno\n/* dos\n   lineas */ int b = 2;\n\n\nconst char* s = "// kept";\n'
    assert bench._strip_comments(code) == bench._strip_comments(other)
    assert "one" not in bench._strip_comments(code)
    assert '"// kept"' in bench._strip_comments(code)
    assert bench._strip_comments("int a = 1;") != bench._strip_comments("int a = 2;")


def test_stage_hash_covers_its_sources_only(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2409_11765_gb300" / "csrc"
    csrc.mkdir(parents=True)
    spec = bench.STAGE_SOURCES["reduction"]
    fname, marker = spec["prefix"]
    (csrc / fname).write_text("__global__ void k_red() { int x = 1; }\n" + marker + "\n"
                              "__global__ void k_other() { int y = 2; }\n")
    for h in spec["headers"]:
        (csrc / h).write_text("constexpr int kX = 3;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.stage_sources_sha("reduction")
    # a change after the marker (another stage's kernel) or in a comment keeps the hash
    (csrc / fname).write_text("// note\n__global__ void k_red() { int x = 1; }\n" + marker + "\n"
                              "__global__ void k_other() { int y = 5; }\n")
    assert bench.stage_sources_sha("reduction") == h0
    # a change to the stage's own code, or to a header it includes, does not
    (csrc / fname).write_text("__global__ void k_red() { int x = 7; }\n" + marker + "\n")
    assert bench.stage_sources_sha("reduction") != h0
    (csrc / fname).write_text("__global__ void k_red() { int x = 1; }\n" + marker + "\n")
    (csrc / spec["headers"][0]).write_text("constexpr int kX = 4;\n")
    assert bench.stage_sources_sha("reduction") != h0
    assert bench.stage_sources_sha("no-such-stage") is None


def test_recorded_traffic_matches_the_current_sources():
    rec = bench.KERNEL_TRAFFIC.get("reduction")
    if rec is None:
        pytest.skip("no traffic recorded")
    assert rec["bytes_per_step"] > 0
    assert bench.stage_sources_sha("reduction") == rec["sources_sha256_16"], \
        "the reduction's kernels changed since their traffic was captured: re-capture it or drop the record"
