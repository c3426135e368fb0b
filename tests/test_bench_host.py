"""Host logic of bench.py that needs no GPU: the fingerprint of the hot
kernels' code that keys the ncu traffic records, the record lookup, and the
labels of the bench line."""

import json
import os
import shutil

import bench

CSRC = ("hca_internal.cuh", "row_ops.cuh", "pcg.cu", "mg.cu")


def _copy_sources(tmp_path):
    dst = tmp_path / "paper_2105_00448_gb300" / "csrc"
    dst.mkdir(parents=True)
    for name in CSRC:
        shutil.copy(os.path.join(bench.ROOT, "paper_2105_00448_gb300", "csrc", name), dst / name)
    return dst


def test_code_lines_drop_comments_and_blanks():
    text = "// header\nint a = 1;  // trailing\n\n   \nint b = 2;\n  // indented comment\n"
    assert bench.code_lines(text) == ["int a = 1;", "int b = 2;"]


def test_fingerprint_ignores_comments_not_code(tmp_path):
    dst = _copy_sources(tmp_path)
    base = bench.kernel_source_sha(str(tmp_path))
    assert base == bench.kernel_source_sha()
    mg = dst / "mg.cu"
    text = mg.read_text()
    mg.write_text("// an added comment line\n\n" + text.replace("\n", "  // note\n", 3))
    assert bench.kernel_source_sha(str(tmp_path)) == base
    mg.write_text(text.replace("constexpr int kMgThreads = 256;", "constexpr int kMgThreads = 128;"))
    assert bench.kernel_source_sha(str(tmp_path)) != base


def test_traffic_records_match_the_current_code():
    # every committed record names a capture summary that exists; records whose
    # fingerprint differs from the current code are ignored by the bench
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        recs = json.load(f)
    for key, rec in recs.items():
        assert key in bench.BYTES_PER_SITE
        assert os.path.exists(os.path.join(bench.ROOT, rec["capture"]))
        got = bench.traffic_record(key)
        if rec["source_sha"] == bench.kernel_source_sha():
            assert got == rec["dram_bytes_per_site"]
            # ncu DRAM bytes at or below the algorithmic bytes: no wasted re-reads
            assert 0 < got <= bench.BYTES_PER_SITE[key] * 1.05
        else:
            assert got is None
    assert bench.traffic_record("no_such_kernel") is None


def test_labels_follow_the_lattice_edge():
    assert bench.metric_name() == bench.METRIC
    assert bench.workload_config()["lattice"] == [bench.N_EDGE] * 3
    assert bench.metric_name(512) == "lattice site-steps/s at 512^3 coupled"
    cfg = bench.workload_config(512)
    assert cfg["lattice"] == [512] * 3 and cfg["workload"].startswith("512^3")
