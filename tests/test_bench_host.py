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
            # ncu DRAM bytes at or below the algorithmic bytes (no wasted
            # re-reads), or a note that says where the excess comes from
            assert got > 0
            assert got <= bench.BYTES_PER_SITE[key] * 1.05 or "re-read" in rec.get("note", "")
        else:
            assert got is None
    assert bench.traffic_record("no_such_kernel") is None


def test_labels_follow_the_lattice_edge():
    assert bench.metric_name() == bench.METRIC
    assert bench.workload_config()["lattice"] == [bench.N_EDGE] * 3
    assert bench.metric_name(512) == "lattice site-steps/s at 512^3 coupled"
    cfg = bench.workload_config(512)
    assert cfg["lattice"] == [512] * 3 and cfg["workload"].startswith("512^3")


def test_coarse_level_fraction_counts_the_hierarchy():
    # 256 -> 128 -> 64 -> 32 -> 16 -> 8 (512 sites: the coarsest level)
    assert bench.coarse_level_fraction(256) == (128 ** 3 + 64 ** 3 + 32 ** 3 + 16 ** 3 + 8 ** 3) / 256 ** 3
    # odd extents round up: 9 -> 5 (125 sites)
    assert bench.coarse_level_fraction(9) == 125 / 729
    assert bench.coarse_level_fraction(8) == 0.0


def test_step_roofline_follows_its_formula():
    steps, sites, ms = 2, 1000, 4.0
    prof = {"pass_a": {"launches": 20, "ms": 0.0}, "residual": {"launches": 6, "ms": 0.0},
            "mg_post0": {"launches": 26, "ms": 0.0}}
    r = bench.step_roofline(prof, steps, sites, ms, 0.125)
    per_site = 70 + 13 * 3 + 40 * 10 + 13 * (29 + 33 * 0.125)
    assert abs(r["bytes_per_site"] - per_site) < 1e-9
    assert abs(r["achieved"] - per_site * sites / 4e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["counts_per_step"] == {"cg_iterations": 10, "dc_sweeps": 3, "vcycles": 13}
    assert r["frac_without_vcycle"] < r["frac"]
    design = 70 + 13 * 3 + 44 * 10 + 13 * (57 + 69 * 0.125)
    assert abs(r["design_bytes_per_site"] - design) < 1e-9
    assert abs(r["frac_design_bytes"] - design * sites / 4e-3 / 1e9 / r["peak"]) < 1e-12


def test_all_core_oracle_sample_runs_in_spawned_processes():
    value, n, wall = bench.oracle_all_cores(1, 8)
    assert n == bench.host_cores() and value > 0 and wall > 0
