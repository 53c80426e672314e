"""Host-side pieces of bench.py that need no GPU: the roofline grouping of a
profile knows every epilogue kind the library names its kernels with."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def library_epilogue_names():
    src = open(os.path.join(ROOT, "paper_1504_02891_gb300", "csrc", "plan.cu")).read()
    m = re.search(r"epis\[\]\s*=\s*\{([^}]*)\}", src)
    return re.findall(r'"(\w+)"', m.group(1))


def test_every_epilogue_kind_has_algorithmic_bytes():
    sys.path.insert(0, ROOT)
    import bench
    names = library_epilogue_names()
    assert "grad" in names and "WS" in names
    for k in names:
        assert k in bench.ALG_REALS_PER_POINT, k


def test_roofline_from_profile_of_a_solve():
    sys.path.insert(0, ROOT)
    import bench
    prof = {}
    for k in library_epilogue_names():
        prof[f"linesx_f32_r_{k}@65536"] = (10, 1.0)
        prof[f"pass_f64_c_{k}@4096"] = (5, 0.5)
    prof["linesy_f32_r_acc@65536"] = (70, 3.0)
    r = bench.roofline_from_profile(prof, {"hbm_gbs": 6780.4})
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and 0 < r["frac"] < 1
    assert r["peak"] == 6780.4


def test_traffic_record_is_used_only_for_the_kernels_it_measured(tmp_path, monkeypatch):
    """The bench's DRAM-traffic figure comes from an ncu record that names
    the SHA-256 of the kernel sources it was captured with; a record of other
    sources is reported as null, never as the current kernel's traffic."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    rec = tmp_path / "happly_traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    assert bench.measured_traffic()[0] is None                      # no record
    rec.write_text(json.dumps({"lines": {"kernel_sources_sha256": "0" * 64, "dram_bytes_per_apply": 1.0}}))
    t, why = bench.measured_traffic("lines")
    assert t is None and "changed" in why
    rec.write_text(json.dumps({"lines": {"kernel_sources_sha256": bench.kernel_sources_sha256("lines"),
                                         "dram_bytes_per_apply": 6.5e8, "capture": "test"}}))
    assert bench.measured_traffic("lines") == (6.5e8, "test")
    assert bench.measured_traffic("fused2d")[0] is None             # no record of the other kernel


def test_fused_profile_names_group_as_operator_applications():
    sys.path.insert(0, ROOT)
    import bench
    prof = {"fused2d_f32_r_WS@65536": (100, 2.0), "fused2d_f32_r_F@65536": (20, 0.5)}
    r = bench.roofline_from_profile(prof, {"hbm_gbs": 6674.2})
    assert r is not None and r["launches_per_application"] == 1.0
    assert r["achieved"] > 0
