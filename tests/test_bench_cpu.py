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
