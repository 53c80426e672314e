"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
and exports every entry point declared in include/gpe.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gpe_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("gpe_plan_create", "gpe_plan_destroy", "gpe_energy", "gpe_grad", "gpe_hessvec",
              "gpe_feasible_step", "gpe_rnewton_solve", "gpe_prolong", "gpe_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1504_02891_gb300 import build as B
    lib_path = B.build()
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n), n
    # error text is available without a device
    lib.gpe_last_error.restype = ctypes.c_char_p
    assert lib.gpe_last_error() is not None


def test_invalid_problem_rejected_without_device():
    """Shape validation happens on the host before any CUDA call."""
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1504_02891_gb300 import build as B
    B.build()
    import paper_1504_02891_gb300 as G
    import workloads as W
    L = G.load()
    bad = [W.problem(2, (100, 64), (-1, -1), (1, 1), "fourier"),           # not a power of two
           W.problem(2, (64, 64), (-1, -1), (1, 1), "sine", omega=0.5, is_complex=True),
           W.problem(1, (64,), (-1,), (1,), "fourier", omega=0.5, is_complex=True)]
    for p in bad:
        pr = G.Problem.from_params(p)
        h = ctypes.c_void_p()
        st = L.gpe_plan_create(ctypes.byref(pr), 1, G.F64, None, ctypes.byref(h))
        assert st == 1, (p, st)
        assert len(L.gpe_last_error()) > 0


def test_batch_rejects_unsupported_grids_without_device():
    """gpe_solve_batch validates every problem on the host before any CUDA
    call: a 3D grid, a sine grid and a grid too large for one cluster."""
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1504_02891_gb300 import build as B
    B.build()
    import paper_1504_02891_gb300 as G
    import workloads as W
    L = G.load()
    for p in (W.problem(3, (32, 32, 32), (-1,) * 3, (1,) * 3, "fourier"),
              W.problem(2, (64, 64), (-1, -1), (1, 1), "sine"),
              W.problem(2, (1024, 1024), (-1, -1), (1, 1), "fourier", omega=0.5, is_complex=True)):
        probs = (G.Problem * 1)(G.Problem.from_params(p))
        dummy = ctypes.c_void_p(16)
        ptrs = (ctypes.c_void_p * 1)(dummy)
        reps = (G.SolveReport * 1)()
        st = L.gpe_solve_batch(probs, 1, ptrs, None, reps, None)
        assert st == 1, (p["dim"], p["disc"], st)
        assert len(L.gpe_last_error()) > 0


def test_solve_options_layout_and_search_validation_without_device():
    """gpe_solve_opts_default fills the documented values (so the binding's
    structure matches the header's), and gpe_solve_batch rejects invalid
    line-search options on the host before any CUDA call."""
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1504_02891_gb300 import build as B
    B.build()
    import paper_1504_02891_gb300 as G
    import workloads as W
    L = G.load()
    o = G.SolveOpts()
    assert L.gpe_solve_opts_default(ctypes.byref(o)) == 0
    assert (o.levels, o.mode, o.k_sub, o.max_iter, o.chunk, o.cluster) == (1, 1, 200, 2000, 16, 1)
    assert (o.search, o.alpha_hat, o.eta) == (0, 1e-3, 0.85)
    p = W.problem(2, (64, 64), (-4, -4), (4, 4), "fourier")
    probs = (G.Problem * 1)(G.Problem.from_params(p))
    ptrs = (ctypes.c_void_p * 1)(ctypes.c_void_p(16))
    reps = (G.SolveReport * 1)()
    for field, value in (("search", 2), ("alpha_hat", 0.0), ("eta", 1.0), ("eta", -0.1)):
        bad = G.SolveOpts()
        L.gpe_solve_opts_default(ctypes.byref(bad))
        setattr(bad, field, value)
        st = L.gpe_solve_batch(probs, 1, ptrs, ctypes.byref(bad), reps, None)
        assert st == 1, (field, value, st)
        assert b"options" in L.gpe_last_error()


def test_autotune_rejects_bad_arguments_without_device():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1504_02891_gb300 import build as B
    B.build()
    import paper_1504_02891_gb300 as G
    L = G.load()
    assert L.gpe_plan_autotune(None, 1) == 1
    assert L.gpe_autotune_report(None, 16) == 1
    buf = ctypes.create_string_buffer(64)
    assert L.gpe_autotune_report(buf, len(buf)) == 0
