"""gpe_feasible_step_noalloc: the allocation-free variant of the Cayley step
for callers that cannot call cudaMalloc (and so cannot create a plan).  Its
output must equal gpe_feasible_step's on the same inputs, call after call,
although every call shares the library's one fixed device scratch array.
This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1504_02891_gb300 as G  # noqa: E402


def _noalloc():
    L = G.load()
    f = L.gpe_feasible_step_noalloc
    f.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_double,
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


@pytest.mark.parametrize("prec,tol", [(G.F64, 1e-12), (G.F32, 2e-6)], ids=["f64", "f32"])
@pytest.mark.parametrize("cplx", [False, True], ids=["real", "complex"])
def test_noalloc_step_matches_plan_step_twice(prec, tol, cplx):
    p = W.problem(2, (64, 128), (-8.0, -8.0), (8.0, 8.0), "fourier", beta=150.0,
                  omega=0.6 if cplx else 0.0, is_complex=cplx)
    f = _noalloc()
    with G.Plan(p, nbatch=2, prec=prec) as plan:
        st = torch.cuda.current_stream()
        for call, (seed, tau) in enumerate(((1, 1e-3), (2, 4e-2))):
            fields = [W.random_field(p, seed=10 * seed + b, smooth=0.05) for b in range(2)]
            psi = torch.stack([G.to_device(a, prec) for a in fields]).contiguous()
            hpsi = plan.grad(psi)
            ref = plan.feasible_step(psi, hpsi, tau)
            out = torch.full_like(psi, float("nan"))
            rc = f(prec, 1 if cplx else 0, plan.M, 2, plan.h_vol, C.c_void_p(psi.data_ptr()),
                   C.c_void_p(hpsi.data_ptr()), tau, C.c_void_p(out.data_ptr()), C.c_void_p(st.cuda_stream))
            assert rc == 0, G.load().gpe_last_error()
            torch.cuda.synchronize()
            a = out.cpu().numpy().astype(np.complex128)
            b = ref.cpu().numpy().astype(np.complex128)
            err = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
            assert err <= tol, (call, err)
            # unit discrete norm per instance
            for k in range(2):
                n2 = plan.h_vol * float(np.sum(np.abs(a[k]) ** 2))
                assert abs(n2 - 1.0) <= (1e-12 if prec == G.F64 else 1e-5)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    f = _noalloc()
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    y = torch.zeros(16, dtype=torch.float64, device="cuda")
    z = torch.zeros(16, dtype=torch.float64, device="cuda")
    ptr = lambda t: C.c_void_p(t.data_ptr())
    assert f(G.F64, 0, 1 << 20, 65, 1.0, ptr(x), ptr(y), 0.1, ptr(z), None) == 1       # nbatch > 64
    assert f(G.F64, 0, 1 << 20, 9, 1.0, ptr(x), ptr(y), 0.1, ptr(z), None) == 1        # 9*512 blocks > 4096
    assert "4096" in G.load().gpe_last_error().decode()
