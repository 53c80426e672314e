"""gpe_feasible_step_noalloc: the allocation-free variant of the Cayley step
for callers that cannot call cudaMalloc (code inside an allocator or
memory-pool callback, a loop whose device memory budget was fixed up front, a
host framework that owns all device memory) and so cannot create a plan.  Its
output must equal gpe_feasible_step's on the same inputs, call after call,
although every call shares the library's one fixed device scratch array.
This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
HAVE_CUDA = torch.cuda.is_available()

import paper_1504_02891_gb300 as G  # noqa: E402


def _noalloc():
    L = G.load()
    f = L.gpe_feasible_step_noalloc
    f.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_double,
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


# Requests the fixed scratch cannot hold: (n_unknowns, nbatch).  The limits
# are nbatch <= 64 and nbatch * min(ceil(n / 256), 512) <= 4096 blocks.
OVERSIZE = [(16, 65),            # more than 64 instances
            (131072, 9),         # 9 * 512 blocks = 4608 > 4096
            (40000, 27)]         # 27 * 157 blocks = 4239 > 4096


@pytest.mark.skipif(HAVE_CUDA, reason="host-only check: the pointers below are not device buffers")
@pytest.mark.parametrize("n,nb", OVERSIZE)
def test_noalloc_rejects_oversize_before_any_device_work(n, nb):
    # The size checks run before the library touches the device or the
    # buffers, so on a machine without a GPU the call still returns
    # GPE_EINVAL (a check that moved after the device lookup would return
    # GPE_ECUDA here instead).
    f = _noalloc()
    fake = [C.c_void_p(0x1000 * (i + 1)) for i in range(3)]
    assert f(G.F64, 0, n, nb, 1.0, fake[0], fake[1], 0.1, fake[2], None) == G.EINVAL
    assert "gpe_feasible_step_noalloc" in G.load().gpe_last_error().decode()


def _compare(p, nbatch, prec, tol, calls=((1, 1e-3), (2, 4e-2))):
    f = _noalloc()
    cplx = p["is_complex"]
    with G.Plan(p, nbatch=nbatch, prec=prec) as plan:
        st = torch.cuda.current_stream()
        for call, (seed, tau) in enumerate(calls):
            fields = [W.random_field(p, seed=10 * seed + b, smooth=0.05) for b in range(nbatch)]
            psi = torch.stack([G.to_device(a, prec) for a in fields]).contiguous()
            hpsi = plan.grad(psi)
            ref = plan.feasible_step(psi, hpsi, tau)
            out = torch.full_like(psi, float("nan"))
            rc = f(prec, 1 if cplx else 0, plan.M, nbatch, plan.h_vol, C.c_void_p(psi.data_ptr()),
                   C.c_void_p(hpsi.data_ptr()), tau, C.c_void_p(out.data_ptr()), C.c_void_p(st.cuda_stream))
            assert rc == 0, G.load().gpe_last_error()
            torch.cuda.synchronize()
            a = out.cpu().numpy().astype(np.complex128)
            b = ref.cpu().numpy().astype(np.complex128)
            err = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
            assert err <= tol, (call, err)
            # unit discrete norm per instance
            for k in range(nbatch):
                n2 = plan.h_vol * float(np.sum(np.abs(a[k]) ** 2))
                assert abs(n2 - 1.0) <= (1e-12 if prec == G.F64 else 1e-5)


@pytest.mark.gpu
@pytest.mark.skipif(not HAVE_CUDA, reason="no CUDA device")
@pytest.mark.parametrize("prec,tol", [(G.F64, 1e-12), (G.F32, 2e-6)], ids=["f64", "f32"])
@pytest.mark.parametrize("cplx", [False, True], ids=["real", "complex"])
def test_noalloc_step_matches_plan_step_twice(prec, tol, cplx):
    p = W.problem(2, (64, 128), (-8.0, -8.0), (8.0, 8.0), "fourier", beta=150.0,
                  omega=0.6 if cplx else 0.0, is_complex=cplx)
    _compare(p, 2, prec, tol)


@pytest.mark.gpu
@pytest.mark.skipif(not HAVE_CUDA, reason="no CUDA device")
@pytest.mark.parametrize("shape,nbatch", [((512, 256), 8),    # 8 * 512 = 4096 blocks: the whole partials area
                                          ((64, 64), 64)],    # 64 instances: the whole results/coefficient area
                         ids=["max_blocks", "max_batch"])
def test_noalloc_step_at_its_limits(shape, nbatch):
    p = W.problem(2, shape, (-8.0, -8.0), (8.0, 8.0), "fourier", beta=150.0, omega=0.5, is_complex=True)
    _compare(p, nbatch, G.F64, 1e-12)


@pytest.mark.gpu
@pytest.mark.skipif(not HAVE_CUDA, reason="no CUDA device")
@pytest.mark.parametrize("n,nb", OVERSIZE)
def test_noalloc_rejects_sizes_beyond_its_scratch(n, nb):
    # buffers hold the whole request, so even a regressed size check could
    # not read or write outside them
    f = _noalloc()
    x = torch.zeros(n * nb, dtype=torch.float64, device="cuda")
    y = torch.zeros(n * nb, dtype=torch.float64, device="cuda")
    z = torch.zeros(n * nb, dtype=torch.float64, device="cuda")
    ptr = lambda t: C.c_void_p(t.data_ptr())
    assert f(G.F64, 0, n, nb, 1.0, ptr(x), ptr(y), 0.1, ptr(z), None) == G.EINVAL
    msg = G.load().gpe_last_error().decode()
    assert ("4096" in msg) if nb <= 64 else ("64" in msg)
