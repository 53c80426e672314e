"""Parity of the fused float32 operator kernel for square 2D Fourier grids
(one persistent launch of independent warps: every line FFT in one warp,
y- and x-tasks per instance) with the FP64 oracle: H psi, E, mu and the
Hessian-vector product, element by element, for every line length the kernel
takes (64 ... 1024 points), real and rotating complex data, one and several
instances per plan (tasks of several instances in flight at once)."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1504_02891_gb300 as G  # noqa: E402


@pytest.fixture(autouse=True)
def fused_path():
    # the fused kernel wherever it applies (the automatic choice may pick the
    # two line kernels for some sizes)
    G.set_operator_path(1)
    yield
    G.set_operator_path(0)

TOL = 2e-5          # float32 operator applications, relative to the largest reference value
ETOL = 1e-5         # float32 energies, relative


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def f32(a):
    return a.astype(np.complex64 if np.iscomplexobj(a) else np.float32).astype(
        np.complex128 if np.iscomplexobj(a) else np.float64)


def host(t):
    a = t.detach().cpu().numpy()
    return a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)


def case(n, cplx):
    if cplx:
        return W.problem(2, (n, n), (-10.0, -9.0), (10.0, 11.0), "fourier", beta=400.0, omega=0.8,
                         is_complex=True, potential={"kind": "harmonic", "gamma": (1.0, 1.1)})
    return W.problem(2, (n, n), (-9.0, -10.0), (9.0, 8.0), "fourier", beta=300.0,
                     potential={"kind": "harmonic", "gamma": (1.0, 1.2)})


@pytest.mark.parametrize("nbatch", [1, 3])
@pytest.mark.parametrize("cplx", [False, True], ids=["real", "complex_rotating"])
@pytest.mark.parametrize("n", [64, 128, 256, 512, 1024])
def test_fused_grad_energy_hessvec(n, cplx, nbatch):
    if n == 1024 and nbatch > 1:
        pytest.skip("one 1024^2 instance covers the size; the batch is covered below it")
    p = case(n, cplx)
    g = O.build_grid(p)
    psis = [f32(W.random_field(p, seed=31 + b, smooth=0.02)) for b in range(nbatch)]
    ds = [f32(W.random_field(p, seed=71 + b)) for b in range(nbatch)]
    with G.Plan(p, nbatch=nbatch, prec=G.F32) as plan:
        tp = torch.stack([G.to_device(a, G.F32) for a in psis]).contiguous()
        td = torch.stack([G.to_device(a, G.F32) for a in ds]).contiguous()
        out, (E, mu) = plan.grad(tp, with_energy=True)
        hv = plan.hessvec(tp, td, 0.21)
        # a second launch on the same plan: the kernel's counters were reset
        out2 = plan.grad(tp)
        torch.cuda.synchronize()
        o, h, o2 = host(out), host(hv), host(out2)
    E = np.atleast_1d(E)
    mu = np.atleast_1d(mu)
    for b in range(nbatch):
        psi, d = psis[b], ds[b]
        ref = O.apply_hlin(g, psi) + g.beta * np.abs(psi) ** 2 * psi
        ob = o[b] if nbatch > 1 else o.reshape(ref.shape)
        assert rel(ob, ref) <= TOL, (n, cplx, b)
        o2b = o2[b] if nbatch > 1 else o2.reshape(ref.shape)
        assert np.array_equal(o2b, ob)                      # same bytes, same result
        Er, mur = O.energy(g, psi), O.chem_potential(g, psi)
        assert abs(E[b] - Er) <= ETOL * max(abs(Er), 1.0)
        assert abs(mu[b] - mur) <= ETOL * max(abs(mur), 1.0)
        refh = (O.apply_hlin(g, d) + g.beta * (np.abs(psi) ** 2 * d + 2.0 * np.real(np.conj(psi) * d) * psi)
                + 0.21 * d)
        hb = h[b] if nbatch > 1 else h.reshape(refh.shape)
        assert rel(hb, refh) <= TOL, (n, cplx, b)


def test_fused_reductions_are_deterministic():
    """The task partials are folded in task order, whichever warp ran a task:
    repeated launches give bit-identical energies."""
    p = case(256, True)
    psi = f32(W.random_field(p, seed=5, smooth=0.02))
    with G.Plan(p, nbatch=4, prec=G.F32) as plan:
        tp = torch.stack([G.to_device(psi, G.F32)] * 4).contiguous()
        vals = [plan.grad(tp, with_energy=True)[1] for _ in range(5)]
    for E, mu in vals[1:]:
        assert np.array_equal(np.atleast_1d(E), np.atleast_1d(vals[0][0]))
        assert np.array_equal(np.atleast_1d(mu), np.atleast_1d(vals[0][1]))
    # the four instances hold the same data: the same sums in every slot
    E0 = np.atleast_1d(vals[0][0])
    assert np.all(E0 == E0[0])
