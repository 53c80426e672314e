"""Operator parity at the largest grids the plan accepts (Fourier 1024 per
axis, sine 512 per axis) and in the launch configuration the benchmark times
(64 instances of the 512^2 rotating grid, complex64, launch shapes from
gpe_plan_autotune), against the oracle's H psi on the same bytes."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1504_02891_gb300 as G  # noqa: E402

TOL = {G.F64: 1e-12, G.F32: 2e-5}


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def rounded(a, prec):
    if prec == G.F64:
        return a
    return a.astype(np.complex64 if np.iscomplexobj(a) else np.float32).astype(
        np.complex128 if np.iscomplexobj(a) else np.float64)


def oracle_hpsi(g, psi):
    return O.apply_hlin(g, psi) + g.beta * np.abs(psi) ** 2 * psi


MAX_CASES = [
    ("fp2d_1024_rot", W.problem(2, (1024, 1024), (-20.0, -20.0), (20.0, 20.0), "fourier", beta=800.0,
                                omega=0.7, is_complex=True)),
    ("sp2d_512", W.problem(2, (512, 512), (-16.0, -16.0), (16.0, 16.0), "sine", beta=500.0,
                           potential={"kind": "lattice", "gamma": (1.0, 1.0), "depth": 50.0, "k": np.pi / 4})),
    ("fp1d_1024", W.problem(1, (1024,), (-20.0,), (20.0,), "fourier", beta=300.0)),
]


@pytest.mark.parametrize("prec", [G.F64, G.F32], ids=["f64", "f32"])
@pytest.mark.parametrize("name,p", MAX_CASES, ids=[c[0] for c in MAX_CASES])
def test_largest_grids_operator_parity(name, p, prec):
    g = O.build_grid(p)
    psi = rounded(W.random_field(p, seed=5, smooth=0.02), prec)
    with G.Plan(p, prec=prec) as plan:
        out, (E, _) = plan.grad(G.to_device(psi, prec), with_energy=True)
        got = out.cpu().numpy().astype(np.complex128 if np.iscomplexobj(psi) else np.float64)
    assert rel(got, oracle_hpsi(g, psi)) <= TOL[prec]
    assert abs(E - O.energy(g, psi)) <= (1e-12 if prec == G.F64 else 1e-5) * abs(E)


def test_benchmark_happly_configuration_parity():
    """The timed H-apply and Hessian-vector product: 64 x 512^2 complex64
    (Omega = 0.9, beta = 1000) after gpe_plan_autotune; instances 0, 31 and 63
    against the oracle, and the H-apply of the whole batch bit for bit against
    the untuned launch shapes."""
    p = W.config("c4")
    g = O.build_grid(p)
    gen = torch.Generator().manual_seed(1504)
    shift = 0.5
    with G.Plan(p, nbatch=64, prec=G.F32) as plan:
        host = torch.randn((64,) + plan.shape, dtype=torch.complex64, generator=gen) * 1e-2
        hd = torch.randn((64,) + plan.shape, dtype=torch.complex64, generator=gen)
        psi = host.cuda()
        out0 = plan.grad(psi)
        plan.autotune()
        out1 = plan.grad(psi)
        hv = plan.hessvec(psi, hd.cuda(), shift)
        torch.cuda.synchronize()
        assert torch.equal(out0, out1)
        got = out1.cpu().numpy()
        goth = hv.cpu().numpy()
    for b in (0, 31, 63):
        x = host[b].numpy().astype(np.complex128)
        d = hd[b].numpy().astype(np.complex128)
        assert rel(got[b].astype(np.complex128), oracle_hpsi(g, x)) <= TOL[G.F32], b
        refh = (O.apply_hlin(g, d) + g.beta * (np.abs(x) ** 2 * d + 2.0 * np.real(np.conj(x) * d) * x)
                + shift * d)
        assert rel(goth[b].astype(np.complex128), refh) <= TOL[G.F32], b
