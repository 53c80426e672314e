"""Bounded device waits run out harmlessly and leave the plan usable.

Two launches wait on other CTAs or warps of the same launch: the persistent
Algorithm 1 kernel at its grid barriers, and the fused 2D operator kernel,
whose x-tasks wait for the y-tasks of their instance.  Each wait polls a
bounded number of times.  gpe_set_wait_limit(1) makes the waits give up after
one poll -- long before the CTAs or warps they wait for are done -- so the
give-up path runs without any fault or hang: the launch ends on its own, the
call returns GPE_ETIMEOUT, and the next call on the same plan, with the
default limit, gives the right result."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1504_02891_gb300 as G  # noqa: E402


def test_persistent_barrier_wait_expires_then_solve_succeeds():
    # float64 Algorithm 1 on a 2D Fourier grid runs as one cooperative
    # persistent launch with grid barriers between its passes
    p = W.problem(2, (128, 128), (-8.0, -8.0), (8.0, 8.0), "fourier", beta=200.0)
    g = O.build_grid(p)
    psi0 = W.gaussian(p)
    opts = dict(mode=0, method=1, levels=1, max_iter=300, res_tol=1e-9, persistent=1, use_graphs=1)
    with G.Plan(p, prec=G.F64) as plan:
        psi = G.to_device(psi0, G.F64)
        G.set_wait_limit(1)
        try:
            with pytest.raises(G.GPEError) as ei:
                plan.solve(psi, **opts)
            assert ei.value.status == G.ETIMEOUT
        finally:
            G.set_wait_limit(0)
        psi = G.to_device(psi0, G.F64)
        r = plan.solve(psi, **opts)
        torch.cuda.synchronize()
        got = psi.cpu().numpy()
    assert r["status"] in (0, 5)
    # the state the solve returned, re-evaluated by the oracle
    assert abs(O.energy(g, got) - r["E"]) <= 1e-10 * abs(r["E"])
    assert abs(O.norm2(g, got) - 1.0) <= 1e-12


def test_fused_task_wait_expires_then_apply_succeeds():
    p = W.problem(2, (512, 512), (-16.0, -16.0), (16.0, 16.0), "fourier", beta=1000.0, omega=0.9,
                  is_complex=True)
    g = O.build_grid(p)
    psi0 = W.random_field(p, seed=9, smooth=0.02).astype(np.complex64).astype(np.complex128)
    G.set_operator_path(1)                 # the fused kernel on this grid
    try:
        with G.Plan(p, prec=G.F32) as plan:
            psi = G.to_device(psi0, G.F32)
            G.set_wait_limit(1)
            try:
                with pytest.raises(G.GPEError) as ei:
                    plan.grad(psi, with_energy=True)
                assert ei.value.status == G.ETIMEOUT
            finally:
                G.set_wait_limit(0)
            out, (E, mu) = plan.grad(psi, with_energy=True)
            got = out.cpu().numpy().astype(np.complex128)
    finally:
        G.set_operator_path(0)
    ref = O.apply_hlin(g, psi0) + g.beta * np.abs(psi0) ** 2 * psi0
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))
    assert abs(E - O.energy(g, psi0)) <= 1e-5 * abs(E)


def test_wait_limit_rejects_negative():
    with pytest.raises(G.GPEError):
        G.set_wait_limit(-1)
