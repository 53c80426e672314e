"""The second-order certificate of Lemma 3.2 on the GPU (gpe_hess_min_eig)
against the oracle's dense tangent-space eigenvalue (oracle.tangent_hessian_min)
on the same state: ground and first excited states at beta = 0, the phase mode
of complex data, interacting and rotating states, and a full-size ground state
from the solver."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1504_02891_gb300 as G  # noqa: E402


def dense_states(g):
    M = g.V.size
    cplx = g.is_complex
    H = np.zeros((M, M), complex if cplx else float)
    for k in range(M):
        e = np.zeros(M, complex if cplx else float)
        e[k] = 1.0
        H[:, k] = O.apply_hlin(g, e.reshape(g.shape)).ravel()
    lam, vec = np.linalg.eigh(0.5 * (H + H.conj().T))
    return lam, [vec[:, i].reshape(g.shape) / np.sqrt(g.h_vol) for i in range(2)]


def gpu_cert(p, psi, prec=G.F64, **kw):
    with G.Plan(p, prec=prec) as plan:
        t = G.to_device(psi, prec)
        return plan.hess_min_eig(t, **kw)


def test_beta0_gap_at_ground_and_excited_state():
    p = W.problem(1, (64,), (-8.0,), (8.0,), "fourier", beta=0.0)
    g = O.build_grid(p)
    lam, (psi0, psi1) = dense_states(g)
    gap = lam[1] - lam[0]
    c0, r0, _ = gpu_cert(p, psi0)
    c1, r1, _ = gpu_cert(p, psi1)
    assert abs(c0 - 2.0 * gap) <= 1e-8 and r0 <= 1e-7
    assert abs(c1 + 2.0 * gap) <= 1e-8 and r1 <= 1e-7


def test_complex_phase_mode_excluded_and_matches_oracle():
    p = W.problem(2, (16, 16), (-6.0, -6.0), (6.0, 6.0), "fourier", beta=0.0, is_complex=True)
    g = O.build_grid(p)
    lam, (psi0, _) = dense_states(g)
    c, r, _ = gpu_cert(p, psi0)
    ref, _ = O.tangent_hessian_min(g, psi0)
    assert abs(c - ref) <= 1e-8 and abs(ref - 2.0 * (lam[1] - lam[0])) <= 1e-9


@pytest.mark.parametrize("prec,tol", [(G.F64, 1e-8), (G.F32, 2e-4)])
def test_interacting_ground_state_matches_oracle(prec, tol):
    p = W.problem(1, (64,), (-8.0,), (8.0,), "fourier", beta=40.0)
    g = O.build_grid(p)
    U = O.Unified(g)
    r = O.regularized_newton(U, U.to_X(W.gaussian(p)), res_tol=1e-11)
    psi = U.to_psi(r.X)
    ref, _ = O.tangent_hessian_min(g, psi)
    c, _, _ = gpu_cert(p, psi, prec)
    assert ref > 0.0
    assert abs(c - ref) <= tol * max(1.0, abs(ref)), (c, ref)


def test_rotating_arbitrary_state_matches_oracle():
    """The certificate is defined for any state (theta = X^*G): a smooth
    random complex state on a rotating 16^2 grid."""
    p = W.problem(2, (16, 16), (-6.0, -6.0), (6.0, 6.0), "fourier", beta=30.0, omega=0.5, is_complex=True)
    g = O.build_grid(p)
    psi = W.random_field(p, seed=4, smooth=0.3)
    ref, _ = O.tangent_hessian_min(g, psi)
    c, res, it = gpu_cert(p, psi, max_iter=400, tol=1e-11)
    assert abs(c - ref) <= 1e-7 * max(1.0, abs(ref)), (c, ref, res, it)


def test_solver_ground_state_certified_against_oracle():
    """A 2D ground state from the GPU's mixed solver (32^2 box of C2, beta =
    1000): the GPU certificate equals the oracle's dense value of the very
    same state and is positive (Lemma 3.2: a strict local minimiser)."""
    p = W.config("c2")
    p["n"] = (32, 32)
    g = O.build_grid(p)
    with G.Plan(p) as plan:
        t = G.to_device(W.gaussian(p))
        rep = plan.solve(t, mode=1, levels=1, res_tol=1e-10)
        c, res, it = plan.hess_min_eig(t, max_iter=400, tol=1e-11)
        psi = t.cpu().numpy()
    ref, _ = O.tangent_hessian_min(g, psi)
    assert rep["status"] == 0
    assert ref > 0.0
    assert abs(c - ref) <= 1e-7 * max(1.0, ref), (c, ref, res, it)


def test_larger_ground_state_converges():
    """64^2 (4094 tangent dimensions): the Lanczos pair converges (small true
    residual) to a positive value.  Finer grids widen the kinetic spectrum and
    need more steps (256^2: about 500, below); the residual returned says
    whether the budget sufficed."""
    p = W.config("c2")
    p["n"] = (64, 64)
    with G.Plan(p) as plan:
        t = G.to_device(W.gaussian(p))
        rep = plan.solve(t, mode=1, levels=2, res_tol=1e-9)
        c, res, it = plan.hess_min_eig(t, max_iter=600, tol=1e-9)
    assert rep["status"] == 0
    assert c > 0.0 and res <= 1e-6 * max(1.0, c), (c, res, it)


def test_full_size_config2_ground_state_certified():
    """Config 2 at its full size (256^2, 65534 tangent dimensions): with a
    Lanczos budget of 800 steps the pair converges to a small true residual,
    and the value is positive (Lemma 3.2: the solver's state is a strict
    local minimiser).  It is a property of the continuous problem resolved by
    both meshes, so the 128^2 state of the same problem gives the same value
    to a few digits (spectral accuracy)."""
    p = W.config("c2")
    vals = {}
    for n in (128, 256):
        q = dict(p)
        q["n"] = (n, n)
        with G.Plan(q) as plan:
            t = G.to_device(W.gaussian(q))
            rep = plan.solve(t, mode=1, levels=3 if n == 256 else 2, res_tol=1e-10, delta_stop=0.0)
            c, res, it = plan.hess_min_eig(t, max_iter=800, tol=1e-9)
        assert rep["status"] == 0
        assert c > 0.0 and res <= 1e-6 * max(1.0, c), (n, c, res, it)
        vals[n] = c
    assert abs(vals[256] - vals[128]) <= 1e-3 * vals[256], vals
