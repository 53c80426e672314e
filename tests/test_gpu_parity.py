"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every GPU result here is compared element by element with the oracle on the
same seeded input bytes.  Tolerances: operator applications within 1e-12
(float64) and 2e-5 (float32) relative to the largest reference value;
energies/ground states as stated per test.
"""
import math

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


def host(t):
    a = t.detach().cpu().numpy()
    return a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def as_prec(a, prec):
    """The input exactly as the device sees it (rounded to the plan precision)."""
    if prec == G.F32:
        return a.astype(np.complex64 if np.iscomplexobj(a) else np.float32).astype(
            np.complex128 if np.iscomplexobj(a) else np.float64)
    return a


def oracle_hpsi(g, psi):
    return O.apply_hlin(g, psi) + g.beta * np.abs(psi) ** 2 * psi


OPERATOR_CASES = [
    # name, params
    ("fp1d", W.problem(1, (64,), (-8.0,), (8.0,), "fourier", beta=37.0)),
    ("fp1d_tiny", W.problem(1, (4,), (-2.0,), (2.0,), "fourier", beta=3.0)),
    ("fp2d_real", W.problem(2, (32, 64), (-6.0, -7.0), (6.0, 9.0), "fourier", beta=50.0,
                            potential={"kind": "harmonic", "gamma": (1.0, 1.3)})),
    ("fp2d_rot", W.problem(2, (64, 32), (-8.0, -6.0), (8.0, 6.0), "fourier", beta=80.0, omega=0.7,
                           is_complex=True)),
    ("fp2d_rot_big", W.problem(2, (256, 128), (-16.0, -12.0), (16.0, 12.0), "fourier", beta=1000.0,
                               omega=0.9, is_complex=True)),
    ("fp3d_real", W.problem(3, (16, 32, 8), (-5.0,) * 3, (5.0,) * 3, "fourier", beta=20.0)),
    ("fp3d_rot", W.problem(3, (16, 8, 16), (-5.0,) * 3, (5.0,) * 3, "fourier", beta=20.0, omega=0.4,
                           is_complex=True)),
    ("sp1d", W.problem(1, (64,), (-8.0,), (8.0,), "sine", beta=25.0,
                       potential={"kind": "lattice", "gamma": (1.0,), "depth": 25.0, "k": math.pi / 4})),
    ("sp1d_tiny", W.problem(1, (4,), (-2.0,), (2.0,), "sine", beta=1.0)),
    ("sp2d", W.problem(2, (32, 16), (-8.0, -4.0), (8.0, 4.0), "sine", beta=100.0)),
    ("sp2d_ragged", W.problem(2, (128, 128), (-16.0, -16.0), (16.0, 16.0), "sine", beta=500.0,
                              potential={"kind": "lattice", "gamma": (1.0, 1.0), "depth": 50.0, "k": math.pi / 4})),
    ("sp3d", W.problem(3, (16, 8, 32), (-8.0,) * 3, (8.0,) * 3, "sine", beta=800.0,
                       potential={"kind": "lattice", "gamma": (1.0, 1.0, 1.0), "depth": 50.0, "k": math.pi / 4})),
    ("fd1d", W.problem(1, (50,), (-8.0,), (8.0,), "fd", beta=30.0)),
    ("fd2d_rot", W.problem(2, (20, 33), (-6.0, -6.0), (6.0, 7.0), "fd", beta=10.0, omega=0.6, is_complex=True)),
    ("fd3d", W.problem(3, (10, 12, 9), (-4.0,) * 3, (4.0,) * 3, "fd", beta=5.0,
                       potential={"kind": "stirrer", "gamma": (1.0, 1.0, 2.0), "w0": 4.0, "delta": 1.0, "r0": 1.0})),
]


@pytest.mark.parametrize("prec", [G.F64, G.F32], ids=["f64", "f32"])
@pytest.mark.parametrize("name,p", OPERATOR_CASES, ids=[c[0] for c in OPERATOR_CASES])
def test_grad_energy_hessvec_parity(name, p, prec):
    g = O.build_grid(p)
    psi = as_prec(W.random_field(p, seed=11, smooth=0.02), prec)
    d = as_prec(W.random_field(p, seed=12), prec)
    with G.Plan(p, prec=prec) as plan:
        tp = G.to_device(psi, prec)
        td = G.to_device(d, prec)
        out, (E, mu) = plan.grad(tp, with_energy=True)
        ref = oracle_hpsi(g, psi)
        assert rel(host(out), ref) <= TOL[prec], name
        E2, mu2, n2 = plan.energy(tp)
        Er, mur = O.energy(g, psi), O.chem_potential(g, psi)
        etol = 1e-12 if prec == G.F64 else 1e-5
        scale = max(abs(Er), 1.0)
        assert abs(E - Er) <= etol * scale and abs(E2 - Er) <= etol * scale
        assert abs(mu - mur) <= etol * max(abs(mur), 1.0)
        assert abs(n2 - O.norm2(g, psi)) <= etol
        shift = 0.37
        hv = plan.hessvec(tp, td, shift)
        refh = (O.apply_hlin(g, d) + g.beta * (np.abs(psi) ** 2 * d + 2.0 * np.real(np.conj(psi) * d) * psi)
                + shift * d)
        assert rel(host(hv), refh) <= TOL[prec], name


@pytest.mark.parametrize("prec", [G.F64, G.F32], ids=["f64", "f32"])
def test_feasible_step_parity(prec):
    """Theorem 3.3 step with the §4 renormalisation, in grid units."""
    p = W.problem(2, (64, 64), (-8.0, -8.0), (8.0, 8.0), "fourier", beta=200.0, omega=0.5, is_complex=True)
    g = O.build_grid(p)
    psi = as_prec(W.random_field(p, seed=3, smooth=0.1), prec)
    with G.Plan(p, prec=prec) as plan:
        tp = G.to_device(psi, prec)
        hp = plan.grad(tp)
        hpsi = host(hp)
        U = O.Unified(g)
        for tau in (0.0, 1e-3, 0.02):
            out, E = plan.feasible_step(tp, hp, tau, with_energy=True)
            X, Gx = U.to_X(psi), 2.0 * math.sqrt(g.h_vol) * hpsi
            Y = O.cayley_step(X, Gx, tau)
            Y = Y / np.linalg.norm(Y)
            ref = U.to_psi(Y)
            assert rel(host(out), ref) <= (1e-12 if prec == G.F64 else 2e-6)
            assert abs(O.norm2(g, host(out)) - 1.0) <= (1e-13 if prec == G.F64 else 1e-6)
            assert abs(E - O.energy(g, as_prec(host(out), prec))) <= (1e-11 if prec == G.F64 else 1e-5) * abs(E)


@pytest.mark.parametrize("disc,dim,cplx", [("fourier", 2, False), ("fourier", 2, True), ("sine", 2, False),
                                           ("sine", 3, False), ("fd", 2, False), ("fourier", 1, False)])
def test_prolong_parity(disc, dim, cplx):
    """Algorithm 3 transfer (reading: spectral zero-padding / linear for FD)."""
    n = {1: (32,), 2: (16, 32), 3: (8, 16, 8)}[dim]
    lo, hi = (-6.0,) * dim, (6.0,) * dim
    pc = W.problem(dim, n, lo, hi, disc, beta=10.0, omega=0.3 if cplx else 0.0, is_complex=cplx)
    pf = W.problem(dim, tuple(2 * v for v in n), lo, hi, disc, beta=10.0, omega=0.3 if cplx else 0.0,
                   is_complex=cplx)
    gc, gf = O.build_grid(pc), O.build_grid(pf)
    psi_c = W.random_field(pc, seed=5, smooth=0.1)
    with G.Plan(pc) as plc, G.Plan(pf) as plf:
        out = plc.prolong_to(plf, G.to_device(psi_c))
        ref = O.prolong(gc, gf, psi_c)
        assert rel(host(out), ref) <= 1e-12


def test_batched_plan_matches_single_instances():
    p = W.problem(2, (32, 32), (-6.0, -6.0), (6.0, 6.0), "fourier", beta=60.0, omega=0.4, is_complex=True)
    g = O.build_grid(p)
    fields = [W.random_field(p, seed=s, smooth=0.05) for s in (1, 2, 3)]
    with G.Plan(p, nbatch=3) as plan:
        t = torch.stack([G.to_device(f) for f in fields]).contiguous()
        out, (E, mu) = plan.grad(t, with_energy=True)
        for b, f in enumerate(fields):
            assert rel(host(out[b]), oracle_hpsi(g, f)) <= 1e-12
            assert abs(E[b] - O.energy(g, f)) <= 1e-12 * abs(E[b])


def test_reductions_deterministic():
    p = W.problem(2, (128, 128), (-8.0, -8.0), (8.0, 8.0), "fourier", beta=100.0, omega=0.8, is_complex=True)
    psi = W.random_field(p, seed=9)
    with G.Plan(p, prec=G.F32) as plan:
        t = G.to_device(psi, G.F32)
        r1 = plan.energy(t)
        r2 = plan.energy(t)
        assert r1 == r2


def test_nonfinite_input_reported():
    p = W.problem(1, (32,), (-4.0,), (4.0,), "fourier", beta=1.0)
    psi = W.random_field(p, seed=1)
    psi[3] = np.nan
    with G.Plan(p) as plan:
        with pytest.raises(G.GPEError) as e:
            plan.energy(G.to_device(psi))
        assert e.value.status == 4


# ------------------------------------------------------------------ full-size sampled parity

@pytest.mark.parametrize("cfg,prec", [("c4", G.F32), ("c4", G.F64), ("c3", G.F32)])
def test_full_size_operator_parity(cfg, prec):
    """Configuration sizes (512^2 complex rotating, 128^3 sine lattice): full
    H psi vs the oracle on the same bytes."""
    p = W.config(cfg)
    g = O.build_grid(p)
    psi = as_prec(W.random_field(p, seed=21, smooth=0.02), prec)
    with G.Plan(p, prec=prec) as plan:
        out, (E, mu) = plan.grad(G.to_device(psi, prec), with_energy=True)
        ref = oracle_hpsi(g, psi)
        assert rel(host(out), ref) <= TOL[prec]
        assert abs(E - O.energy(g, psi)) <= (1e-12 if prec == G.F64 else 1e-5) * abs(E)


# ------------------------------------------------------------------ solvers

def _align_phase(a, ref):
    """Multiply a by the unit phase that best matches ref (ground states are
    unique only up to a global phase)."""
    z = np.vdot(a, ref)
    return a * (z / abs(z)) if abs(z) > 0 else a


@pytest.mark.parametrize("iters", [1, 3, 12])
def test_algorithm1_iterates_match_oracle(iters):
    """Device Algorithm 1 (float64) follows the oracle's iterates: same BB
    steps, same nonmonotone decisions, same Cayley update."""
    p = W.problem(1, (128,), (-12.0,), (12.0,), "fourier", beta=100.0)
    g = O.build_grid(p)
    U = O.Unified(g)
    psi0 = W.gaussian(p)
    r = O.feasible_gradient(U.fg, U.to_X(psi0), max_iter=iters, eps0=0.0)
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, method=1, mode=0, levels=1, max_iter=iters, eps0=0.0, res_tol=0.0)
        got = host(t)
    ref = U.to_psi(r.X)
    assert rel(got, ref) <= 1e-9
    assert abs(rep["E"] - r.F) <= 1e-12 * abs(r.F)


@pytest.mark.parametrize("iters", [1, 2, 5, 30])
def test_algorithm1_iterates_match_oracle_2d(iters):
    """Same as above on a 2D real grid (two passes per evaluation, the Cayley
    step formed while loading the first pass)."""
    p = W.config("c2")
    p["n"] = (64, 64)
    g = O.build_grid(p)
    U = O.Unified(g)
    psi0 = W.gaussian(p)
    r = O.feasible_gradient(U.fg, U.to_X(psi0), max_iter=iters, eps0=0.0)
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, method=1, mode=0, levels=1, max_iter=iters, eps0=0.0, res_tol=0.0)
        got = host(t)
    ref = U.to_psi(r.X)
    assert rel(got, ref) <= 1e-9, rel(got, ref)
    assert abs(rep["E"] - r.F) <= 1e-12 * abs(r.F)


@pytest.mark.parametrize("outer", [1, 2, 4, 8])
@pytest.mark.parametrize("delta0", [1.0, 1e-4], ids=["delta1", "delta1e-4"])
def test_regularized_newton_outer_steps_match_oracle(outer, delta0):
    """Device Algorithm 2 (float64) follows the oracle's outer steps: the
    subproblem of Eq. tr-sub by Algorithm 1, the ratio of Eq. TR-ratio in
    difference form (the device's sums against the oracle's rn_ratio_terms,
    pinned to exact differences), the acceptance of Eq. update-X and the
    regularisation update of Eq. tau-up.  A wrong ratio flips an accept or a
    delta update and the states part; a small delta0 makes early steps be
    rejected, so that branch is followed too."""
    p = W.problem(1, (128,), (-12.0,), (12.0,), "fourier", beta=100.0)
    g = O.build_grid(p)
    U = O.Unified(g)
    psi0 = W.gaussian(p)
    r = O.regularized_newton(U, U.to_X(psi0), k_init=10, k_sub=15, delta0=delta0, max_outer=outer,
                             delta_stop=0.0, res_tol=0.0, record=True)
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, method=0, mode=0, levels=1, k_init=10, k_sub=15, delta0=delta0, max_outer=outer,
                         delta_stop=0.0, res_tol=0.0)
        got = host(t)
    ref = U.to_psi(r.X)
    assert rep["outer_f64"] == outer
    assert rel(got, ref) <= 1e-8, (rel(got, ref), [h[5] for h in r.history])
    assert abs(rep["E"] - r.F) <= 1e-12 * abs(r.F)


def test_algorithm1_float32_tracks_oracle():
    """Float32 Algorithm 1 (100 iterations, 2D) reaches the oracle's float64
    energy after 100 iterations to float32 accuracy."""
    p = W.config("c2")
    p["n"] = (64, 64)
    g = O.build_grid(p)
    U = O.Unified(g)
    psi0 = W.gaussian(p)
    r = O.feasible_gradient(U.fg, U.to_X(psi0), max_iter=100, eps0=0.0)
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, method=1, mode=2, levels=1, max_iter=100, eps0=0.0, res_tol=0.0, switch_rel=0.0)
    assert abs(rep["E"] - r.F) <= 1e-4 * abs(r.F), (rep["E"], r.F)


@pytest.mark.parametrize("iters", [1, 3, 12, 40])
def test_monotone_armijo_iterates_match_oracle(iters):
    """search = 1 (Remark after Theorem 3.4, Eq. Armijo1): every search starts
    at alpha_hat and halves; the device follows the oracle's iterates."""
    p = W.problem(1, (128,), (-12.0,), (12.0,), "fourier", beta=100.0)
    g = O.build_grid(p)
    U = O.Unified(g)
    psi0 = W.gaussian(p)
    r = O.armijo_gradient(U.fg, U.to_X(psi0), alpha_hat=0.01, delta_bt=0.5, max_bt=60, max_iter=iters, eps0=0.0)
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, method=1, mode=0, levels=1, max_iter=iters, eps0=0.0, res_tol=0.0,
                         search=1, alpha_hat=0.01)
        got = host(t)
    assert rel(got, U.to_psi(r.X)) <= 1e-9
    assert abs(rep["E"] - r.F) <= 1e-12 * abs(r.F)


def test_monotone_test_with_bb_steps_matches_oracle():
    """eta = 0 in Eq. NMLS-Armijo (C^(k) = F(X^(k))) with BB first steps, 2D."""
    p = W.config("c2")
    p["n"] = (64, 64)
    g = O.build_grid(p)
    U = O.Unified(g)
    psi0 = W.gaussian(p)
    r = O.feasible_gradient(U.fg, U.to_X(psi0), eta=0.0, max_iter=20, eps0=0.0)
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, method=1, mode=0, levels=1, max_iter=20, eps0=0.0, res_tol=0.0, eta=0.0)
        got = host(t)
    assert rel(got, U.to_psi(r.X)) <= 1e-9
    assert abs(rep["E"] - r.F) <= 1e-12 * abs(r.F)


@pytest.mark.parametrize("mode", [0, 2], ids=["fp64", "fp32_cluster"])
def test_monotone_armijo_converges_to_ground_state(mode):
    """search = 1 run to convergence reaches the ground state of the default
    solver (float64 per-launch path; float32 cluster engine on 2D Fourier)."""
    p = W.problem(2, (32, 32), (-6.0, -6.0), (6.0, 6.0), "fourier", beta=50.0, omega=0.3, is_complex=True)
    psi0 = W.gaussian(p, dtype=np.complex128)
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        ref = plan.solve(t, res_tol=1e-10)
    prec = G.F64 if mode == 0 else G.F32
    with G.Plan(p, prec=prec) as plan:
        t = G.to_device(psi0, prec)
        rep = plan.solve(t, method=1, mode=mode, levels=1, max_iter=30000, eps0=0.0,
                         res_tol=1e-7 if mode == 0 else 0.0, search=1, alpha_hat=0.02,
                         switch_rel=1e-5)
    tol = 1e-10 if mode == 0 else 2e-6
    assert abs(rep["E"] - ref["E"]) <= tol * abs(ref["E"]), (rep, ref["E"])


@pytest.mark.parametrize("case", ["c2_128_fp64", "c2_128_mixed", "c3_32_fp64"])
def test_persistent_launch_matches_per_iteration_launches(case):
    """The persistent Algorithm 1 launch (grid barriers, control in every CTA)
    runs the same algorithm as one launch per pass: comparable iteration
    counts and the same state and energy to the convergence tolerance.  The per-launch path of 2D Fourier grids uses
    the register-FFT line kernels, so the two differ in rounding order."""
    cfg, n, mode = {"c2_128_fp64": ("c2", (128, 128), 0), "c2_128_mixed": ("c2", (128, 128), 1),
                    "c3_32_fp64": ("c3", (32, 32, 32), 0)}[case]
    p = W.config(cfg)
    p["n"] = n
    psi0 = W.gaussian(p)
    outs, reps = [], []
    for persistent in (0, 1):
        with G.Plan(p) as plan:
            t = G.to_device(psi0)
            reps.append(plan.solve(t, mode=mode, levels=2, res_tol=1e-9, persistent=persistent))
            outs.append(host(t))
    scale = np.abs(outs[0]).max()
    assert np.abs(outs[0] - outs[1]).max() <= 2e-8 * scale   # both stop near res 1e-9
    assert abs(reps[0]["E"] - reps[1]["E"]) <= 1e-13 * abs(reps[0]["E"])
    assert abs(reps[0]["mu"] - reps[1]["mu"]) <= 1e-10 * abs(reps[0]["mu"])
    # Barzilai-Borwein runs amplify rounding differences into different step
    # sequences; the work stays comparable
    it = [r["inner_f32"] + r["inner_f64"] for r in reps]
    assert max(it) <= 1.5 * min(it) + 10, it
    for r in reps:
        assert r["status"] == 0


@pytest.mark.parametrize("case", ["real128", "rot64", "rot256", "real128x64", "rot256x128"])
def test_cluster_engine_tracks_cta_grid_path(case):
    """The float32 cluster engine (state in distributed shared memory) follows
    the CTA-grid path's Algorithm 1 iterates to float32 accuracy, and both
    agree with the float64 oracle after 60 iterations to float32 accuracy.
    Square grids take the engine's register line FFTs, the two non-square
    cases its shared-memory line stages."""
    if case == "real128":
        p = W.config("c2")
        p["n"] = (128, 128)
        psi0 = W.gaussian(p)
    elif case == "real128x64":
        p = W.problem(2, (128, 64), (-16.0, -8.0), (16.0, 8.0), "fourier", beta=400.0,
                      potential={"kind": "harmonic", "gamma": (1.0, 2.0)})
        psi0 = W.gaussian(p)
    elif case == "rot256x128":
        p = W.problem(2, (256, 128), (-16.0, -12.0), (16.0, 12.0), "fourier", beta=500.0, omega=0.6,
                      is_complex=True, potential={"kind": "harmonic", "gamma": (1.0, 1.2)})
        psi0 = W.rotating_initial(p, "c", noise=1e-2, seed=5)
    else:
        n = 64 if case == "rot64" else 256
        p = W.problem(2, (n, n), (-12.0, -12.0), (12.0, 12.0), "fourier", beta=500.0, omega=0.7,
                      is_complex=True, potential={"kind": "harmonic", "gamma": (1.0, 1.1)})
        psi0 = W.rotating_initial(p, "c", noise=1e-2, seed=5)
    g = O.build_grid(p)
    U = O.Unified(g)
    outs = {}
    for iters in (3, 400):
        for cluster in (0, 1):
            with G.Plan(p) as plan:
                t = G.to_device(psi0)
                rep = plan.solve(t, method=1, mode=2, levels=1, max_iter=iters, eps0=0.0, res_tol=0.0,
                                 switch_rel=0.0, cluster=cluster)
                outs[(iters, cluster)] = (host(t), rep["E"])
    # same iterates while float32 rounding has not yet been amplified by the
    # nonmonotone BB iteration
    assert rel(outs[(3, 1)][0], outs[(3, 0)][0]) <= 1e-4
    # the reported energy is the float64 oracle's energy of the returned state
    # (float32 arithmetic, float64 sums)
    for cluster in (0, 1):
        psi, E = outs[(400, cluster)]
        assert abs(E - O.energy(g, psi)) <= 1e-5 * abs(E), (cluster, E, O.energy(g, psi))
    if case in ("real128", "real128x64"):
        # non-rotating: both runs have converged to the oracle's minimum
        r = O.feasible_gradient(U.fg, U.to_X(psi0), max_iter=400, eps0=0.0)
        for cluster in (0, 1):
            assert abs(outs[(400, cluster)][1] - r.F) <= 1e-5 * abs(r.F), (cluster, outs[(400, cluster)][1], r.F)


def test_c1_regularized_newton_fp64():
    """Config 1 (1D Fourier 512, beta = 400): Algorithm 2 in float64 to
    ||H psi - mu psi||_h < 1e-10; E, mu, x_rms vs the oracle and §4.1's values."""
    p = W.config("c1")
    g = O.build_grid(p)
    psi0 = W.gaussian(p)
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, mode=0, levels=1, res_tol=1e-10, delta_stop=0.0)
        psi = host(t)
    U = O.Unified(g)
    ro = O.regularized_newton(U, U.to_X(psi0), res_tol=2e-10, delta_stop=0.0)
    psi_o = U.to_psi(ro.X)
    E_o = O.energy(g, psi_o)
    assert rep["res"] < 1e-10
    assert abs(rep["E"] - E_o) <= 1e-9 * E_o
    assert abs(O.energy(g, psi) - E_o) <= 1e-9 * E_o
    assert rel(psi * np.sign(np.vdot(psi, psi_o).real), psi_o) <= 1e-6
    assert abs(rep["E"] - 21.3601) <= 1e-4 and abs(rep["mu"] - 35.5775) <= 1e-4
    assert abs(O.rms(g, psi, 0) - 3.7751) <= 1e-4


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "mixed"])
def test_c2_cascade(mode):
    """Config 2 (2D Fourier 256^2, beta = 1000, cascade 64->128->256):
    float64 and float32-bulk/float64-refined solves vs the oracle's cascade."""
    p = W.config("c2")
    psi0 = W.gaussian(p)
    gf, psi_o, _ = O.cascadic(p, psi0, levels=3, method="rn", res_tol_psi=1e-10)
    E_o = O.energy(gf, psi_o)
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, mode=mode, levels=3, res_tol=1e-9)
        psi = host(t)
    assert abs(rep["E"] - E_o) <= 1e-9 * E_o, (rep, E_o)
    assert abs(O.energy(gf, psi) - E_o) <= 1e-9 * E_o
    assert rel(psi * np.sign(np.vdot(psi, psi_o).real), psi_o) <= 1e-5
    assert abs(rep["E"] - 11.9718) <= 1e-4
    if mode == 1:
        # the float32 bulk must leave only a short float64 refinement
        assert rep["outer_f64"] <= 6, rep


def test_c3_reduced_sine_lattice_mixed():
    """Config 3's discretisation and trap (sine, depth-100 lattice, beta = 1600)
    on 32^3 intervals, cascade 16 -> 32, mixed precision, vs the oracle."""
    p = W.config("c3")
    p["n"] = (32, 32, 32)
    psi0 = W.gaussian(p)
    gf, psi_o, _ = O.cascadic(p, psi0, levels=2, method="rn", res_tol_psi=1e-9)
    E_o = O.energy(gf, psi_o)
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, mode=1, levels=2, res_tol=1e-9)
        psi = host(t)
    assert abs(rep["E"] - E_o) <= 1e-9 * E_o
    assert rel(psi * np.sign(np.vdot(psi, psi_o).real), psi_o) <= 1e-5


def _certify(g, psi, rep, tol_res):
    """Oracle-side check of a GPU state: the oracle's energy and residual of the
    very same state agree with the GPU's report (1e-9 relative in E), and the
    state is stationary to tol_res in ||H psi - mu psi||_h."""
    hp = oracle_hpsi(g, psi)
    mu = O.chem_potential(g, psi)
    r = math.sqrt(O.norm2(g, hp - mu * psi))
    E = O.energy(g, psi)
    assert abs(E - rep["E"]) <= 1e-9 * abs(E), (E, rep["E"])
    assert abs(mu - rep["mu"]) <= 1e-9 * abs(mu), (mu, rep["mu"])
    assert abs(r - rep["res"]) <= 1e-2 * r + 1e-12, (r, rep["res"])
    assert r <= tol_res, r
    return E, mu, r


def test_c4_reduced_rotating_mixed():
    """Rotating config (Omega = 0.9, beta = 1000, phi_c + phase noise) on 128^2
    with the cascade 32 -> 64 -> 128 and 300 outer steps.  Rotating ground
    states are vortex lattices whose energy landscape is nearly flat (the
    isotropic trap makes lattice rotations a zero mode): the subproblems run to
    K_sub and the residual falls slowly, so the test certifies the state the
    GPU returns instead of a converged one: the oracle's energy, chemical
    potential and residual of that very state agree with the GPU's report, the
    residual fell by four orders from the initial data, and the energy lies
    near the paper's 6.3607 for this Omega and beta (Table 9; its grid is
    (-12, 12)^2 with 257^2 nodes, so only near)."""
    p = W.config("c4")
    p["n"] = (128, 128)
    g = O.build_grid(p)
    psi0 = W.rotating_initial(p, "c", noise=1e-2, seed=1504)
    r0 = math.sqrt(O.norm2(g, oracle_hpsi(g, psi0) - O.chem_potential(g, psi0) * psi0))
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, mode=1, levels=3, res_tol=1e-9, max_outer=300)
        psi = host(t)
    _certify(g, psi, rep, 1e-4 * r0)
    assert 6.358 <= rep["E"] <= 6.363, rep["E"]


def test_c4_full_size_certified():
    """Config 4 at its full size (512^2 complex, cascade 128 -> 256 -> 512),
    mixed schedule, 100 outer steps: the oracle certifies the state at full
    size (energy, chemical potential and residual as reported), the residual
    fell by three orders from the initial data, and the energy lies near the
    paper's 6.3607 (Table 9).  The run stops at its outer-step cap in one of
    the metastable lattice states (6.3602 ... 6.3629 over the rounding paths
    seen), so the band is a sanity bound, not a parity tolerance."""
    p = W.config("c4")
    g = O.build_grid(p)
    psi0 = W.rotating_initial(p, "c", noise=1e-2, seed=1504)
    r0 = math.sqrt(O.norm2(g, oracle_hpsi(g, psi0) - O.chem_potential(g, psi0) * psi0))
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, mode=1, levels=3, res_tol=1e-9, max_outer=100)
        psi = host(t)
    _certify(g, psi, rep, 1e-3 * r0)
    assert 6.358 <= rep["E"] <= 6.364, rep["E"]