"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test names the passage or identity it checks.  None of them compares the
oracle with itself: closed forms, library routines (numpy.fft, dense
numpy.linalg solves/eigensolves), independent coefficient-space formulas,
printed values and finite differences.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.discretize import fourier_matrices, sine_matrix, kinetic_axis
from oracle.unified import inner

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def paper_values():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, q, v, tol, _cite = [s.strip() for s in line.split("|")]
        out[(name, q)] = (float(v), float(tol))
    return out


# ---------------------------------------------------------------- transforms

@pytest.mark.parametrize("N", [8, 16, 64])
def test_fourier_plane_wave_is_delta(N):
    """Eq. fftp36: the coefficients of e^{2 pi i j p0/N} are delta_{p,p0}."""
    fwd, inv, lam = fourier_matrices(N, 2.0)
    j = np.arange(N)
    for p0 in (-N // 2, -1, 0, 3, N // 2 - 1):
        c = fwd @ np.exp(2j * math.pi * j * p0 / N)
        e = np.zeros(N)
        e[p0 + N // 2] = 1.0
        assert np.max(np.abs(c - e)) < 1e-13


@pytest.mark.parametrize("N", [16, 32])
def test_fourier_matches_numpy_fft(N):
    """Eq. fftp36 is numpy's forward FFT / N with p reordered to -N/2..N/2-1."""
    rng = np.random.default_rng(1)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    fwd, inv, _ = fourier_matrices(N, 1.0)
    ref = np.fft.fftshift(np.fft.fft(f)) / N
    assert np.max(np.abs(fwd @ f - ref)) < 1e-14
    assert np.max(np.abs(inv @ (fwd @ f) - f)) < 1e-13


@pytest.mark.parametrize("N", [8, 32, 64])
def test_sine_involution_and_modes(N):
    """Eq. tpll: C C = (N/2) I (DST-I), and sine modes map to deltas."""
    C, lam = sine_matrix(N, 3.0)
    assert np.max(np.abs(C @ C - (N / 2.0) * np.eye(N - 1))) < 1e-12
    j = np.arange(1, N)
    for l0 in (1, 2, N - 1):
        coef = (2.0 / N) * C @ np.sin(j * l0 * math.pi / N)
        e = np.zeros(N - 1)
        e[l0 - 1] = 1.0
        assert np.max(np.abs(coef - e)) < 1e-13
    assert abs(lam[0] - math.pi / 3.0) < 1e-15


def test_spectral_second_derivative_exact_on_modes():
    """Eq. fftp35 / spdo1: -1/2 d_xx of a resolved plane wave / sine mode is exact."""
    p = W.problem(1, (32,), (-3.0,), (5.0,), "fourier", is_complex=True)
    g = O.build_grid(p)
    x = g.nodes[0]
    for q in (-15, -4, 1, 7, 15):
        lam = 2 * math.pi * q / 8.0
        f = np.exp(1j * lam * (x + 3.0))
        assert np.max(np.abs(kinetic_axis(g, f, 0) - 0.5 * lam * lam * f)) < 1e-11
    p = W.problem(1, (32,), (-3.0,), (5.0,), "sine")
    g = O.build_grid(p)
    x = g.nodes[0]
    for l in (1, 5, 31):
        lam = math.pi * l / 8.0
        f = np.sin(lam * (x + 3.0))
        assert np.max(np.abs(kinetic_axis(g, f, 0) - 0.5 * lam * lam * f)) < 1e-11


# ---------------------------------------------------------------- operator

@pytest.mark.parametrize("disc", ["fourier", "sine"])
def test_harmonic_ground_state_closed_form(disc):
    """beta = 0, Omega = 0, Eq. harmpen: prod (g/pi)^{1/4} e^{-g x^2/2} is an
    eigenfunction with eigenvalue sum g/2; spectral grids reach ~1e-13."""
    gam = (1.0, 2.0, 1.5)
    p = W.problem(3, (48, 64, 48), (-8.0,) * 3, (8.0,) * 3, disc,
                  potential={"kind": "harmonic", "gamma": gam})
    g = O.build_grid(p)
    f = np.ones(g.shape)
    for a in range(3):
        f = f * np.exp(-0.5 * gam[a] * g.mesh(a) ** 2)
    lam = sum(gam) / 2.0
    r = O.apply_hlin(g, f) - lam * f
    assert np.max(np.abs(r)) < 1e-10
    f = f / math.sqrt(O.norm2(g, f))
    assert abs(O.energy(g, f) - lam) < 1e-10


def test_rotation_sign_from_lz_eigenfunctions():
    """-Omega L_z with L_z = -i(x d_y - y d_x) (Eq. GPE): (x +- iy) e^{-r^2/2}
    has L_z = +-1, so its energy at beta = 0 is 2 -+ Omega; the isotropic
    Gaussian has L_z = 0 and energy 1."""
    om = 0.7
    p = W.problem(2, (64, 64), (-10.0, -10.0), (10.0, 10.0), "fourier", omega=om, is_complex=True)
    g = O.build_grid(p)
    x, y = g.mesh(0), g.mesh(1)
    pa = np.broadcast_to(np.exp(-(x * x + y * y) / 2) + 0j, g.shape)
    for f, lam in ((pa, 1.0), ((x + 1j * y) * pa, 2.0 - om), ((x - 1j * y) * pa, 2.0 + om)):
        assert np.max(np.abs(O.apply_hlin(g, f) - lam * f)) < 1e-12
        f = f / math.sqrt(O.norm2(g, f))
        assert abs(O.energy(g, f) - lam) < 1e-12


def test_rotation_in_3d_acts_in_xy_planes():
    """3D Fourier grid with trap (1, 1, gamma_z) and -Omega L_z: the rotation
    acts in every z-plane, so (x +- iy) e^{-(x^2+y^2)/2} e^{-gamma_z z^2/2} is
    an eigenfunction with eigenvalue (2 + gamma_z)/2 + 1 -+ Omega and the
    ground Gaussian keeps (2 + gamma_z)/2; a z-odd state z e^{...} is not
    rotated (eigenvalue (2 + gamma_z)/2 + gamma_z)."""
    om, gz = 0.6, 2.0
    p = W.problem(3, (48, 48, 64), (-8.0,) * 3, (8.0,) * 3, "fourier", omega=om, is_complex=True,
                  potential={"kind": "harmonic", "gamma": (1.0, 1.0, gz)})
    g = O.build_grid(p)
    x, y, z = g.mesh(0), g.mesh(1), g.mesh(2)
    pa = np.exp(-(x * x + y * y) / 2 - gz * z * z / 2) + 0j
    e0 = (2.0 + gz) / 2.0
    for f, lam in ((pa, e0), ((x + 1j * y) * pa, e0 + 1.0 - om), ((x - 1j * y) * pa, e0 + 1.0 + om),
                   (z * pa, e0 + gz)):
        f = np.broadcast_to(f, g.shape)
        assert np.max(np.abs(O.apply_hlin(g, f) - lam * f)) < 1e-10, lam
        f = f / math.sqrt(O.norm2(g, f))
        assert abs(O.energy(g, f) - lam) < 1e-10


def test_fd_second_order():
    """§2.1: the FD operator is second-order accurate (error ratio ~4 per halving)."""
    errs = []
    for N in (64, 128, 256):
        p = W.problem(1, (N,), (-10.0,), (10.0,), "fd")
        g = O.build_grid(p)
        f = np.exp(-g.mesh(0) ** 2 / 2)
        errs.append(np.max(np.abs(O.apply_hlin(g, f) - 0.5 * f)))
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4


def test_fd_matrix_is_paper_tridiagonal():
    """§2.1: A has a_jj = 1/h^2 + V(x_j), a_j,j+-1 = -1/(2h^2); E_h = h[Phi^T A Phi + beta/2 sum phi^4]."""
    p = W.problem(1, (10,), (-2.0,), (3.0,), "fd", beta=3.0)
    g = O.build_grid(p)
    h = g.h[0]
    M = 9
    A = np.diag(1.0 / h ** 2 + g.V) - np.diag(np.full(M - 1, 0.5 / h ** 2), 1) \
        - np.diag(np.full(M - 1, 0.5 / h ** 2), -1)
    rng = np.random.default_rng(2)
    phi = rng.standard_normal(M)
    assert np.max(np.abs(O.apply_hlin(g, phi) - A @ phi)) < 1e-12
    E = h * (phi @ A @ phi + 1.5 * np.sum(phi ** 4))
    assert abs(O.energy(g, phi) - E) < 1e-10


@pytest.mark.parametrize("case", ["fourier2d_rot", "fourier3d", "sine2d"])
def test_energy_parseval_forms(case):
    """E_h via Eq. energy-discrete-FP (coefficients, rotation folded per line) or
    Eq. BCD equals h_vol sum conj(psi) H psi + beta/2|psi|^4 on random data."""
    rng = np.random.default_rng(3)
    if case == "fourier2d_rot":
        p = W.problem(2, (16, 32), (-4.0, -5.0), (4.0, 6.0), "fourier", beta=7.0, omega=0.6,
                      is_complex=True)
    elif case == "fourier3d":
        p = W.problem(3, (8, 16, 8), (-4.0,) * 3, (4.0,) * 3, "fourier", beta=3.0)
    else:
        p = W.problem(2, (16, 12), (-4.0, -3.0), (4.0, 5.0), "sine", beta=5.0,
                      potential={"kind": "lattice", "gamma": (1.0, 1.0), "depth": 10.0, "k": 0.7})
    g = O.build_grid(p)
    psi = rng.standard_normal(g.shape)
    if g.is_complex:
        psi = psi + 1j * rng.standard_normal(g.shape)
    assert abs(O.energy(g, psi) - O.energy_parseval(g, psi)) < 1e-10 * abs(O.energy(g, psi))


def test_hermitian_operator():
    """A is Hermitian (Eq. prob): <u, H v> = conj<v, H u> on random complex data."""
    rng = np.random.default_rng(4)
    p = W.problem(2, (16, 16), (-4.0, -4.0), (4.0, 4.0), "fourier", omega=0.9, is_complex=True)
    g = O.build_grid(p)
    u = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
    v = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
    a = np.vdot(u, O.apply_hlin(g, v))
    b = np.conj(np.vdot(v, O.apply_hlin(g, u)))
    assert abs(a - b) < 1e-10 * abs(a)


# ---------------------------------------------------------------- unified problem

def _unified_case(omega=0.5, beta=30.0):
    p = W.problem(2, (8, 8), (-3.0, -3.0), (3.0, 3.0), "fourier", beta=beta, omega=omega,
                  is_complex=True)
    g = O.build_grid(p)
    U = O.Unified(g)
    rng = np.random.default_rng(5)
    X = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
    X /= np.linalg.norm(X)
    D = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
    return g, U, X, D


def test_rescaling_matches_energy():
    """Reading of 'a proper rescaling' (§3): F(sqrt(h) psi) = E_h(psi), theta = 2 mu."""
    p = W.config("c1")
    g = O.build_grid(p)
    U = O.Unified(g)
    psi = W.gaussian(p)
    X = U.to_X(psi)
    F, G = U.fg(X)
    assert abs(F - O.energy(g, psi)) < 1e-12 * F
    assert abs(inner(X, G) - 2 * O.chem_potential(g, psi)) < 1e-11 * F


def test_gradient_and_hessian_vs_finite_differences():
    """Lemma 3.1: directional derivatives agree with central differences of F
    and of the gradient (truncation O(eps^2))."""
    g, U, X, D = _unified_case()
    eps = 1e-5
    fd1 = (U.F(X + eps * D) - U.F(X - eps * D)) / (2 * eps)
    G = U.grad(X)
    assert abs(fd1 - inner(D, G)) < 1e-6 * max(1.0, abs(fd1))
    fd2 = (U.grad(X + eps * D) - U.grad(X - eps * D)) / (2 * eps)
    HD = U.hessvec(X, D)
    assert np.max(np.abs(fd2 - HD)) < 1e-5 * np.max(np.abs(HD))
    assert abs(inner(D, HD) - U.hess_quad(X, D)) < 1e-10 * abs(inner(D, HD))


def test_homogeneity_identities():
    """F = F2 + F4 with F2 quadratic, F4 quartic: Re<X,G> = X*AX + 4 alpha sum|X|^4
    and Re<X,H[X]> = X*AX + 12 alpha sum|X|^4 (Euler's theorem)."""
    g, U, X, _ = _unified_case()
    xax = inner(X, U.A(X))
    s4 = float(np.sum(np.abs(X) ** 4))
    assert abs(inner(X, U.grad(X)) - (xax + 4 * U.alpha * s4)) < 1e-10 * abs(xax)
    assert abs(inner(X, U.hessvec(X, X)) - (xax + 12 * U.alpha * s4)) < 1e-10 * abs(xax)


def test_phase_invariance_kernel():
    """F(e^{it}X) = F(X): the gradient is orthogonal to iX, and H[iX] = i G - ...:
    the derivative of G(e^{it}X) at t=0 is i G, so H[iX] = i G."""
    g, U, X, _ = _unified_case()
    G = U.grad(X)
    assert abs(inner(1j * X, G)) < 1e-10 * np.linalg.norm(G)
    assert np.max(np.abs(U.hessvec(X, 1j * X) - 1j * G)) < 1e-10 * np.max(np.abs(G))


@pytest.mark.parametrize("cplx", [False, True])
def test_cayley_closed_form_vs_dense_solve(cplx):
    """Theorem 3.3 equals the solution of Eq. eq-Y by a dense linear solve, and
    preserves the norm; Y(0) = X; Y'(0) = -2 A(X)X."""
    omega = 0.5 if cplx else 0.0
    p = W.problem(1, (12,), (-3.0,), (3.0,), "fourier", beta=20.0, omega=0.0, is_complex=cplx)
    g = O.build_grid(p)
    U = O.Unified(g)
    rng = np.random.default_rng(6)
    X = rng.standard_normal(g.shape) + (1j * rng.standard_normal(g.shape) if cplx else 0)
    X /= np.linalg.norm(X)
    G = U.grad(X)
    for tau in (0.0, 1e-3, 0.05, 0.7):
        Y = O.cayley_step(X, G, tau)
        Yd = O.cayley_dense(X, G, tau)
        assert np.max(np.abs(Y - Yd)) < 1e-12
        assert abs(np.linalg.norm(Y) - 1.0) < 1e-13
    t = 1e-6
    dY = (O.cayley_step(X, G, t) - O.cayley_step(X, G, -t)) / (2 * t)
    assert np.max(np.abs(dY + 2 * O.proj_grad(X, G))) < 1e-6 * np.max(np.abs(G))
    del omega
    # near a stationary point (G almost parallel to X) the printed coefficients
    # lose their digits and the guarded form is taken: still the dense solution
    Gs = 7.0 * X + 1e-7 * (G - inner(X, G) * X)
    for tau in (1e-3, 0.05, 0.7, 30.0):
        Y = O.cayley_step(X, Gs, tau)
        Yd = O.cayley_dense(X, Gs, tau)
        assert np.max(np.abs(Y - Yd)) < 1e-12
        assert abs(np.linalg.norm(Y) - 1.0) < 1e-13


def test_ratio_model_second_order():
    """§3.2: the RN model is F's second-order expansion, so
    |ared - (pred - delta/2 ||D||^2)| = O(||D||^3) and rho -> 1 as D -> 0."""
    g, U, X, D = _unified_case()
    G = U.grad(X)
    F0 = U.F(X)
    errs = []
    for s in (1e-2, 5e-3, 2.5e-3):
        Dd = s * D
        ared = U.F(X + Dd) - F0
        model = inner(G, Dd) + 0.5 * U.hess_quad(X, Dd)
        errs.append(abs(ared - model))
    assert 6.0 < errs[0] / errs[1] < 10.0 and 6.0 < errs[1] / errs[2] < 10.0
    # the same through the oracle's ratio terms (delta = 0.3): rho -> 1
    rhos = []
    for s in (1e-2, 1e-3, 1e-4):
        ared, pred = O.rn_ratio_terms(U, X, G, X + s * D, 0.3)
        rhos.append(ared / (pred - 0.15 * s * s * inner(D, D)))
    assert abs(rhos[2] - 1.0) < 1e-3 and abs(rhos[2] - 1.0) < abs(rhos[0] - 1.0)


# Exact arithmetic for the ratio-test pins: every float64 number is a dyadic
# rational, so with the operator written as the explicit real matrix of
# X -> A X (its columns are A applied to unit vectors) the objective and the
# model can be evaluated without rounding in fractions.Fraction.

def _real_vec(X):
    X = np.asarray(X)
    if np.iscomplexobj(X):
        return np.concatenate([X.real.ravel(), X.imag.ravel()])
    return X.ravel().astype(np.float64)


def _op_matrix(U, shape, cplx):
    """Real matrix Ahat with Re<X, A Y> = r(X) . Ahat r(Y), r = _real_vec."""
    M = int(np.prod(shape))
    cols = []
    for k in range(M):
        e = np.zeros(M)
        e[k] = 1.0
        cols.append(_real_vec(U.A(e.reshape(shape) + (0j if cplx else 0.0))))
    if cplx:
        for k in range(M):
            e = np.zeros(M, dtype=np.complex128)
            e[k] = 1j
            cols.append(_real_vec(U.A(e.reshape(shape))))
    return np.array(cols).T


def _fr(v):
    from fractions import Fraction
    return [Fraction(float(t)) for t in v]


def _exact_quad(Ah, x, y):
    """x . Ahat y in exact arithmetic (x, y lists of Fractions)."""
    from fractions import Fraction
    tot = Fraction(0)
    for i, xi in enumerate(x):
        if xi == 0:
            continue
        row = Ah[i]
        acc = Fraction(0)
        for j, yj in enumerate(y):
            if yj != 0 and row[j] != 0.0:
                acc += Fraction(float(row[j])) * yj
        tot += xi * acc
    return tot


def _exact_abs2(x, M, cplx):
    """|X_j|^2 per point from the real vector (exact)."""
    if cplx:
        return [x[j] * x[j] + x[M + j] * x[M + j] for j in range(M)]
    return [x[j] * x[j] for j in range(M)]


def _ratio_case(cplx, seed):
    omega = 0.7 if cplx else 0.0
    p = W.problem(2, (8, 8), (-3.0, -3.0), (3.0, 3.0), "fourier", beta=40.0, omega=omega, is_complex=cplx)
    g = O.build_grid(p)
    U = O.Unified(g)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal(g.shape) + (1j * rng.standard_normal(g.shape) if cplx else 0.0)
    X = X / np.linalg.norm(X)
    E = rng.standard_normal(g.shape) + (1j * rng.standard_normal(g.shape) if cplx else 0.0)
    E = E / np.linalg.norm(E)
    return g, U, X, E


@pytest.mark.parametrize("cplx", [False, True], ids=["real", "complex_rotating"])
def test_ratio_terms_equal_exact_differences(cplx):
    """Eq. TR-ratio: the oracle's difference-form numerator and denominator
    (rn_ratio_terms) equal F(Z) - F(X^k) and W(Z) - W(X^k), W the model of §3.2
    written out from its definition, evaluated here in exact rational
    arithmetic, for ||D|| = 1e-1, 1e-3, 1e-6 (beta > 0; Omega > 0 for complex
    data).  A wrong factor or sign in any term of either expression changes the
    value at first or second order in D and fails at every size."""
    from fractions import Fraction
    g, U, X, E = _ratio_case(cplx, 11)
    M = X.size
    Ah = _op_matrix(U, g.shape, cplx)
    alpha = Fraction(float(U.alpha))
    Gk = U.grad(X)
    x = _fr(_real_vec(X))
    ax = _exact_quad(Ah, x, x)
    x2 = _exact_abs2(x, M, cplx)
    for size in (1e-1, 1e-3, 1e-6):
        delta = 0.37
        D = size * E
        Z = X + D
        ared, pred = O.rn_ratio_terms(U, X, Gk, Z, delta)
        # the floats actually used: D is Z - X^k as the oracle forms it
        d = _fr(_real_vec(Z - X))
        z = [a + b for a, b in zip(x, d)]
        z2 = _exact_abs2(z, M, cplx)
        d2 = _exact_abs2(d, M, cplx)
        # F(Z) - F(X) from Eq. prob
        F_diff = (_exact_quad(Ah, z, z) - ax) / 2 + alpha * sum(a * a - b * b for a, b in zip(z2, x2))
        # W(Z) - W(X^k) from the model's definition (W(X^k) = X^k*AX^k / 2)
        if cplx:
            R = [x[j] * d[j] + x[M + j] * d[M + j] for j in range(M)]
        else:
            R = [x[j] * d[j] for j in range(M)]
        Wz = (_exact_quad(Ah, z, z) / 2 + 4 * alpha * sum(a * r for a, r in zip(x2, R))
              + 2 * alpha * sum(a * b + 2 * r * r for a, b, r in zip(x2, d2, R))
              + Fraction(delta) / 2 * sum(d2))
        W_diff = Wz - ax / 2
        # rounding scale of the float evaluation: size of its terms
        scale = size * float(np.linalg.norm(Gk)) + size * size * float(np.linalg.norm(Ah, 2))
        assert abs(ared - float(F_diff)) <= 1e-13 * scale, (size, ared, float(F_diff))
        assert abs(pred - float(W_diff)) <= 1e-13 * scale, (size, pred, float(W_diff))
        # the plain float difference cancels at small D; the difference form does not
        if size == 1e-6:
            assert abs(float(F_diff)) > 1e-9


@pytest.mark.parametrize("cplx", [False, True], ids=["real", "complex"])
def test_quartic_diff_exact(cplx):
    """sum |X+D|^4 - sum |X|^4 (the quartic part of ared), against exact
    rational arithmetic, for ||D|| from 1e-1 to 1e-8."""
    g, U, X, E = _ratio_case(cplx, 12)
    M = X.size
    x = _fr(_real_vec(X))
    x2 = _exact_abs2(x, M, cplx)
    for size in (1e-1, 1e-4, 1e-8):
        D = size * E
        q = O.quartic_diff(X, D)
        d = _fr(_real_vec(D))
        z = [a + b for a, b in zip(x, d)]          # X + D without rounding
        z2 = _exact_abs2(z, M, cplx)
        exact = float(sum(a * a - b * b for a, b in zip(z2, x2)))
        assert abs(q - exact) <= 1e-13 * (size * 4 * float(np.sum(np.abs(X) ** 3)) + size * size), (size, q, exact)


@pytest.mark.parametrize("cplx", [False, True], ids=["real", "complex_rotating"])
def test_rn_model_gradient_is_its_derivative(cplx):
    """The model gradient of §3.2 (rn_model) is the derivative of the model
    value: W is quadratic in Z, so a central difference is exact up to
    rounding, along random directions and at random points."""
    g, U, X, E = _ratio_case(cplx, 13)
    rng = np.random.default_rng(14)
    wg = O.rn_model(U, X, 0.25)
    for _ in range(3):
        Z = X + 0.1 * (rng.standard_normal(g.shape) + (1j * rng.standard_normal(g.shape) if cplx else 0.0))
        Dir = rng.standard_normal(g.shape) + (1j * rng.standard_normal(g.shape) if cplx else 0.0)
        eps = 1e-3
        Wp, _ = wg(Z + eps * Dir)
        Wm, _ = wg(Z - eps * Dir)
        _, gW = wg(Z)
        fd = (Wp - Wm) / (2 * eps)
        assert abs(fd - inner(gW, Dir)) <= 1e-8 * (abs(fd) + 1.0), (fd, inner(gW, Dir))
    # at Z = X^k the model gradient is the gradient of F (first-order match)
    _, g0 = wg(X)
    assert np.max(np.abs(g0 - U.grad(X))) <= 1e-12 * np.max(np.abs(g0))


# ---------------------------------------------------------------- solvers

def test_fg_tiny_grid_reaches_dense_eigenvalue():
    """beta = 0: min of F on the sphere is the smallest eigenvalue of A/2 = H_lin,
    here from numpy.linalg.eigh of the explicit matrix (library routine)."""
    p = W.problem(2, (8, 8), (-4.0, -4.0), (4.0, 4.0), "fourier", beta=0.0, omega=0.4,
                  is_complex=True, potential={"kind": "harmonic", "gamma": (1.0, 1.3)})
    g = O.build_grid(p)
    M = 64
    H = np.zeros((M, M), complex)
    for k in range(M):
        e = np.zeros(M, complex)
        e[k] = 1.0
        H[:, k] = O.apply_hlin(g, e.reshape(g.shape)).ravel()
    lam_min = np.linalg.eigvalsh(0.5 * (H + H.conj().T))[0]
    U = O.Unified(g)
    rng = np.random.default_rng(7)
    X0 = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
    X0 /= np.linalg.norm(X0)
    r = O.feasible_gradient(U.fg, X0, max_iter=5000, eps0=0.0, res_tol=1e-11)
    assert abs(r.F - lam_min) < 1e-10
    r2 = O.regularized_newton(U, X0, res_tol=1e-11)
    assert abs(r2.F - lam_min) < 1e-10


def test_paper_1d_values_case1_and_case2():
    """§4.1: printed E_g, mu_g, x_rms for Case I (Fourier 512, our C1 grid) and
    Case II (sine, h = 1/8)."""
    pv = paper_values()
    for name in ("c1", "1d_case2"):
        p = W.config(name)
        g = O.build_grid(p)
        U = O.Unified(g)
        r = O.feasible_gradient(U.fg, U.to_X(W.gaussian(p)), max_iter=5000, eps0=1e-12)
        psi = U.to_psi(r.X)
        got = {"E": O.energy(g, psi), "mu": O.chem_potential(g, psi), "xrms": O.rms(g, psi, 0)}
        for q, val in got.items():
            ref, tol = pv[(name, q)]
            assert abs(val - ref) <= tol, (name, q, val, ref)


def test_paper_c2_value_and_virial_and_tf():
    """§4.3 Table 9 (Omega = 0, beta = 1000): E = 11.9718 via Algorithm 3 + 2.
    Virial identity for harmonic traps (textbook): 2 E_kin - 2 E_pot + d E_int = 0.
    Thomas-Fermi limit: E -> (d+2)/(d+4) mu_TF, mu_TF = (beta/pi)^{1/2} in 2D."""
    pv = paper_values()
    p = W.config("c2")
    g, psi, res = O.cascadic(p, W.gaussian(p), levels=3, method="rn", res_tol_psi=1e-10)
    E = O.energy(g, psi)
    ref, tol = pv[("c2", "E")]
    assert abs(E - ref) <= tol
    a2 = np.abs(psi) ** 2
    from oracle.discretize import apply_kinetic
    ekin = g.h_vol * float(np.sum(np.real(np.conj(psi) * apply_kinetic(g, psi))))
    epot = g.h_vol * float(np.sum(g.V * a2))
    eint = g.h_vol * 0.5 * g.beta * float(np.sum(a2 * a2))
    assert abs(2 * ekin - 2 * epot + 2 * eint) < 1e-6 * E
    mu_tf = math.sqrt(g.beta / math.pi)
    assert abs(E - (4.0 / 6.0) * mu_tf) < 0.02 * E


def test_tf_limit_1d():
    """1D Thomas-Fermi: mu_TF = 1/2 (3 beta/2)^{2/3}, E_TF = 3/5 mu_TF (Eq. TFA)."""
    p = W.config("c1")
    g = O.build_grid(p)
    U = O.Unified(g)
    r = O.feasible_gradient(U.fg, U.to_X(W.gaussian(p)), max_iter=3000, eps0=1e-10)
    mu_tf = 0.5 * (1.5 * 400.0) ** (2.0 / 3.0)
    assert abs(r.F - 0.6 * mu_tf) < 0.01 * r.F


def test_rn_result_independent_of_delta0():
    """§3.2 says results are insensitive to the RN parameters: the final E is
    the same for delta0 = 1e-2, 1, 100."""
    p = W.problem(1, (128,), (-12.0,), (12.0,), "fourier", beta=100.0)
    g = O.build_grid(p)
    U = O.Unified(g)
    X0 = U.to_X(W.gaussian(p))
    Es = [O.regularized_newton(U, X0, delta0=d, k_init=20, res_tol=1e-11).F for d in (1e-2, 1.0, 100.0)]
    assert max(Es) - min(Es) < 1e-11 * Es[0]


# ---------------------------------------------------------------- prolongation

@pytest.mark.parametrize("disc", ["fourier", "sine"])
def test_prolongation_exact_on_band_limited_and_injects(disc):
    """Algorithm 3 transfer (reading: spectral zero-padding): a function resolved
    on the coarse grid is reproduced exactly on the fine grid; restricting back
    to the coarse nodes gives the coarse values (injection)."""
    Nc = 16
    L = 6.0
    pc = W.problem(2, (Nc, Nc), (-3.0, -3.0), (3.0, 3.0), disc)
    pf = W.problem(2, (2 * Nc, 2 * Nc), (-3.0, -3.0), (3.0, 3.0), disc)
    gc, gf = O.build_grid(pc), O.build_grid(pf)

    def f(g):
        x, y = g.mesh(0) + 3.0, g.mesh(1) + 3.0
        if disc == "fourier":
            return np.cos(2 * math.pi * 3 * x / L) * np.sin(2 * math.pi * 5 * y / L) + 0.3 * np.cos(2 * math.pi * 7 * x / L)
        return np.sin(math.pi * 2 * x / L) * np.sin(math.pi * 13 * y / L) + 0.5 * np.sin(math.pi * 15 * x / L) * np.sin(math.pi * y / L)
    fc = f(gc)
    ff = f(gf)
    pro = O.prolong(gc, gf, fc)
    scale = math.sqrt(O.norm2(gf, ff))
    assert np.max(np.abs(pro * scale - ff)) < 1e-12
    inj = O.inject(gf, gc, pro * scale)
    assert np.max(np.abs(inj - fc)) < 1e-12


def test_fd_prolongation_linear_exact():
    """FD transfer (reading: linear interpolation) reproduces piecewise-linear data."""
    pc = W.problem(1, (8,), (0.0,), (8.0,), "fd")
    pf = W.problem(1, (16,), (0.0,), (8.0,), "fd")
    gc, gf = O.build_grid(pc), O.build_grid(pf)
    tent = lambda x: np.minimum(x, 8.0 - x)
    pro = O.prolong(gc, gf, tent(gc.nodes[0]))
    ff = tent(gf.nodes[0])
    assert np.max(np.abs(pro * math.sqrt(O.norm2(gf, ff)) - ff)) < 1e-12


# ---------------------------------------------------------------- second-order certificate

def _dense_hlin(g):
    M = g.V.size
    cplx = g.is_complex
    H = np.zeros((M, M), complex if cplx else float)
    for k in range(M):
        e = np.zeros(M, complex if cplx else float)
        e[k] = 1.0
        H[:, k] = O.apply_hlin(g, e.reshape(g.shape)).ravel()
    return 0.5 * (H + H.conj().T)


def test_certificate_beta0_ground_and_first_excited_states():
    """beta = 0: grad^2 F - theta on T_X equals 2 (H_lin - lambda) restricted to
    the complement of the state, so the certificate is 2 (lambda_1 - lambda_0)
    at the ground state and 2 (lambda_0 - lambda_1) at the first excited state
    (lambda_i from numpy eigh of the explicit matrix); the 1D harmonic trap has
    lambda_1 - lambda_0 = 1 to grid accuracy (Lemma 3.2: a minimiser and a
    saddle)."""
    p = W.problem(1, (64,), (-8.0,), (8.0,), "fourier", beta=0.0)
    g = O.build_grid(p)
    lam, vec = np.linalg.eigh(_dense_hlin(g))
    gap = lam[1] - lam[0]
    assert abs(gap - 1.0) < 1e-9
    c0, D0 = O.tangent_hessian_min(g, vec[:, 0].reshape(g.shape))
    c1, _ = O.tangent_hessian_min(g, vec[:, 1].reshape(g.shape))
    assert abs(c0 - 2.0 * gap) < 1e-9
    assert abs(c1 + 2.0 * gap) < 1e-9
    # the minimiser is the first excited state (up to sign), tangent to X
    assert abs(abs(np.dot(D0.ravel(), vec[:, 1])) - 1.0) < 1e-8


def test_certificate_complex_data_exclude_the_phase_mode():
    """Complex data, beta = 0, Omega = 0, 2D harmonic: iX is tangent in the
    real sense and a zero mode, but T_X = {D : X^* D = 0} (Eq. tangent-St)
    excludes it, so the certificate is the gap 2 (lambda_1 - lambda_0) = 2."""
    p = W.problem(2, (16, 16), (-6.0, -6.0), (6.0, 6.0), "fourier", beta=0.0, is_complex=True)
    g = O.build_grid(p)
    lam, vec = np.linalg.eigh(_dense_hlin(g))
    c0, _ = O.tangent_hessian_min(g, vec[:, 0].reshape(g.shape))
    assert abs(c0 - 2.0 * (lam[1] - lam[0])) < 1e-9
    assert abs(lam[1] - lam[0] - 1.0) < 1e-4     # grid accuracy at h = 0.75


def test_certificate_3d_rotating_beta0_is_the_eigen_gap():
    """3D, rotating (Omega = 0.5), trap (1, 1, 2), beta = 0, complex data: on
    T_X the certificate is 2 (lambda_1 - lambda_0) of the explicit Hermitian
    H_lin of the same grid (numpy eigh), at the ground state; at the first
    excited state it is 2 (lambda_0 - lambda_1)."""
    p = W.problem(3, (8, 8, 8), (-5.0,) * 3, (5.0,) * 3, "fourier", beta=0.0, omega=0.5, is_complex=True,
                  potential={"kind": "harmonic", "gamma": (1.0, 1.0, 2.0)})
    g = O.build_grid(p)
    lam, vec = np.linalg.eigh(_dense_hlin(g))
    assert lam[1] - lam[0] > 1e-3                 # a simple ground state
    c0, _ = O.tangent_hessian_min(g, vec[:, 0].reshape(g.shape))
    c1, _ = O.tangent_hessian_min(g, vec[:, 1].reshape(g.shape))
    assert abs(c0 - 2.0 * (lam[1] - lam[0])) < 1e-9
    assert abs(c1 - 2.0 * (lam[0] - lam[1])) < 1e-9


def test_certificate_is_a_minimum_over_random_tangent_directions():
    """beta > 0 ground state (oracle solve): no random tangent direction has a
    smaller Rayleigh quotient of grad^2 F - theta than the certificate, and the
    certificate is positive (a strict local minimiser, Lemma 3.2 part 2)."""
    p = W.problem(1, (48,), (-8.0,), (8.0,), "fourier", beta=40.0)
    g = O.build_grid(p)
    U = O.Unified(g)
    X0 = U.to_X(W.gaussian(p))
    r = O.regularized_newton(U, X0, res_tol=1e-11)
    X = r.X
    psi = U.to_psi(X)
    c, D = O.tangent_hessian_min(g, psi)
    assert c > 0.0
    theta = float(np.real(np.vdot(X, U.grad(X))))
    rng = np.random.default_rng(11)
    for _ in range(50):
        Z = rng.standard_normal(g.shape)
        Z = Z - X * float(np.vdot(X, Z))
        Z /= np.linalg.norm(Z)
        q = U.hess_quad(X, Z) - theta
        assert q >= c - 1e-9
    q = U.hess_quad(X, D) - theta
    assert abs(q - c) < 1e-9


# ---------------------------------------------------------------- accuracy study

def _accuracy_rows(table):
    path = os.path.join(os.path.dirname(__file__), "golden", "accuracy_tables.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        t, case, disc, h, em, ee, emu = [x.strip() for x in line.split("|")]
        if t == table:
            rows.append((case, disc, float(h), float(em), float(ee), float(emu)))
    return rows


def _agrees(ours, printed):
    """Above the rounding floor within 10%; at the floor (printed < 1e-9) both small."""
    if printed < 1e-9:
        return ours < 1e-8
    return abs(ours / printed - 1.0) <= 0.10


# The paper stops Algorithm 1 at Eq. crit1 (eps0 = 1e-6): its energies carry
# all printed digits, its chemical potentials and widths a few units of the
# last one (first order in the state's error; the 3D x-widths printed after
# Table 4 lie 2e-4 below the converged ones in both cases).
LOOSE = {"mu": 5e-4, "xrms": 3e-4, "yrms": 3e-4, "zrms": 3e-4}

# §4.2 Table 4, SP at h = 2 (7 interior nodes per axis, the stirrer of width 1
# unresolved): the printed errors belong to a state whose energy is 0.187 away
# from E_g, while the discrete SP problem has a local minimiser (second-order
# certificate positive) with a lower energy than either E_g -/+ 0.187.  The row
# is checked as that inequality, not as printed.
LOWER_THAN_PRINTED = {("T4", "sine", 2.0)}


def _ground_oracle(case, disc, n):
    p, psi0 = W.accuracy_case(case, disc, n)
    g = O.build_grid(p)
    U = O.Unified(g)
    r = O.regularized_newton(U, U.to_X(psi0), res_tol=1e-11)
    psi = U.to_psi(r.X)
    psi = psi * np.sign(psi.flat[np.argmax(np.abs(psi))])
    return p, psi, O.energy(g, psi), O.chem_potential(g, psi)


@pytest.mark.parametrize("table,n_fine", [("T1", 512), ("T2", 512), ("T3", 64), ("T4", 64)])
def test_accuracy_tables(table, n_fine):
    """§4.1 Tables 1-2 and §4.2 Tables 3-4: FD (second order) and SP (spectral)
    errors of the ground state against a fine-mesh SP solution, on the paper's
    meshes, equal to the printed errors (10%, or both at rounding level).  In
    3D the fine mesh here is h = 1/4 (64 intervals per axis), so the rows at
    h = 1/4 are left to the GPU test; the 3D fine-mesh state also gives the
    energy, chemical potential and rms widths printed after Table 4."""
    rows = _accuracy_rows(table)
    case = rows[0][0]
    dim = 1 if case.startswith("1d") else 3
    L = 32.0 if dim == 1 else 16.0
    p, pex, Eex, muex = _ground_oracle(case, "sine", n_fine)
    checked = 0
    for _, disc, h, em, ee, emu in rows:
        n = int(round(L / h))
        if n >= n_fine:
            continue
        pc, psi, E, mu = _ground_oracle(case, disc, n)
        if (table, disc, h) in LOWER_THAN_PRINTED:
            assert E < Eex - ee
            assert O.tangent_hessian_min(O.build_grid(pc), psi)[0] > 0.0
            continue
        r = n_fine // n
        err = float(np.max(np.abs(pex[(slice(r - 1, None, r),) * dim] - psi)))
        for ours, printed, what in ((err, em, "max"), (abs(E - Eex), ee, "E"), (abs(mu - muex), emu, "mu")):
            assert _agrees(ours, printed), (disc, h, what, ours, printed)
        checked += 1
    assert checked >= 5
    if dim == 3:
        h = W.cell_volume(p)
        q = {"E": Eex, "mu": muex}
        for a, key in enumerate(("xrms", "yrms", "zrms")):
            x = W.axis_nodes(p, a)
            shape = [1, 1, 1]
            shape[2 - a] = x.size
            q[key] = float(np.sqrt(h * np.sum(x.reshape(shape) ** 2 * pex ** 2)))
        for (name, k), (v, tol) in paper_values().items():
            if name != case:
                continue
            assert abs(q[k] - v) <= max(tol, LOOSE.get(k, 0.0)), (case, k, q[k], v)


# ---------------------------------------------------------------- monotone Armijo search

def _tiny_rotating(beta=0.0):
    p = W.problem(2, (8, 8), (-4.0, -4.0), (4.0, 4.0), "fourier", beta=beta, omega=0.4,
                  is_complex=True, potential={"kind": "harmonic", "gamma": (1.0, 1.3)})
    g = O.build_grid(p)
    rng = np.random.default_rng(11)
    X0 = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
    return g, X0 / np.linalg.norm(X0)


def test_armijo_tiny_grid_reaches_dense_eigenvalue():
    """Remark after Theorem 3.4 (Eq. Armijo1), beta = 0: the monotone search
    reaches min F = smallest eigenvalue of H_lin (numpy eigh of the explicit
    matrix), from random data."""
    g, X0 = _tiny_rotating()
    M = X0.size
    H = np.zeros((M, M), complex)
    for k in range(M):
        e = np.zeros(M, complex)
        e[k] = 1.0
        H[:, k] = O.apply_hlin(g, e.reshape(g.shape)).ravel()
    lam_min = np.linalg.eigvalsh(0.5 * (H + H.conj().T))[0]
    U = O.Unified(g)
    r = O.armijo_gradient(U.fg, X0, alpha_hat=0.05, max_iter=20000, eps0=0.0, res_tol=1e-6)
    assert r.res <= 1e-6
    assert abs(r.F - lam_min) < 1e-9


def test_armijo_steps_are_the_armijo_points():
    """Each accepted step is alpha_hat delta^m with m the smallest integer
    meeting Eq. Armijo1 (checked by brute force: the step before it fails),
    so F decreases monotonically; interacting, rotating data."""
    g, X0 = _tiny_rotating(beta=40.0)
    U = O.Unified(g)
    ah, dl, rho1 = 0.03, 0.5, 1e-4
    X = X0
    F, G = U.fg(X)
    ms = []
    for k in range(25):
        P = O.proj_grad(X, G)
        res2 = float(np.real(np.vdot(P, P)))
        r = O.armijo_gradient(U.fg, X, alpha_hat=ah, delta_bt=dl, rho1=rho1, max_iter=1, eps0=0.0, record=True)
        tau = r.history[0][2]
        m = math.log(ah / tau) / math.log(1.0 / dl)
        assert abs(m - round(m)) < 1e-9
        ms.append(round(m))
        assert r.F <= F - rho1 * tau * res2
        if round(m) > 0:
            Y = O.cayley_step(X, G, tau / dl)
            Y = Y / math.sqrt(float(np.real(np.vdot(Y, Y))))
            assert U.fg(Y)[0] > F - rho1 * (tau / dl) * res2
        X = r.X
        F, G = U.fg(X)
    assert min(ms) == 0 and max(ms) >= 1, ms


@pytest.mark.parametrize("kind,odd_axes", [("10", (1,)), ("01", (0,)), ("11", (0, 1))])
def test_table10_parity_classes_are_invariant(kind, odd_axes):
    """§4.4 (Table 10): the asymmetric initial data are exactly odd under the
    reflections they name (reversing an array axis of the sine grid's
    symmetric interior nodes) and even under the others, and the discrete
    gradient of the energy keeps that parity, so Algorithm 1 (Cayley steps
    of X and G) stays in the class in exact arithmetic: re-imposing the
    parity only removes rounding (reading S33)."""
    p = W.config("t10")
    p["n"] = (32, 32)
    X = W.excited_initial(p, kind)
    for ax in (0, 1):
        sign = -1.0 if ax in odd_axes else 1.0
        assert np.array_equal(np.flip(X, axis=ax), sign * X), (kind, ax)
    g = O.build_grid(p)
    U = O.Unified(g)
    _, G = U.fg(U.to_X(X))
    scale = np.abs(G).max()
    for ax in (0, 1):
        sign = -1.0 if ax in odd_axes else 1.0
        assert np.abs(np.flip(G, axis=ax) - sign * G).max() <= 1e-12 * scale, (kind, ax)
