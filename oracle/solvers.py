"""Algorithms 1-3 of the paper (§3.1, §3.2, cascadic multigrid), FP64 numpy.

TEST INFRASTRUCTURE (see package docstring).

Constants the paper leaves open, and the readings taken:
  * first step tau = 1e-3; BB alternates tau^{k,1} (even k) / tau^{k,2}
    (odd k), clamped to [1e-20, 1e20] (§3.1 Eq. bb-1, "reset to a finite
    number"); the real inner product Re<S, W> is used for complex data.
  * rho1 = 1e-4, eta = 0.85, backtracking factor 0.1, at most 10 backtracks
    (Eq. NMLS-Armijo; the factor 1/2 on the BB step is kept).
  * renormalise when |X^*X - 1| > 1e-14 (§4 text).
  * RN: eta1 = 0.01, eta2 = 0.9; rho > eta2 halves delta, eta1 <= rho <= eta2
    keeps it, otherwise delta is multiplied by 4 (Eq. tau-up with gamma1 = 2,
    gamma2 = 4); delta0 = 1 (X units); delta clamped to [1e-12, 1e12].
  * The RN model W^(k) of §3.2 is taken with delta outside the alpha term
    and delta (not tau) in its gradient (the printed W and grad W are garbled).
  * The ratio's numerator and denominator are evaluated in difference form,
    algebraically identical to F(Z)-F(X) and W(Z)-W(X) (Eq. TR-ratio).
  * The subproblem (Eq. tr-sub) is solved by Algorithm 1 to
    ||A(Z)Z|| <= max(1e-2 ||A(X)X||, 1e-14) or K_sub iterations.
  * crit2 (Eq. crit2) is tested on accepted steps only.
  * Prolongation (Algorithm 3 leaves the interpolation open): Fourier --
    zero-padding of the centred spectrum with the Nyquist coefficient split
    evenly; sine -- zero-padding of the DST coefficients; FD -- linear
    interpolation; then renormalisation in ||.||_h.

  * Monotone Armijo search (Remark after Theorem 3.4): delta = 1/2, at most
    60 halvings, alpha_hat given by the caller.

Pins: rn_ratio_terms (ared, pred) equals F(Z) - F(X^k) and W(Z) - W(X^k)
evaluated in exact rational arithmetic from Eq. prob and the model's
definition, for ||D|| down to 1e-6, real and rotating complex data;
quartic_diff equals sum |X+D|^4 - |X|^4 exactly; rn_model's gradient is the
derivative of its value (central differences, exact for a quadratic) and
equals grad F at X^k; the monotone search reaches the beta = 0 dense eigenvalue and every
step it takes is the Armijo point (the step before it fails Eq. Armijo1);
Algorithm 1/2 reach the beta = 0 ground-state energy (closed form d/2,
and the smallest eigenvalue of the dense operator on tiny grids), the printed
E, mu, x_rms of §4.1, the virial identity for harmonic traps and the
Thomas-Fermi limit; prolongation is exact on band-limited data and injects.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .discretize import build_grid, fourier_matrices, sine_matrix
from .unified import Unified, cayley_step, inner, proj_grad


@dataclass
class SolveResult:
    X: np.ndarray
    F: float
    iters: int
    nfe: int
    res: float                      # ||A(X)X||_2 at exit
    history: list = field(default_factory=list)
    outer: int = 0


def feasible_gradient(fg, X0, *, tau0=1e-3, rho1=1e-4, eta=0.85, delta_bt=0.1,
                      max_bt=10, max_iter=2000, eps0=1e-6, res_tol=0.0,
                      renorm_tol=1e-14, record=False):
    """Algorithm 1 (feasible gradient method with BB steps and the
    nonmonotone curvilinear search).  ``fg(X) -> (F, G)``.

    Stops when ||X^{k+1}-X^k||_inf / tau^(k) <= eps0 (Eq. crit1), when
    ||A(X)X||_2 <= res_tol, or after max_iter iterations.
    """
    X = X0.copy()
    F, G = fg(X)
    nfe = 1
    C, Q = F, 1.0
    P = proj_grad(X, G)
    Xp = Pp = None
    hist = []
    k = 0
    while k < max_iter:
        pn = math.sqrt(inner(P, P))
        if res_tol > 0.0 and pn <= res_tol:
            break
        if k == 0:
            tau = tau0
        else:
            S = X - Xp
            W = P - Pp
            ss, sw, ww = inner(S, S), abs(inner(S, W)), inner(W, W)
            if k % 2 == 0:
                tb = ss / sw if sw > 0.0 else 1e20
            else:
                tb = sw / ww if ww > 0.0 else 1e20
            if not math.isfinite(tb):
                tb = 1e20
            tb = min(max(tb, 1e-20), 1e20)
            tau = 0.5 * tb
        thresh_rhs = rho1 * pn * pn
        for m in range(max_bt + 1):
            Y = cayley_step(X, G, tau)
            ny = inner(Y, Y)
            if abs(ny - 1.0) > renorm_tol:
                Y = Y / math.sqrt(ny)
            FY, GY = fg(Y)
            nfe += 1
            if FY <= C - tau * thresh_rhs or m == max_bt:
                break
            tau *= delta_bt
        Xp, Pp = X, P
        X, F, G = Y, FY, GY
        P = proj_grad(X, G)
        Qn = eta * Q + 1.0
        C = (eta * Q * C + F) / Qn
        Q = Qn
        k += 1
        step_inf = float(np.max(np.abs(X - Xp)))
        if record:
            hist.append((F, math.sqrt(inner(P, P)), tau, step_inf))
        if step_inf / tau <= eps0:
            break
    return SolveResult(X, F, k, nfe, math.sqrt(inner(P, P)), hist)


def armijo_gradient(fg, X0, *, alpha_hat=1.0, rho1=1e-4, delta_bt=0.5, max_bt=60,
                    max_iter=2000, eps0=1e-6, res_tol=0.0, renorm_tol=1e-14, record=False):
    """Algorithm 1 with the monotone Armijo search of the Remark after
    Theorem 3.4: tau^(k) = alpha_hat * delta^m with m the smallest nonnegative
    integer such that F(Y(tau)) <= F(X^k) - rho1 tau ||A(X^k) X^k||_2^2
    (Eq. Armijo1); then X^(k+1) = Y(tau^(k)).  Same Cayley curve, stopping
    tests and renormalisation as feasible_gradient.  At most max_bt
    reductions; the last one is taken even if the test fails (the test can
    fail only at rounding level).
    """
    X = X0.copy()
    F, G = fg(X)
    nfe = 1
    P = proj_grad(X, G)
    hist = []
    k = 0
    while k < max_iter:
        pn = math.sqrt(inner(P, P))
        if res_tol > 0.0 and pn <= res_tol:
            break
        tau = alpha_hat
        for m in range(max_bt + 1):
            Y = cayley_step(X, G, tau)
            ny = inner(Y, Y)
            if abs(ny - 1.0) > renorm_tol:
                Y = Y / math.sqrt(ny)
            FY, GY = fg(Y)
            nfe += 1
            if FY <= F - rho1 * tau * pn * pn or m == max_bt:
                break
            tau *= delta_bt
        Xp = X
        X, F, G = Y, FY, GY
        P = proj_grad(X, G)
        k += 1
        step_inf = float(np.max(np.abs(X - Xp)))
        if record:
            hist.append((F, math.sqrt(inner(P, P)), tau, step_inf))
        if step_inf / tau <= eps0:
            break
    return SolveResult(X, F, k, nfe, math.sqrt(inner(P, P)), hist)


def quartic_diff(X, D):
    """sum |X+D|^4 - sum |X|^4, written per point as a difference of squares:
    |X+D|^4 - |X|^4 = (|X+D|^2 - |X|^2)(|X+D|^2 + |X|^2) with
    |X+D|^2 - |X|^2 = 2 Re(conj(X) D) + |D|^2, so that no two large terms
    cancel when D is small."""
    x2 = np.abs(X) ** 2
    z2 = np.abs(X + D) ** 2
    return float(np.sum((2.0 * np.real(np.conj(X) * D) + np.abs(D) ** 2) * (z2 + x2)))


def rn_model(U: Unified, Xk, delta):
    """The model of §3.2 at X^k as a function of Z, with its gradient:
    W(Z) = 1/2 Z^*AZ + 4 alpha sum |X^k|^2 R + 2 alpha sum (|X^k|^2 |D|^2 + 2 R^2)
           + delta/2 ||D||^2,   D = Z - X^k,  R = Re(conj(X^k) D)
    (Eq. mL with delta taken outside the alpha term, as in the model W-tilde
    that precedes it), and
    grad W(Z) = AZ + 4 alpha |X^k|^2 Z + 8 alpha R X^k + delta D
    (the printed gradient, with delta for the printed tau).  Returns
    wg(Z) -> (W(Z), grad W(Z))."""
    alpha = U.alpha
    x2 = np.abs(Xk) ** 2

    def wg(Z):
        D = Z - Xk
        AZ = U.A(Z)
        R = np.real(np.conj(Xk) * D)
        W = (0.5 * inner(Z, AZ) + 4.0 * alpha * float(np.sum(x2 * R))
             + 2.0 * alpha * float(np.sum(x2 * np.abs(D) ** 2 + 2.0 * R * R))
             + 0.5 * delta * inner(D, D))
        gW = AZ + 4.0 * alpha * x2 * Z + 8.0 * alpha * R * Xk + delta * D
        return W, gW

    return wg


def rn_ratio_terms(U: Unified, Xk, Gk, Z, delta):
    """Numerator and denominator of Eq. TR-ratio for the trial point Z:
        ared = F(Z) - F(X^k),   pred = W(Z) - W(X^k),
    each written as a sum of terms in D = Z - X^k (no difference of two
    objective values, which would cancel near convergence):
        ared = Re<A X^k, D> + 1/2 D^*AD + alpha (sum |X^k+D|^4 - |X^k|^4)
        pred = Re<G_k, D> + 1/2 grad^2 F(X^k)[D, D] + delta/2 ||D||^2
    with A X^k = G_k - 4 alpha |X^k|^2 X^k (Lemma 3.1) and grad^2 F[D, D] as
    printed in Lemma 3.1.  Both are algebraically identical to the plain
    differences."""
    alpha = U.alpha
    x2 = np.abs(Xk) ** 2
    D = Z - Xk
    AD = U.A(D)
    AX = Gk - 4.0 * alpha * x2 * Xk
    dAd = inner(D, AD)
    R = np.real(np.conj(Xk) * D)
    ared = inner(AX, D) + 0.5 * dAd + alpha * quartic_diff(Xk, D)
    hq = dAd + 4.0 * alpha * float(np.sum(x2 * np.abs(D) ** 2 + 2.0 * R * R))
    pred = inner(Gk, D) + 0.5 * hq + 0.5 * delta * inner(D, D)
    return ared, pred


def regularized_newton(U: Unified, X0, *, k_init=100, k_sub=200, delta0=1.0,
                       eta1=0.01, eta2=0.9, gamma1=2.0, gamma2=4.0, max_outer=200,
                       delta_stop=1e-8, res_tol=0.0, sub_rel=1e-2, eps0_init=1e-6,
                       record=False):
    """Algorithm 2 (regularized Newton with the trust-region ratio test).

    Warm start: Algorithm 1 for at most k_init iterations.  Each outer step
    solves min_{||X||=1} W^(k)(X) by Algorithm 1 (<= k_sub iterations), then
    applies Eq. TR-ratio, Eq. update-X and Eq. tau-up.
    """
    r0 = feasible_gradient(U.fg, X0, max_iter=k_init, eps0=eps0_init, res_tol=res_tol)
    X = r0.X
    F, G = U.fg(X)
    nfe = r0.nfe + 1
    inner_total = r0.iters
    delta = delta0
    hist = []
    outer = 0
    while outer < max_outer:
        P = proj_grad(X, G)
        pn = math.sqrt(inner(P, P))
        if res_tol > 0.0 and pn <= res_tol:
            break
        Xk, Gk = X, G
        wg = rn_model(U, Xk, delta)
        sub = feasible_gradient(wg, Xk, max_iter=k_sub, eps0=0.0,
                                res_tol=max(sub_rel * pn, 1e-14))
        nfe += sub.nfe
        inner_total += sub.iters
        Z = sub.X
        D = Z - Xk
        ared, pred = rn_ratio_terms(U, Xk, Gk, Z, delta)
        if abs(pred) <= 1e-15 * max(abs(F), 1.0):
            rho = 1.0
        else:
            rho = ared / pred
        accepted = rho >= eta1
        step_inf = float(np.max(np.abs(D)))
        if accepted:
            X = Z
            F, G = U.fg(X)
            nfe += 1
        if rho > eta2:
            delta = delta / gamma1
        elif rho >= eta1:
            pass
        else:
            delta = delta * gamma2
        delta = min(max(delta, 1e-12), 1e12)
        outer += 1
        if record:
            hist.append((F, pn, rho, delta, sub.iters, accepted))
        if accepted and step_inf <= delta_stop:
            break
    P = proj_grad(X, G)
    return SolveResult(X, F, inner_total, nfe, math.sqrt(inner(P, P)), hist, outer)


# ---------------------------------------------------------------------------
# Algorithm 3: grid transfer and the cascade
# ---------------------------------------------------------------------------

def _fourier_prolong_axis(c_arr, ax, Nc, Nf):
    """Spectral zero-padding along one axis: evaluate the centred trigonometric
    interpolant of the coarse samples at the fine nodes."""
    fwd, _, _ = fourier_matrices(Nc, 1.0)
    p = np.arange(-Nc // 2, Nc // 2)
    m = np.arange(Nf)
    mp = np.mod(np.outer(m, p), Nf).astype(np.float64)
    E = np.exp(2j * math.pi * mp / Nf)
    # Nyquist coefficient split evenly between p = -Nc/2 and +Nc/2:
    # (e^{-i pi m Nc/Nf} + e^{+i pi m Nc/Nf})/2 = cos(pi m Nc / Nf)
    E[:, 0] = np.cos(math.pi * m * Nc / Nf)
    T = E @ fwd                                          # fine <- coarse
    moved = np.moveaxis(c_arr.astype(np.complex128), ax, -1)
    return np.moveaxis(moved @ T.T, -1, ax)


def _sine_prolong_axis(c_arr, ax, Nc, Nf):
    C, _ = sine_matrix(Nc, 1.0)
    l = np.arange(1, Nc)
    m = np.arange(1, Nf)
    ml = np.mod(np.outer(m, l), 2 * Nf).astype(np.float64)
    S = np.sin(math.pi * ml / Nf)                         # fine sine modes
    T = S @ ((2.0 / Nc) * C)
    moved = np.moveaxis(c_arr, ax, -1)
    return np.moveaxis(moved @ T.T, -1, ax)


def _fd_prolong_axis(c_arr, ax, Nc, Nf):
    r = Nf // Nc
    xc = np.arange(0, Nc + 1) * r                         # coarse nodes incl. boundary
    xf = np.arange(1, Nf)
    W = np.zeros((Nf - 1, Nc - 1))
    for i, x in enumerate(xf):
        j = x // r
        t = (x - j * r) / r
        for jj, w in ((j, 1.0 - t), (j + 1, t)):
            if 1 <= jj <= Nc - 1 and w != 0.0:
                W[i, jj - 1] += w
    del xc
    moved = np.moveaxis(c_arr, ax, -1)
    return np.moveaxis(moved @ W.T, -1, ax)


def prolong(gc, gf, psi_c):
    """Coarse -> fine grid function, then renormalised in ||.||_h (fine)."""
    out = psi_c
    for a in range(gc.dim):
        ax = gc.axis_of(a)
        Nc, Nf = gc.n[a], gf.n[a]
        if gc.disc == "fourier":
            out = _fourier_prolong_axis(out, ax, Nc, Nf)
        elif gc.disc == "sine":
            out = _sine_prolong_axis(out, ax, Nc, Nf)
        else:
            out = _fd_prolong_axis(out, ax, Nc, Nf)
    if not gf.is_complex:
        out = np.real(out)
    nrm = math.sqrt(gf.h_vol * float(np.sum(np.abs(out) ** 2)))
    return out / nrm


def inject(gf, gc, psi_f):
    """Fine -> coarse by taking the fine values at the coarse nodes."""
    sl = []
    for a in reversed(range(gf.dim)):
        r = gf.n[a] // gc.n[a]
        if gf.disc == "fourier":
            sl.append(slice(0, None, r))
        else:
            sl.append(slice(r - 1, None, r))
    return psi_f[tuple(sl)].copy()


def level_params(p, levels):
    """Parameter dicts from the coarsest to the finest mesh (halving N)."""
    out = []
    for lev in reversed(range(levels)):
        q = dict(p)
        q["n"] = tuple(n >> lev for n in p["n"])
        out.append(q)
    return out


def cascadic(p, psi0_fine, *, levels=3, method="rn", res_tol_psi=1e-10, **kw):
    """Algorithm 3: solve on the coarsest mesh, prolong, solve again.

    psi0_fine is the initial guess on the finest grid; it is injected to the
    coarsest.  ``method`` is "rn" (Algorithm 2) or "fg" (Algorithm 1).
    res_tol_psi bounds ||H psi - mu psi||_h, i.e. ||A(X)X||_2 / 2.
    Returns (grid, psi, per-level SolveResult list).
    """
    params = level_params(p, levels)
    grids = [build_grid(q) for q in params]
    psi = inject(grids[-1], grids[0], psi0_fine)
    psi = psi / math.sqrt(grids[0].h_vol * float(np.sum(np.abs(psi) ** 2)))
    results = []
    for li, g in enumerate(grids):
        if li > 0:
            psi = prolong(grids[li - 1], g, psi)
        U = Unified(g)
        X = U.to_X(psi)
        if method == "rn":
            r = regularized_newton(U, X, res_tol=2.0 * res_tol_psi, **kw)
        else:
            r = feasible_gradient(U.fg, X, res_tol=2.0 * res_tol_psi, **kw)
        results.append(r)
        psi = U.to_psi(r.X)
    return grids[-1], psi, results
