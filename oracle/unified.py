"""The unified finite-dimensional problem (paper §3, Eq. prob) in FP64.

TEST INFRASTRUCTURE (see package docstring).

Rescaling (the paper says only "via a proper rescaling"; the reading taken):
X = sqrt(h_vol) * psi, A = 2 * H_lin, alpha = beta / (2 h_vol), so
that F(X) = 1/2 X^* A X + alpha sum |X_j|^4 equals E_h(psi), ||X||_2 = ||psi||_h,
grad F = 2 sqrt(h_vol) H(psi) psi and theta = X^* G = 2 mu_h.

  * F, grad           -- Eq. prob and Lemma 3.1 (first derivative).
                         Pinned: central finite differences of F; Euler
                         homogeneity Re<X,G> = X^*AX + 4 alpha sum|X|^4.
  * hessvec           -- Lemma 3.1 (second derivative).  Pinned: central
                         differences of grad; Re<X,H[X]> = X^*AX + 12 alpha sum|X|^4.
  * proj_grad         -- Eq. optim-cond, A(X)X = G X^*X - X G^*X.
  * cayley_step       -- Theorem 3.3 closed form.  Pinned: dense solve of
                         Eq. eq-Y (cayley_dense, a library linear solve of the
                         defining equation), ||Y|| = ||X||, Y(0) = X.
"""
from __future__ import annotations

import numpy as np

from .discretize import apply_hlin


class Unified:
    """F, gradient and Hessian of Eq. prob for one discretised problem."""

    def __init__(self, grid):
        self.grid = grid
        self.alpha = grid.beta / (2.0 * grid.h_vol)
        self.s = np.sqrt(grid.h_vol)

    # unit conversions -----------------------------------------------------
    def to_X(self, psi):
        return self.s * psi

    def to_psi(self, X):
        return X / self.s

    # operator -------------------------------------------------------------
    def A(self, X):
        """A X = 2 H_lin X (H_lin is linear, so units cancel)."""
        return 2.0 * apply_hlin(self.grid, X)

    def F(self, X, AX=None):
        AX = self.A(X) if AX is None else AX
        a2 = np.abs(X) ** 2
        return 0.5 * float(np.real(np.vdot(X, AX))) + self.alpha * float(np.sum(a2 * a2))

    def grad(self, X, AX=None):
        """G = A X + 4 alpha |X|^2 X   (Lemma 3.1: grad F[D] = Re<D, G>)."""
        AX = self.A(X) if AX is None else AX
        return AX + 4.0 * self.alpha * np.abs(X) ** 2 * X

    def fg(self, X):
        AX = self.A(X)
        return self.F(X, AX), self.grad(X, AX)

    def hessvec(self, X, D):
        """H[D] = A D + 4 alpha (|X|^2 D + 2 Re(conj(X) D) X)   (Lemma 3.1)."""
        return self.A(D) + 4.0 * self.alpha * (np.abs(X) ** 2 * D
                                               + 2.0 * np.real(np.conj(X) * D) * X)

    def hess_quad(self, X, D):
        """grad^2 F[D, D] as printed in Lemma 3.1."""
        a2 = np.abs(X) ** 2
        R = np.real(np.conj(X) * D)
        return (float(np.real(np.vdot(D, self.A(D))))
                + 4.0 * self.alpha * float(np.sum(a2 * np.abs(D) ** 2 + 2.0 * R * R)))


def inner(U, V):
    """Real inner product Re(U^* V) over R^{2M}."""
    return float(np.real(np.vdot(U, V)))


def proj_grad(X, G):
    """A(X) X = G (X^* X) - X (G^* X)   (Eq. optim-cond)."""
    return G * np.vdot(X, X) - X * np.vdot(G, X)


def cayley_step(X, G, tau):
    """Y(tau) = a(tau) X + b(tau) G with Theorem 3.3's coefficients, as printed:
        a = ((1 + tau X^*G)^2 - tau^2 ||X||^2 ||G||^2) / den,
        b = -2 tau ||X||^2 / den,
        den = 1 - tau^2 (X^*G)^2 + tau^2 ||X||^2 ||G||^2.

    X^* G is real for Hermitian A (the tangent-space reading for complex data);
    its real part is used.

    Guarded fallback: the printed expressions contain
    c = ||X||^2 ||G||^2 - (X^*G)^2 >= 0 (Cauchy-Schwarz) as a difference of two
    nearly equal numbers once G is almost parallel to X (near a stationary
    point c ~ ||A(X)X||^2 while ||X||^2 ||G||^2 ~ (2 mu)^2).  When more than
    half of the digits of c cancel, c is taken instead as
    ||X||^2 |G - (X^*G / ||X||^2) X|^2, the same number by Pythagoras, which
    cannot come out negative; the coefficients are then the printed ones with
    this value of c.
    """
    xg = float(np.real(np.vdot(X, G)))
    nx = float(np.real(np.vdot(X, X)))
    ng = float(np.real(np.vdot(G, G)))
    if nx * ng - xg * xg > 1e-8 * nx * ng:
        # the printed form
        den = 1.0 - tau * tau * xg * xg + tau * tau * nx * ng
        a = ((1.0 + tau * xg) ** 2 - tau * tau * nx * ng) / den
        b = -2.0 * tau * nx / den
        return a * X + b * G
    P = G - (xg / nx) * X
    cs = nx * float(np.real(np.vdot(P, P)))
    den = 1.0 + tau * tau * cs
    a = (1.0 + 2.0 * tau * xg - tau * tau * cs) / den
    b = -2.0 * tau * nx / den
    return a * X + b * G


def cayley_dense(X, G, tau):
    """Y solving (I + tau A(X)) Y = (I - tau A(X)) X with A(X) = G X^* - X G^*,
    by a dense linear solve (Eq. eq-Y); small M only."""
    M = X.size
    x = X.reshape(M, 1).astype(np.complex128)
    g = G.reshape(M, 1).astype(np.complex128)
    Acal = g @ x.conj().T - x @ g.conj().T
    I = np.eye(M)
    Y = np.linalg.solve(I + tau * Acal, (I - tau * Acal) @ x)
    return Y.reshape(X.shape)
