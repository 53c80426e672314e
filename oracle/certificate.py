"""Second-order optimality test of Lemma 3.2 (Eq. sec-opt) in FP64.

TEST INFRASTRUCTURE (see package docstring).

A stationary point X (unit norm, theta = X^* G) is a local minimiser only if
grad^2 F(X)[D, D] - theta D^* D >= 0 for every D in the tangent set
T_X = {D : X^* D = 0} (Eq. tangent-St).  The Hessian of Lemma 3.1 is linear
over the reals (it contains Re(conj(X) D)), so the quadratic form is a real
symmetric matrix on R^M (real data) or R^{2M} (complex data, real and
imaginary parts).  For complex data X^* D = 0 removes both X and iX; iX is a
zero mode of every state (phase invariance).

  * tangent_hessian_min -- the definition written out: the dense matrix of
    D -> grad^2 F[D] - theta D built column by column from Unified.hessvec,
    an orthonormal basis of T_X from a library QR, and numpy's eigvalsh of
    the restricted matrix.  Pinned (tests/test_oracle_pins.py): at beta = 0 the
    value is 2 (lambda_1 - lambda_0) at the ground state and 2 (lambda_0 -
    lambda_1) at the first excited state, lambda_i the eigenvalues of the
    dense discrete H_lin (eigh); the harmonic trap gives 2 and -2 to grid
    accuracy; complex data do not report the phase zero mode; no random
    tangent direction has a smaller Rayleigh quotient.
"""
from __future__ import annotations

import numpy as np

from .unified import Unified


def _to_real(Z, cplx):
    z = Z.ravel()
    return np.concatenate([z.real, z.imag]) if cplx else z.real.copy()


def _from_real(v, shape, cplx):
    if cplx:
        n = v.size // 2
        return (v[:n] + 1j * v[n:]).reshape(shape)
    return v.reshape(shape)


def tangent_hessian_min(grid, psi):
    """Smallest value of grad^2 F[D,D] - theta |D|^2 over unit D in T_X
    (unified units of Eq. prob, X = sqrt(h_vol) psi normalised) and its
    minimiser D (as a grid array, unit 2-norm)."""
    U = Unified(grid)
    X = U.to_X(np.asarray(psi))
    X = X / np.sqrt(float(np.real(np.vdot(X, X))))
    cplx = np.iscomplexobj(X) or grid.is_complex
    if cplx:
        X = X.astype(np.complex128)
    G = U.grad(X)
    theta = float(np.real(np.vdot(X, G)))
    shape = X.shape
    m = X.size * (2 if cplx else 1)
    K = np.empty((m, m))
    for k in range(m):
        e = np.zeros(m)
        e[k] = 1.0
        D = _from_real(e, shape, cplx)
        K[:, k] = _to_real(U.hessvec(X, D) - theta * D, cplx)
    K = 0.5 * (K + K.T)                       # symmetric up to rounding
    C = [_to_real(X, cplx)]
    if cplx:
        C.append(_to_real(1j * X, cplx))
    Qfull, _ = np.linalg.qr(np.column_stack(C), mode="complete")
    Q = Qfull[:, len(C):]                     # orthonormal basis of T_X
    w, V = np.linalg.eigh(Q.T @ K @ Q)
    D = _from_real(Q @ V[:, 0], shape, cplx)
    return float(w[0]), D
