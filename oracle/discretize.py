"""Discretised energy and operator (paper §2), plain FP64 numpy.

TEST INFRASTRUCTURE (see package docstring): never imported by product code.

What each function follows, and what pins it (tests/test_oracle_*.py):
  * fourier_matrices   -- §2.3 Eq. fftp36 (forward, 1/N) and Eq. fftp35
                          (inverse), p = -N/2..N/2-1.  Pinned: plane waves map
                          to Kronecker deltas; equals numpy.fft after reordering.
  * sine_matrix        -- §2.2 Eq. tpll, c_jk = sin(jk pi/N).  Pinned:
                          C C = (N/2) I; sine modes map to deltas.
  * apply_kinetic      -- sum over axes of the per-axis spectral second
                          derivative (Eq. spdo1 / fftp35) with the rotation
                          folded into the x- and y-line symbols as in Eq.
                          energy-discrete-FP; FD: the tridiagonal of §2.1.
                          Pinned: harmonic-oscillator eigenfunctions (closed
                          form, incl. the L_z eigenfunctions (x +- iy)e^{-r^2/2}
                          whose energies 2 -+ Omega fix the rotation sign),
                          Parseval forms below, FD O(h^2) convergence.
  * energy / chem_potential / norm2 / rms -- Eq. energy-discrete-FP with unit
                          periodic weights, Eq. energy-discrete-SP-34, Eq.
                          energyFD1, Eq. chemical-potential, Eq. rms.  Pinned:
                          Parseval forms (Eq. energy-discrete-FP and Eq. BCD,
                          written independently), printed values of §4.1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np


@dataclass
class Grid:
    dim: int
    n: tuple            # paper's N per axis (points for fourier, intervals otherwise)
    lo: tuple
    hi: tuple
    disc: str           # "fourier" | "sine" | "fd"
    beta: float
    omega: float
    is_complex: bool
    h: tuple = field(default=())
    nodes: tuple = field(default=())
    shape: tuple = field(default=())
    h_vol: float = 0.0
    V: np.ndarray = None

    def axis_of(self, a):
        """numpy axis holding physical axis a (x = 0 is the last numpy axis)."""
        return self.dim - 1 - a

    def mesh(self, a):
        """Coordinate of axis a broadcast against the array shape."""
        s = [1] * self.dim
        s[self.axis_of(a)] = len(self.nodes[a])
        return self.nodes[a].reshape(s)


def potential(pot, coords):
    """External trap on the grid.

    harmonic: Eq. harmpen, V = 1/2 sum gamma_i^2 x_i^2.
    lattice:  Eq. optic98 / asypon / §4.1 Case II, harmonic + depth*sum sin^2(k x_i).
    stirrer:  §4.2 Case II, 1/2(x^2+gy^2 y^2+gz^2 z^2) + w0 exp(-delta((x-r0)^2+y^2)).
    """
    g = pot.get("gamma", (1.0, 1.0, 1.0))
    V = 0.0
    for a, x in enumerate(coords):
        V = V + 0.5 * g[a] ** 2 * x * x
    kind = pot["kind"]
    if kind == "harmonic":
        pass
    elif kind == "lattice":
        for x in coords:
            V = V + pot["depth"] * np.sin(pot["k"] * x) ** 2
    elif kind == "stirrer":
        x, y = coords[0], coords[1]
        V = V + pot["w0"] * np.exp(-pot["delta"] * ((x - pot["r0"]) ** 2 + y * y))
    else:
        raise ValueError(kind)
    return V


def build_grid(p):
    """Grid, cell volume and V from a workload parameter dict (§2)."""
    dim = p["dim"]
    h, nodes = [], []
    for a in range(dim):
        n, lo, hi = p["n"][a], p["lo"][a], p["hi"][a]
        ha = (hi - lo) / n
        j = np.arange(n) if p["disc"] == "fourier" else np.arange(1, n)
        h.append(ha)
        nodes.append(lo + j * ha)
    g = Grid(dim, tuple(p["n"]), tuple(p["lo"]), tuple(p["hi"]), p["disc"],
             float(p["beta"]), float(p["omega"]), bool(p["is_complex"]))
    g.h = tuple(h)
    g.nodes = tuple(nodes)
    g.shape = tuple(len(nodes[a]) for a in reversed(range(dim)))
    g.h_vol = float(np.prod(h))
    coords = [g.mesh(a) for a in range(dim)]
    g.V = np.broadcast_to(potential(p["potential"], coords), g.shape).astype(np.float64).copy()
    return g


# ---------------------------------------------------------------------------
# Transforms as dense matrices (plain definitions)
# ---------------------------------------------------------------------------

@lru_cache(maxsize=32)
def fourier_matrices(N, L):
    """(Fwd, Inv, lam): Fwd[p, j] = exp(-2 pi i j p/N)/N, Inv[j, p] = exp(2 pi i j p/N),
    lam_p = 2 pi p / L, for p = -N/2..N/2-1 in that order (Eq. fftp36, fftp35).
    Angles are reduced exactly: (j p mod N) / N."""
    p = np.arange(-N // 2, N // 2)
    j = np.arange(N)
    jp = np.mod(np.outer(j, p), N).astype(np.float64)
    ang = 2.0 * math.pi * jp / N                      # [j, p]
    inv = np.cos(ang) + 1j * np.sin(ang)
    fwd = np.conj(inv).T / N
    lam = 2.0 * math.pi * p / L
    return fwd, inv, lam


@lru_cache(maxsize=32)
def sine_matrix(N, L):
    """(C, lam): c_jl = sin(j l pi / N), j, l = 1..N-1; lam_l = pi l / L (Eq. tpll)."""
    j = np.arange(1, N)
    jl = np.mod(np.outer(j, j), 2 * N).astype(np.float64)
    C = np.sin(math.pi * jl / N)
    lam = math.pi * j / L
    return C, lam


def _along(M, arr, ax):
    """Apply matrix M (out x in) along numpy axis ax."""
    moved = np.moveaxis(arr, ax, -1)
    res = moved @ M.T
    return np.moveaxis(res, -1, ax)


def fourier_coeffs(grid, psi, a):
    """tilde-phi along physical axis a (Eq. fftp36); coefficient axis in place of a."""
    fwd, _, _ = fourier_matrices(grid.n[a], grid.hi[a] - grid.lo[a])
    return _along(fwd, psi.astype(np.complex128), grid.axis_of(a))


def sine_coeffs(grid, psi, a):
    """tilde-phi_l = (2/N) sum_j phi_j sin(j l pi/N) along axis a (Eq. tpll)."""
    C, _ = sine_matrix(grid.n[a], grid.hi[a] - grid.lo[a])
    return _along((2.0 / grid.n[a]) * C, psi, grid.axis_of(a))


def _rot_symbol(grid, a):
    """Rotation part of the line symbol (Eq. energy-discrete-FP):
    x-lines: +Omega*y_k*lam_p ; y-lines: -Omega*x_j*eta_q ; other axes: none.
    Returned as (coefficient, coordinate array broadcast to the data shape)."""
    if grid.omega == 0.0 or grid.dim < 2 or a > 1:
        return None
    if a == 0:
        return grid.omega, grid.mesh(1)
    return -grid.omega, grid.mesh(0)


def kinetic_axis(grid, psi, a):
    """Per-axis part of -1/2 Laplacian (and of -Omega L_z) applied to psi."""
    if grid.disc == "fourier":
        N, L = grid.n[a], grid.hi[a] - grid.lo[a]
        fwd, inv, lam = fourier_matrices(N, L)
        ax = grid.axis_of(a)
        c = _along(fwd, psi.astype(np.complex128), ax)
        shape = [1] * grid.dim
        shape[ax] = N
        lam_b = lam.reshape(shape)
        sym = 0.5 * lam_b ** 2
        rot = _rot_symbol(grid, a)
        if rot is not None:
            coef, coord = rot
            sym = sym + coef * coord * lam_b
        out = _along(inv, c * sym, ax)
        return out if grid.is_complex else out.real
    if grid.disc == "sine":
        N, L = grid.n[a], grid.hi[a] - grid.lo[a]
        C, lam = sine_matrix(N, L)
        ax = grid.axis_of(a)
        c = _along((2.0 / N) * C, psi, ax)
        shape = [1] * grid.dim
        shape[ax] = N - 1
        # -1/2 d_xx^s phi_j = 1/2 sum_l lam_l^2 tilde-phi_l sin(j l pi/N)   (Eq. spdo1)
        return _along(C, 0.5 * lam.reshape(shape) ** 2 * c, ax)
    if grid.disc == "fd":
        ax = grid.axis_of(a)
        h2 = grid.h[a] ** 2
        pad = [(0, 0)] * grid.dim
        pad[ax] = (1, 1)
        q = np.pad(psi, pad)
        n = psi.shape[ax]
        lo = np.take(q, np.arange(0, n), axis=ax)
        hi = np.take(q, np.arange(2, n + 2), axis=ax)
        # a_jj = 1/h^2, a_j,j+-1 = -1/(2h^2)   (§2.1 tridiagonal A without V)
        return psi / h2 - (lo + hi) / (2.0 * h2)
    raise ValueError(grid.disc)


def _fd_central(grid, psi, a):
    """Second-order central difference d/dx_a with zero Dirichlet values."""
    ax = grid.axis_of(a)
    pad = [(0, 0)] * grid.dim
    pad[ax] = (1, 1)
    q = np.pad(psi, pad)
    n = psi.shape[ax]
    return (np.take(q, np.arange(2, n + 2), axis=ax) - np.take(q, np.arange(0, n), axis=ax)) / (2.0 * grid.h[a])


def apply_kinetic(grid, psi):
    """-1/2 Delta_h psi - Omega L_z,h psi (rotation folded per axis for the
    spectral grids; central differences for FD, reading of §2.1's omitted
    2D/3D rotating case)."""
    out = sum(kinetic_axis(grid, psi, a) for a in range(grid.dim))
    if grid.disc == "fd" and grid.omega != 0.0 and grid.dim >= 2:
        x, y = grid.mesh(0), grid.mesh(1)
        # -Omega L_z = i Omega (x d_y - y d_x)
        out = out + 1j * grid.omega * (x * _fd_central(grid, psi, 1) - y * _fd_central(grid, psi, 0))
    return out


def apply_hlin(grid, psi):
    """H_lin psi = (-1/2 Delta_h + V - Omega L_z,h) psi (the matrix A of §2.1,
    B of Eq. energy-discrete-SP-34, or its Fourier analogue)."""
    return apply_kinetic(grid, psi) + grid.V * psi


def energy(grid, psi):
    """E_h(psi) = h_vol * sum [Re(conj(psi) H_lin psi) + beta/2 |psi|^4]."""
    hl = apply_hlin(grid, psi)
    a2 = np.abs(psi) ** 2
    return grid.h_vol * float(np.sum(np.real(np.conj(psi) * hl)) + 0.5 * grid.beta * np.sum(a2 * a2))


def chem_potential(grid, psi):
    """mu_h = E_h + h_vol * beta/2 * sum |psi|^4 (Eq. chemical-potential)."""
    a2 = np.abs(psi) ** 2
    return energy(grid, psi) + grid.h_vol * 0.5 * grid.beta * float(np.sum(a2 * a2))


def norm2(grid, psi):
    """||psi||_h^2 = h_vol sum |psi|^2."""
    return grid.h_vol * float(np.sum(np.abs(psi) ** 2))


def rms(grid, psi, a):
    """alpha_rms = sqrt(h_vol sum alpha^2 |psi|^2) (Eq. rms)."""
    return math.sqrt(grid.h_vol * float(np.sum(grid.mesh(a) ** 2 * np.abs(psi) ** 2)))


def energy_parseval(grid, psi):
    """E_h from the coefficient (Parseval) forms, written independently of
    apply_hlin: Eq. energy-discrete-FP for Fourier grids (kinetic + rotation
    per line, N_a * sum_p symbol |tilde-phi|^2) and Eq. BCD for sine grids
    (N/4 sum lam^2 tilde-phi^2 per line)."""
    a2 = np.abs(psi) ** 2
    pot_int = float(np.sum(grid.V * a2 + 0.5 * grid.beta * a2 * a2))
    kin = 0.0
    for a in range(grid.dim):
        N, L = grid.n[a], grid.hi[a] - grid.lo[a]
        ax = grid.axis_of(a)
        shape = [1] * grid.dim
        if grid.disc == "fourier":
            c = fourier_coeffs(grid, psi, a)
            _, _, lam = fourier_matrices(N, L)
            shape[ax] = N
            lam_b = lam.reshape(shape)
            sym = 0.5 * lam_b ** 2
            rot = _rot_symbol(grid, a)
            if rot is not None:
                coef, coord = rot
                sym = sym + coef * coord * lam_b
            kin += N * float(np.sum(sym * np.abs(c) ** 2))
        elif grid.disc == "sine":
            c = sine_coeffs(grid, psi, a)
            _, lam = sine_matrix(N, L)
            shape[ax] = N - 1
            kin += 0.5 * (N / 2.0) * float(np.sum(lam.reshape(shape) ** 2 * np.abs(c) ** 2))
        else:
            raise ValueError("Parseval form exists for the spectral grids only")
    return grid.h_vol * (kin + pot_int)
