"""Seeded synthetic inputs for the Gross-Pitaevskii ground-state workloads.

This module is shared by the tests, ``bench.py`` and ``__graft_entry__``.  It
holds problem *parameters* (grids, traps, beta, Omega) and *initial data*
sampled on the grid.  It contains none of the method's arithmetic: no
transform, no operator, no energy, no optimisation step.  Both the FP64 CPU
oracle and the CUDA library read the parameter dictionaries below and each
builds its own grid, potential and operator from them.

Grid convention (paper §2):
  * Fourier pseudospectral ("fourier"): N points per axis, x_j = a + j h,
    j = 0..N-1, h = (b-a)/N (periodic).
  * Sine pseudospectral ("sine") and finite difference ("fd"): N intervals,
    N-1 interior unknowns x_j = a + j h, j = 1..N-1 (homogeneous Dirichlet).
Arrays are C-ordered with x fastest: shape (n_x,), (n_y, n_x) or
(n_z, n_y, n_x).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "problem", "axis_nodes", "array_shape", "cell_volume", "normalise",
    "gaussian", "rotating_initial", "config", "CONFIGS", "batched_sweep", "sweep_initial", "random_field",
    "thomas_fermi", "excited_initial", "accuracy_case",
]


def problem(dim, n, lo, hi, disc="fourier", beta=0.0, omega=0.0,
            potential=None, is_complex=None):
    """Parameter dictionary for one ground-state problem.

    ``n`` is the paper's N per axis (points for Fourier, intervals for sine
    and FD).  ``potential`` is one of
      {"kind": "harmonic", "gamma": (gx, gy, gz)}                 (Eq. harmpen)
      {"kind": "lattice", "gamma": (...), "depth": A, "k": k}     V = harmonic + A*sum sin^2(k x)
      {"kind": "stirrer", "gamma": (...), "w0":, "delta":, "r0":}  (§4.2 Case II)
    """
    n = tuple(int(v) for v in n)
    lo = tuple(float(v) for v in lo)
    hi = tuple(float(v) for v in hi)
    assert len(n) == dim and len(lo) == dim and len(hi) == dim
    if potential is None:
        potential = {"kind": "harmonic", "gamma": (1.0,) * dim}
    pot = dict(potential)
    g = tuple(float(v) for v in pot.get("gamma", (1.0,) * dim))
    pot["gamma"] = g + (1.0,) * (3 - len(g))
    if is_complex is None:
        is_complex = omega != 0.0
    return {"dim": dim, "n": n, "lo": lo, "hi": hi, "disc": disc,
            "beta": float(beta), "omega": float(omega), "potential": pot,
            "is_complex": bool(is_complex)}


def axis_nodes(p, axis):
    """Coordinates of the unknowns along one axis (x = axis 0)."""
    n, a, b = p["n"][axis], p["lo"][axis], p["hi"][axis]
    h = (b - a) / n
    if p["disc"] == "fourier":
        j = np.arange(n, dtype=np.float64)
    else:
        j = np.arange(1, n, dtype=np.float64)
    return a + j * h


def array_shape(p):
    """Numpy shape of a grid function, x fastest (last)."""
    ext = [len(axis_nodes(p, a)) for a in range(p["dim"])]
    return tuple(reversed(ext))


def cell_volume(p):
    return float(np.prod([(p["hi"][a] - p["lo"][a]) / p["n"][a] for a in range(p["dim"])]))


def _mesh(p):
    """Coordinate arrays broadcast to the array shape, ordered (x, y, z)."""
    d = p["dim"]
    axes = [axis_nodes(p, a) for a in range(d)]
    out = []
    for a in range(d):
        shape = [1] * d
        shape[d - 1 - a] = len(axes[a])
        out.append(axes[a].reshape(shape))
    return out


def normalise(p, psi):
    """Scale so that h_vol * sum |psi|^2 = 1 (discrete constraint)."""
    nrm = math.sqrt(cell_volume(p) * float(np.sum(np.abs(psi) ** 2)))
    return psi / nrm


def gaussian(p, dtype=np.float64):
    """Normalised Gaussian prod_i exp(-gamma_i x_i^2 / 2) sampled on the grid."""
    xs = _mesh(p)
    g = p["potential"]["gamma"]
    psi = np.ones(array_shape(p), dtype=np.float64)
    for a, x in enumerate(xs):
        psi = psi * np.exp(-0.5 * g[a] * x * x)
    psi = normalise(p, psi)
    if p["is_complex"]:
        psi = psi.astype(np.complex128)
    return psi.astype(dtype) if dtype is not None else psi


def rotating_initial(p, kind="c", noise=0.0, seed=1504):
    """Initial data (a), (b), (b-bar), (c), (c-bar), (d), (d-bar) of §4.3.

    phi_a = exp(-(x^2+y^2)/2)/sqrt(pi), phi_b = (x+iy) phi_a; (c) is the
    normalised mean of (a) and (b); (d) mixes them with weights (1-Omega) and
    Omega.  A bar conjugates.  In 3D phi_a also carries exp(-gamma_z z^2/2).  ``noise`` > 0 multiplies by exp(i*noise*xi),
    xi iid standard normal from numpy default_rng(seed) in C order, then
    renormalises.
    """
    xs = _mesh(p)
    x, y = xs[:2]
    pa = np.exp(-(x * x + y * y) / 2.0) / math.sqrt(math.pi) + 0j
    if p["dim"] == 3:     # 3D: the trap's Gaussian along z
        gz = p["potential"]["gamma"][2]
        pa = pa * np.exp(-0.5 * gz * xs[2] * xs[2])
    pa = np.broadcast_to(pa, array_shape(p)).astype(np.complex128)
    pb = (x + 1j * y) * pa
    base = kind.split("_")[0]
    conj = kind.endswith("_bar")
    if base == "a":
        psi = pa
    elif base == "b":
        psi = pb
    elif base == "c":
        psi = (pa + pb) / 2.0
    elif base == "d":
        om = p["omega"]
        psi = (1.0 - om) * pa + om * pb
    else:
        raise ValueError(kind)
    if conj:
        psi = np.conj(psi)
    if noise > 0.0:
        xi = np.random.default_rng(seed).standard_normal(array_shape(p))
        psi = psi * np.exp(1j * noise * xi)
    return normalise(p, psi)


def _trap(p):
    """The trap of the problem on the grid (its definition: Eq. harmpen, plus
    the lattice term of Eq. optic98 / Eq. asypon), as initial-data input."""
    xs = _mesh(p)
    pot = p["potential"]
    g = pot["gamma"]
    V = np.zeros(array_shape(p))
    for a, x in enumerate(xs):
        V = V + 0.5 * g[a] ** 2 * x * x
        if pot["kind"] == "lattice":
            V = V + pot["depth"] * np.sin(pot["k"] * x) ** 2
    if pot["kind"] not in ("harmonic", "lattice"):
        raise ValueError("Thomas-Fermi data for harmonic or lattice traps only")
    return V


def thomas_fermi(p):
    """The Thomas-Fermi initial data of Eq. TFA, normalised on the grid:
    phi_0 = sqrt((mu_TF - V)/beta) where V <= mu_TF, else 0, with mu_TF =
    (3 beta / 2)^(2/3) / 2, (beta gamma_y / pi)^(1/2) and
    (15 beta gamma_y gamma_z / (4 pi))^(2/5) / 2 for d = 1, 2, 3 (gamma_x = 1)."""
    d, beta = p["dim"], p["beta"]
    gy, gz = p["potential"]["gamma"][1], p["potential"]["gamma"][2]
    if d == 1:
        mu = 0.5 * (1.5 * beta) ** (2.0 / 3.0)
    elif d == 2:
        mu = math.sqrt(beta * gy / math.pi)
    else:
        mu = 0.5 * (15.0 * beta * gy * gz / (4.0 * math.pi)) ** 0.4
    phi = np.sqrt(np.maximum(mu - _trap(p), 0.0) / beta)
    if p["is_complex"]:
        phi = phi.astype(np.complex128)
    return normalise(p, phi)


def excited_initial(p, kind):
    """Asymmetric initial data of §4.4 (2D): "10" sqrt(2) x e^{-r^2/2}/sqrt(pi),
    "01" the same in y, "11" 2 x y e^{-r^2/2}/sqrt(pi); normalised on the grid."""
    x, y = _mesh(p)[:2]
    e = np.exp(-(x * x + y * y) / 2.0) / math.sqrt(math.pi)
    f = {"10": math.sqrt(2.0) * x * e, "01": math.sqrt(2.0) * y * e, "11": 2.0 * x * y * e}[kind]
    f = np.broadcast_to(f, array_shape(p)).astype(np.float64)
    return normalise(p, f)


_LATTICE_K = math.pi / 4.0


def accuracy_case(case, disc, n):
    """Problems of the accuracy study (§4.1 Tables 1-2, §4.2 Tables 3-4) with
    n intervals per axis and discretisation disc ("fd" or "sine"), and the
    initial data used: 1d_I harmonic beta=400 on (-16,16) (Thomas-Fermi data);
    1d_II x^2/2 + 25 sin^2(pi x/4), beta=250 (Gaussian); 3d_I gamma (1,2,4),
    beta=200 on (-8,8)x(-6,6)x(-4,4) (Thomas-Fermi); 3d_II harmonic (1,1,2) +
    stirrer 4 exp(-((x-1)^2+y^2)), beta=200 on (-8,8)^3 (Gaussian)."""
    if case == "1d_I":
        p = problem(1, (n,), (-16.0,), (16.0,), disc, beta=400.0)
        return p, thomas_fermi(p)
    if case == "1d_II":
        p = problem(1, (n,), (-16.0,), (16.0,), disc, beta=250.0,
                    potential={"kind": "lattice", "gamma": (1.0,), "depth": 25.0, "k": math.pi / 4.0})
        return p, gaussian(p)
    if case == "3d_I":
        p = problem(3, (n,) * 3, (-8.0, -6.0, -4.0), (8.0, 6.0, 4.0), disc, beta=200.0,
                    potential={"kind": "harmonic", "gamma": (1.0, 2.0, 4.0)})
        return p, thomas_fermi(p)
    if case == "3d_II":
        p = problem(3, (n,) * 3, (-8.0,) * 3, (8.0,) * 3, disc, beta=200.0,
                    potential={"kind": "stirrer", "gamma": (1.0, 1.0, 2.0), "w0": 4.0, "delta": 1.0, "r0": 1.0})
        return p, gaussian(p)
    raise KeyError(case)


def config(name):
    """The named workloads (parameters only)."""
    if name == "c1":      # 1D, Fourier 512, harmonic, beta=400
        return problem(1, (512,), (-16.0,), (16.0,), "fourier", beta=400.0)
    if name == "c2":      # 2D, Fourier 256^2, harmonic, beta=1000, cascade 64->128->256
        return problem(2, (256, 256), (-16.0, -16.0), (16.0, 16.0), "fourier", beta=1000.0)
    if name == "c3":      # 3D sine 128^3, harmonic + depth-100 lattice, beta=1600
        return problem(3, (128,) * 3, (-8.0,) * 3, (8.0,) * 3, "sine", beta=1600.0,
                       potential={"kind": "lattice", "gamma": (1.0, 1.0, 1.0),
                                  "depth": 100.0, "k": _LATTICE_K})
    if name == "c3p":     # Table 5 validation: depth 50, beta=800
        return problem(3, (128,) * 3, (-8.0,) * 3, (8.0,) * 3, "sine", beta=800.0,
                       potential={"kind": "lattice", "gamma": (1.0, 1.0, 1.0),
                                  "depth": 50.0, "k": _LATTICE_K})
    if name == "c4":      # 2D rotating, Fourier 512^2, Omega=0.9, beta=1000
        return problem(2, (512, 512), (-16.0, -16.0), (16.0, 16.0), "fourier",
                       beta=1000.0, omega=0.9, is_complex=True)
    if name == "r3":      # 3D rotating, Fourier 64^3 on (-8,8)^3, gamma (1,1,2), beta=200, Omega=0.7
        return problem(3, (64,) * 3, (-8.0,) * 3, (8.0,) * 3, "fourier", beta=200.0, omega=0.7,
                       is_complex=True, potential={"kind": "harmonic", "gamma": (1.0, 1.0, 2.0)})
    if name == "t10":     # §4.4, Table 10: 2D sine (-16,16)^2, 257 nodes, harmonic + 50 lattice, beta=500
        return problem(2, (256, 256), (-16.0, -16.0), (16.0, 16.0), "sine", beta=500.0,
                       potential={"kind": "lattice", "gamma": (1.0, 1.0), "depth": 50.0, "k": _LATTICE_K})
    if name == "t5_100":  # §4.2, Table 5: 3D sine (-8,8)^3, 129^3 nodes, lattice 50, beta=100
        return problem(3, (128,) * 3, (-8.0,) * 3, (8.0,) * 3, "sine", beta=100.0,
                       potential={"kind": "lattice", "gamma": (1.0, 1.0, 1.0), "depth": 50.0, "k": _LATTICE_K})
    if name == "t5_6400":  # §4.2, Table 5: 3D sine (-12,12)^3, 129^3 nodes, lattice 50, beta=6400
        return problem(3, (128,) * 3, (-12.0,) * 3, (12.0,) * 3, "sine", beta=6400.0,
                       potential={"kind": "lattice", "gamma": (1.0, 1.0, 1.0), "depth": 50.0, "k": _LATTICE_K})
    if name == "1d_case2":  # §4.1 Case II (sine): V = x^2/2 + 25 sin^2(pi x/4), beta=250
        return problem(1, (256,), (-16.0,), (16.0,), "sine", beta=250.0,
                       potential={"kind": "lattice", "gamma": (1.0,), "depth": 25.0,
                                  "k": _LATTICE_K})
    raise KeyError(name)


CONFIGS = ("c1", "c2", "c3", "c3p", "c4", "r3", "1d_case2", "t10", "t5_100", "t5_6400")


def batched_sweep(count=256, seed=20150410):
    """The batched-sweep instance list: grids from {64,128,256}^2 on [-12,12]^2,
    beta ~ U[100,1000], Omega ~ U[0,0.9], gamma_y ~ U[1,1.2], gamma_x = 1."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([64, 128, 256]))
        beta = float(rng.uniform(100.0, 1000.0))
        om = float(rng.uniform(0.0, 0.9))
        gy = float(rng.uniform(1.0, 1.2))
        out.append(problem(2, (n, n), (-12.0, -12.0), (12.0, 12.0), "fourier",
                           beta=beta, omega=om, is_complex=True,
                           potential={"kind": "harmonic", "gamma": (1.0, gy)}))
    return out


def sweep_initial(p, i):
    """Initial data of batched-sweep instance i: phi_c with seeded phase noise
    of amplitude 1e-2 (as config 4), noise seed 1504 + i."""
    return rotating_initial(p, "c", noise=1e-2, seed=1504 + i)


def random_field(p, seed=0, smooth=0.0):
    """Seeded random grid function of unit discrete norm (complex if the
    problem is complex).  smooth > 0 multiplies by a Gaussian envelope
    exp(-smooth |x|^2) so that the values decay towards the box edges."""
    rng = np.random.default_rng(seed)
    shape = array_shape(p)
    psi = rng.standard_normal(shape)
    if p["is_complex"]:
        psi = psi + 1j * rng.standard_normal(shape)
    if smooth > 0.0:
        env = np.ones(shape)
        for x in _mesh(p):
            env = env * np.exp(-smooth * x * x)
        psi = psi * env
    return normalise(p, psi)
