"""The paper's printed results for the lattice workloads, computed on the GPU
from the paper's initial data: Table 10 (2D harmonic + optical lattice,
beta = 500, SP on (-16,16)^2 with 257^2 nodes; the ground state from the
Thomas-Fermi data of Eq. TFA, the asymmetric excited states from their odd
data within their parity class) and Table 5 (3D lattice, beta = 100 and 6400,
129^3 nodes), checked against tests/golden/paper_values.txt; and the
second-order certificate (Lemma 3.2) on the printed beta = 100 state."""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1504_02891_gb300 as G  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def paper_values():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, q, v, tol, _cite = [s.strip() for s in line.split("|")]
        out.setdefault(name, {})[q] = (float(v), float(tol))
    return out


def quantities(p, psi, rep):
    """max|phi|^2, E, mu (from the solver's report) and the rms widths
    sqrt(h_vol sum x_a^2 |phi|^2) of the returned state."""
    h = W.cell_volume(p)
    a2 = np.abs(psi) ** 2
    q = {"maxphi2": float(a2.max()), "E": rep["E"], "mu": rep["mu"]}
    for a, name in enumerate(("xrms", "yrms", "zrms")[:p["dim"]]):
        x = W.axis_nodes(p, a)
        shape = [1] * p["dim"]
        shape[p["dim"] - 1 - a] = x.size
        q[name] = float(np.sqrt(h * np.sum(x.reshape(shape) ** 2 * a2)))
    return q


# The paper stops Algorithm 1 at Eq. crit1 with eps0 = 1e-6: its energies are
# converged to the printed digits (second order in the state's error), its
# chemical potentials and widths to a few units of the last digit (first
# order).  Our states are converged to ||H psi - mu psi|| <= 1e-9.
LOOSE = {"mu": 5e-4, "xrms": 2e-4, "yrms": 2e-4}


def check(name, q, keys=None):
    ref = paper_values()[name]
    for k, (v, tol) in ref.items():
        if keys and k not in keys:
            continue
        tol = max(tol, LOOSE.get(k, 0.0))
        assert abs(q[k] - v) <= tol, (name, k, q[k], v)


def solve(p, psi0, cert=False, **opts):
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, **opts)
        c = plan.hess_min_eig(t, max_iter=300, tol=1e-8) if cert else None
        return t.cpu().numpy(), rep, c


def test_table10_ground_state_from_thomas_fermi():
    p = W.config("t10")
    psi, rep, _ = solve(p, W.thomas_fermi(p), mode=1, levels=1, res_tol=1e-9)
    assert rep["status"] == 0
    check("t10_g", quantities(p, psi, rep))


def _odd_part(psi, axes):
    """The part of psi odd under x -> -x (array axis 1) and/or y -> -y (axis
    0); the sine grid's interior nodes are symmetric about 0, so reversing an
    axis is the reflection."""
    for ax in axes:
        psi = 0.5 * (psi - np.flip(psi, axis=ax))
    return psi


@pytest.mark.parametrize("kind,axes", [("10", (1,)), ("01", (0,)), ("11", (0, 1))])
def test_table10_excited_states_within_their_symmetry_class(kind, axes):
    """Table 10's asymmetric excited states phi_10, phi_01, phi_11 from the
    paper's odd initial data (§4.4).  They are saddles of the energy on the
    whole sphere: rounding seeds the even component, and an unrestricted
    Algorithm 1 run passes through the printed state and leaves it for a
    state below 32.21 within ~800 iterations.  Restricted to their parity
    class they are minimisers: Algorithm 1 runs of at most 100 iterations,
    the test re-imposing the parity of the initial data between runs (it
    removes only the rounding-seeded component, which grows by about e^8 in
    100 iterations near these saddles), reach ||H psi - mu psi|| <= 1e-9,
    and the state matches the printed row."""
    p = W.config("t10")
    psi = W.excited_initial(p, kind)
    for _ in range(40):
        psi = W.normalise(p, _odd_part(psi, axes))
        psi, rep, _ = solve(p, psi, method=1, mode=0, levels=1, eps0=0.0, res_tol=1e-9, max_iter=100)
        if rep["status"] == 0:
            break
    assert rep["status"] == 0 and rep["res"] <= 1e-9, rep
    # the returned state is still odd to rounding (one run of <= 100 steps)
    assert np.abs(psi - _odd_part(psi, axes)).max() <= 1e-6 * np.abs(psi).max()
    check("t10_" + kind, quantities(p, psi, rep))
    # the unrestricted iteration leaves it: the state of a 1600-step run from
    # the same data lies well below the printed energy
    _, rep2, _ = solve(p, W.excited_initial(p, kind), method=1, mode=0, levels=1, eps0=0.0, res_tol=0.0,
                       max_iter=1600)
    assert rep2["E"] < paper_values()["t10_" + kind]["E"][0] - 1.0, rep2["E"]


def test_table5_beta100_printed_state_is_a_saddle():
    """Table 5, beta = 100: Algorithm 1 from the Thomas-Fermi data reproduces
    the printed row (on the 65^3-node grid, where it is resolved to the printed
    digits), but the second-order certificate of Lemma 3.2 is negative there:
    a saddle.  From a Gaussian the GPU reaches a state of lower energy with a
    positive certificate, on that grid and on the paper's 129^3 nodes: the
    ground state has E = 23.2352 (printed 23.2356), mu = 27.437 and
    x_rms = 1.8823."""
    p = W.config("t5_100")
    p["n"] = (64, 64, 64)
    psi, rep, (c, res, _) = solve(p, W.thomas_fermi(p), cert=True, mode=0, levels=1, res_tol=1e-9)
    assert rep["status"] == 0
    check("t5_100", quantities(p, psi, rep))
    assert c < -0.1 and res <= 1e-6, (c, res)
    E_printed = paper_values()["t5_100"]["E"][0]
    for n in (64, 128):
        p["n"] = (n, n, n)
        psi, rep, (c, res, _) = solve(p, W.gaussian(p), cert=True, mode=0, levels=1, res_tol=1e-9)
        assert rep["status"] == 0
        assert rep["E"] < E_printed - 3e-4, (n, rep["E"])
        assert c > 0.1 and res <= 1e-6, (n, c, res)


def test_table5_beta6400():
    """Table 5, beta = 6400 on (-12,12)^3 with 129^3 nodes: Algorithm 1 on the
    finest grid from the Thomas-Fermi data (as in §4.2)."""
    p = W.config("t5_6400")
    psi, rep, _ = solve(p, W.thomas_fermi(p), mode=0, levels=1, res_tol=1e-9)
    assert rep["status"] == 0
    check("t5_6400", quantities(p, psi, rep))
