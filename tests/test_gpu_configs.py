"""The benchmark configurations at full size on the GPU, certified by the
FP64 oracle: config 3 (3D sine 128^3, depth-100 lattice, beta = 1600) solved
in the mixed schedule and in float64 to ||H psi - mu psi||_h <= 1e-9, with
the oracle's energy, chemical potential and residual of the returned state;
the Table 5 validation row of config 3's code path (depth 50, beta = 800,
§4.2); and the float64 operator at config 3's full size."""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1504_02891_gb300 as G  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def paper_values(name):
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        n, q, v, tol, _cite = [s.strip() for s in line.split("|")]
        if n == name:
            out[q] = (float(v), float(tol))
    return out


def oracle_state_check(g, psi):
    """The oracle's E, mu and ||H psi - mu psi||_h of a grid function."""
    hp = O.apply_hlin(g, psi) + g.beta * np.abs(psi) ** 2 * psi
    mu = O.chem_potential(g, psi)
    return O.energy(g, psi), mu, math.sqrt(O.norm2(g, hp - mu * psi))


def test_c3_full_size_mixed_and_fp64_certified():
    p = W.config("c3")
    g = O.build_grid(p)
    psi0 = W.gaussian(p)
    out = {}
    for mode in (1, 0):
        with G.Plan(p) as plan:
            t = G.to_device(psi0)
            rep = plan.solve(t, mode=mode, levels=3, res_tol=1e-9, delta_stop=0.0, max_outer=60)
            psi = t.cpu().numpy()
        E, mu, r = oracle_state_check(g, psi)
        assert abs(E - rep["E"]) <= 1e-9 * abs(E), (mode, E, rep["E"])
        assert abs(mu - rep["mu"]) <= 1e-9 * abs(mu), (mode, mu, rep["mu"])
        assert r <= 1.5e-9, (mode, r, rep["res"])
        assert abs(r - rep["res"]) <= 0.05 * r + 1e-11, (mode, r, rep["res"])
        out[mode] = (E, psi)
    # both schedules reach the same ground state
    (Em, pm), (Ed, pd) = out[1], out[0]
    assert abs(Em - Ed) <= 1e-9 * abs(Ed), (Em, Ed)
    pm = pm * np.sign(np.vdot(pm, pd).real)
    assert np.max(np.abs(pm - pd)) <= 1e-5 * np.max(np.abs(pd))


def test_c3p_table5_beta800():
    """Table 5 (§4.2): lattice depth 50, beta = 800 on (-8,8)^3 with 129^3
    nodes -- E 33.8023, mu 40.4476, x_rms 2.6620 -- from a Gaussian by the
    cascade in the mixed schedule."""
    p = W.config("c3p")
    with G.Plan(p) as plan:
        t = G.to_device(W.gaussian(p))
        rep = plan.solve(t, mode=1, levels=3, res_tol=1e-9)
        psi = t.cpu().numpy()
    assert rep["status"] == 0
    ref = paper_values("c3p")
    h = W.cell_volume(p)
    x = W.axis_nodes(p, 0)
    xrms = math.sqrt(h * float(np.sum(x[None, None, :] ** 2 * np.abs(psi) ** 2)))
    got = {"E": rep["E"], "mu": rep["mu"], "xrms": xrms}
    # the paper stops Algorithm 1 at Eq. crit1 (eps0 = 1e-6): E is converged to
    # its printed digits, mu and the width to a few units of the last digit
    loose = {"mu": 5e-4, "xrms": 2e-4}
    for k, (v, tol) in ref.items():
        assert abs(got[k] - v) <= max(tol, loose.get(k, 0.0)), (k, got[k], v)


def test_c3_full_size_operator_parity_fp64():
    p = W.config("c3")
    g = O.build_grid(p)
    psi = W.random_field(p, seed=21, smooth=0.02)
    d = W.random_field(p, seed=22)
    with G.Plan(p, prec=G.F64) as plan:
        out, (E, mu) = plan.grad(G.to_device(psi, G.F64), with_energy=True)
        hv = plan.hessvec(G.to_device(psi, G.F64), G.to_device(d, G.F64), 0.3)
        o, h = out.cpu().numpy(), hv.cpu().numpy()
    ref = O.apply_hlin(g, psi) + g.beta * np.abs(psi) ** 2 * psi
    assert np.max(np.abs(o - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert abs(E - O.energy(g, psi)) <= 1e-12 * abs(E)
    refh = O.apply_hlin(g, d) + g.beta * (np.abs(psi) ** 2 * d + 2.0 * psi * psi * d) + 0.3 * d
    assert np.max(np.abs(h - refh)) <= 1e-12 * np.max(np.abs(refh))
