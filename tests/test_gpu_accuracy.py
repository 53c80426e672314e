"""Accuracy of the discretisations against the paper's printed errors, computed
on the GPU (arXiv:1504.02891 §4.1 Tables 1-2, §4.2 Tables 3-4): the ground
state on coarse meshes by FD and SP, against a fine-mesh SP solution, and the
fine-mesh energy, chemical potential and rms widths of the 3D Cases I and II
printed after Table 4."""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1504_02891_gb300 as G  # noqa: E402

HERE = os.path.join(os.path.dirname(__file__), "golden")


def _rows(table):
    rows = []
    for line in open(os.path.join(HERE, "accuracy_tables.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        t, case, disc, h, em, ee, emu = [x.strip() for x in line.split("|")]
        if t == table:
            rows.append((case, disc, float(h), float(em), float(ee), float(emu)))
    return rows


def _printed(name):
    out = {}
    for line in open(os.path.join(HERE, "paper_values.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        n, q, v, tol, _ = [x.strip() for x in line.split("|")]
        if n == name:
            out[q] = (float(v), float(tol))
    return out


# Energies carry all printed digits; chemical potentials and widths a few units
# of the last one (the paper stops Algorithm 1 at Eq. crit1, eps0 = 1e-6).
LOOSE = {"mu": 5e-4, "xrms": 3e-4, "yrms": 3e-4, "zrms": 3e-4}

# §4.2 Table 4, SP at h = 2: the discrete problem has a local minimiser with a
# lower energy than the printed row's state; checked as that inequality.
LOWER_THAN_PRINTED = {("T4", "sine", 2.0)}


def _agrees(ours, printed):
    """Within 10% above the rounding floor; both tiny below it (printed < 1e-9)."""
    if printed < 1e-9:
        return ours < 1e-8
    return abs(ours / printed - 1.0) <= 0.10


def _ground(case, disc, n, cert=False):
    p, psi0 = W.accuracy_case(case, disc, n)
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        rep = plan.solve(t, mode=1, levels=1, res_tol=1e-11, delta_stop=1e-14)
        c = plan.hess_min_eig(t, max_iter=300, tol=1e-8)[0] if cert else None
        psi = t.cpu().numpy().real
    assert rep["status"] == 0, (case, disc, n, rep)
    return p, psi * np.sign(psi.flat[np.argmax(np.abs(psi))]), rep["E"], rep["mu"], c


def _check_table(table, n_fine):
    rows = _rows(table)
    case = rows[0][0]
    dim = 1 if case.startswith("1d") else 3
    _, pex, Eex, muex, _ = _ground(case, "sine", n_fine)
    L = 32.0 if dim == 1 else 16.0
    for _, disc, h, em, ee, emu in rows:
        n = int(round(L / h))
        special = (table, disc, h) in LOWER_THAN_PRINTED
        _, psi, E, mu, c = _ground(case, disc, n, cert=special)
        if special:
            assert E < Eex - ee and c > 0.0, (E, Eex, c)
            continue
        r = n_fine // n
        sub = pex[(slice(r - 1, None, r),) * dim]
        err = float(np.max(np.abs(sub - psi)))
        for ours, printed, what in ((err, em, "max"), (abs(E - Eex), ee, "E"), (abs(mu - muex), emu, "mu")):
            assert _agrees(ours, printed), (table, disc, h, what, ours, printed)
    return pex, Eex, muex


@pytest.mark.parametrize("table", ["T1", "T2"])
def test_accuracy_1d(table):
    _check_table(table, 512)


@pytest.mark.parametrize("table,name", [("T3", "3d_I"), ("T4", "3d_II")])
def test_accuracy_3d_and_printed_values(table, name):
    pex, E, mu = _check_table(table, 128)
    p, _ = W.accuracy_case(name, "sine", 128)
    h = W.cell_volume(p)
    a2 = pex ** 2
    q = {"E": E, "mu": mu}
    for a, key in enumerate(("xrms", "yrms", "zrms")):
        x = W.axis_nodes(p, a)
        shape = [1, 1, 1]
        shape[2 - a] = x.size
        q[key] = float(np.sqrt(h * np.sum(x.reshape(shape) ** 2 * a2)))
    for k, (v, tol) in _printed(name).items():
        assert abs(q[k] - v) <= max(tol, LOOSE.get(k, 0.0)), (name, k, q[k], v)
