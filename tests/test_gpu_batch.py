"""Batched solves (gpe_solve_batch): many independent ground-state problems
(the batched sweep's mix of grids, beta, Omega and traps) in one call.

Checks: every instance's result is bit-identical to solving that instance
alone (the batch only schedules; the arithmetic per instance is the same);
the FP64 oracle certifies each returned state (its energy, chemical potential
and residual of that very state agree with the report); a non-rotating
instance reaches the float64 solver's ground-state energy to float32
accuracy."""
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


def host(t):
    a = t.detach().cpu().numpy()
    return a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)


def small_mix():
    """Eight sweep instances on 64^2 and 128^2 (plus two of them real, Omega = 0)."""
    sweep = W.batched_sweep(64)
    picks = [p for p in sweep if p["n"][0] <= 128][:6]
    real = []
    for p in picks[:2]:
        q = dict(p)
        q["omega"] = 0.0
        q["is_complex"] = False
        real.append(q)
    return picks + real


def initial(ps):
    out = []
    for i, p in enumerate(ps):
        a = W.sweep_initial(p, i)
        if not p["is_complex"]:
            a = W.normalise(p, np.abs(a))
        out.append(torch.from_numpy(a.astype(np.complex64 if p["is_complex"] else np.float32)).cuda())
    return out


OPTS = dict(max_iter=400, res_tol=1e-7)


def test_batch_equals_one_at_a_time():
    ps = small_mix()
    batch = initial(ps)
    reps = G.solve_batch(ps, batch, **OPTS)
    for i, p in enumerate(ps):
        one = initial([p])
        one[0].copy_(initial(ps)[i])
        r1 = G.solve_batch([p], one, **OPTS)[0]
        assert torch.equal(one[0], batch[i]), i
        for k in ("E", "mu", "res", "inner_f32", "nfe", "status"):
            assert r1[k] == reps[i][k], (i, k)


def test_batch_states_certified_by_oracle():
    ps = small_mix()
    psis = initial(ps)
    reps = G.solve_batch(ps, psis, **OPTS)
    for i, p in enumerate(ps):
        g = O.build_grid(p)
        psi = host(psis[i])
        assert abs(O.norm2(g, psi) - 1.0) <= 1e-5
        hp = O.apply_hlin(g, psi) + p["beta"] * np.abs(psi) ** 2 * psi
        mu = O.chem_potential(g, psi)
        E = O.energy(g, psi)
        r = math.sqrt(O.norm2(g, hp - mu * psi))
        assert abs(E - reps[i]["E"]) <= 2e-6 * abs(E), (i, E, reps[i]["E"])
        assert abs(mu - reps[i]["mu"]) <= 2e-5 * abs(mu), (i, mu, reps[i]["mu"])
        assert abs(r - reps[i]["res"]) <= 0.05 * r + 1e-4, (i, r, reps[i]["res"])
        assert reps[i]["status"] in (0, 5)
        assert reps[i]["inner_f32"] >= 1


def test_batch_nonrotating_energy_matches_fp64_solver():
    p = W.problem(2, (128, 128), (-12.0, -12.0), (12.0, 12.0), "fourier", beta=600.0,
                  potential={"kind": "harmonic", "gamma": (1.0, 1.1)})
    psi0 = W.gaussian(p)
    t32 = torch.from_numpy(psi0.astype(np.float32)).cuda()
    r32 = G.solve_batch([p], [t32], max_iter=2000, res_tol=1e-9)[0]
    with G.Plan(p) as plan:
        t = G.to_device(psi0)
        r64 = plan.solve(t, mode=0, levels=1, res_tol=1e-10)
    assert r64["status"] == 0
    assert abs(r32["E"] - r64["E"]) <= 2e-6 * r64["E"], (r32["E"], r64["E"])
    assert abs(r32["mu"] - r64["mu"]) <= 1e-4 * r64["mu"], (r32["mu"], r64["mu"])
