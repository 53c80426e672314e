"""gpe_plan_autotune: measured launch shapes for the line kernels and the
cluster engine change how the work is spread, not what is computed; the
measured choice between the fused operator kernel and the two line kernels
changes the FFT factorisation, so the operator values agree to float32
rounding (identical bytes when the implementation stays the same)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1504_02891_gb300 as G  # noqa: E402


def test_autotune_keeps_operator_values_and_records_choices():
    p = W.config("c2")
    with G.Plan(p, nbatch=4, prec=G.F32) as plan:
        psi = plan.empty()
        psi.normal_()
        out0, out1 = plan.empty(), plan.empty()
        plan.grad(psi, out0)
        plan.autotune(levels=3)
        plan.grad(psi, out1)
        torch.cuda.synchronize()
        rep = G.autotune_report()
        assert float((out0 - out1).abs().max()) <= 2e-5 * float(out0.abs().max())
    assert "lines f32 256x256 nbatch 4" in rep, rep
    assert "operator f32 256x256 nbatch 4:" in rep, rep
    for n in (256, 128, 64):
        assert f"cluster {n}x{n}: share" in rep, rep


def test_solve_after_autotune_reaches_the_same_ground_state():
    p = W.config("c2")
    init = G.to_device(W.gaussian(p))
    with G.Plan(p) as plan:
        t = init.clone()
        ref = plan.solve(t, mode=1, levels=3, res_tol=1e-9)
        plan.autotune(levels=3)
        t = init.clone()
        rep = plan.solve(t, mode=1, levels=3, res_tol=1e-9)
    assert rep["status"] == 0 and ref["status"] == 0
    assert abs(rep["E"] - ref["E"]) <= 1e-9 * ref["E"], (rep["E"], ref["E"])
