"""FP64 CPU oracle for the regularized Newton ground-state method of
Wu, Wen & Bao, "A Regularized Newton Method for Computing Ground States of
Bose-Einstein Condensates" (arXiv:1504.02891).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import or run anything in this package.  It shares no
code with the CUDA library (``paper_1504_02891_gb300``) and never imports it.

Everything here is plain numpy in float64/complex128: transforms are the
paper's sums written as dense matrices (§2.2 Eq. tpll/spdo1, §2.3 Eq.
fftp35/fftp36), the optimisation follows Lemma 3.1, Theorem 3.3, Eq. bb-1,
Eq. NMLS-Armijo, Algorithm 1, the ratio test of Eq. TR-ratio/update-X/tau-up,
Algorithm 2 and Algorithm 3.

Parity status per function (what pins it) is listed in each module header.
"""
from .discretize import (Grid, build_grid, potential, apply_kinetic, apply_hlin,
                         energy, energy_parseval, chem_potential, norm2, rms)
from .unified import (Unified, cayley_step, cayley_dense, proj_grad)
from .solvers import (feasible_gradient, armijo_gradient, regularized_newton, prolong, inject,
                      cascadic, SolveResult, rn_model, rn_ratio_terms, quartic_diff)
from .certificate import tangent_hessian_min

__all__ = [
    "Grid", "build_grid", "potential", "apply_kinetic", "apply_hlin", "energy",
    "energy_parseval", "chem_potential", "norm2", "rms", "Unified", "cayley_step",
    "cayley_dense", "proj_grad", "feasible_gradient", "armijo_gradient", "regularized_newton",
    "prolong", "inject", "cascadic", "SolveResult", "tangent_hessian_min",
    "rn_model", "rn_ratio_terms", "quartic_diff",
]
