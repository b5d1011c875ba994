"""The reading behind the library's LM linear tolerance: LM needs no exact
damped step.  The LM schedule of the oracle is driven here from Python with
its exact sparse-Cholesky step perturbed by a relative error eta (what a
linear solve to a relative residual of about eta leaves), and reaches the
same final cost as the exact LM, with the same iteration count.  CPU only."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2603_17201_gb300 import synthetic as syn  # noqa: E402


def lm_with_step_error(og, poses, eta, rng, max_iters=20, tau=1e-5, ftol=1e-14):
    """The oracle's LM rules (lambda_0 = tau max diag H, gain ratio
    (F - F') / (d^T (lambda d - b)), Nielsen's lambda update, stop once
    |F - F'| <= ftol F) with every step d replaced by d (1 + eta n), n a
    standard normal per entry."""
    p = poses.copy()
    F, Hd, Ho, b = og.linearize(p)
    lam = tau * max(np.diag(Hd[v]).max() for v in range(len(Hd)))
    nu = 2.0
    its = 0
    for _ in range(max_iters):
        its += 1
        d = og.solve_system(Hd, Ho, b, lam)
        d = d * (1.0 + eta * rng.standard_normal(d.shape))
        pn = og.apply_update(p, d)
        Fn = og.cost(pn)
        pred = float(np.sum(d * (lam * d - b)))
        rho = (F - Fn) / pred if pred > 0 else -1.0
        flat = abs(F - Fn) <= ftol * F
        if rho > 0:
            lam *= max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)
            nu = 2.0
            p = pn
            F, Hd, Ho, b = og.linearize(p)
        else:
            lam *= nu
            nu *= 2.0
        if flat:
            break
    return F, its


@pytest.mark.parametrize("name,eta", [("c1_circle200", 0.0), ("c1_circle200", 1e-6), ("c1_circle200", 1e-4),
                                      ("c1_circle200", 1e-3), ("c2_figure8_2k", 1e-4)])
def test_inexact_steps_reach_the_exact_optimum(name, eta):
    g = syn.make_config(name)
    og = O.OracleGraph.from_synthetic(g)
    _, ref = og.lm(g.poses_init, max_iters=20)
    F, its = lm_with_step_error(og, g.poses_init, eta, np.random.default_rng(3))
    assert abs(F - ref["final_cost"]) <= 1e-12 * ref["final_cost"], (eta, F, ref)
    assert abs(its - ref["iterations"]) <= 1, (eta, its, ref["iterations"])
