"""Pins of the oracle's Lagrangian multipliers (Sec. 2.3.1-2.3.4).

The decisive pin is the Lagrangian theorem itself: at the multipliers, the
partial derivative of the Lagrangian with respect to the integrals equals the
total derivative of the state energy (gradient) or of the bra-frozen overlap
(coupling), which the test takes by central finite differences of fully
re-converged SCCSD solutions (ground state, both EOM states and zeta solved
again at the perturbed integrals). A dropped term, a wrong sign or a wrong
closed form in the multiplier equations breaks that equality.
"""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle import multipliers as mu
from paper_2403_01007_gb300 import synthetic as syn

TARGETS = [("gradient", 0), ("gradient", 1), ("coupling", 0, 1), ("coupling", 1, 0)]


@pytest.fixture(scope="module")
def system():
    o, v, J = 2, 4, 10
    eps, L = syn.system(o, v, J, 0.1, 1)
    prob = cc.Problem(eps, L, o)
    st = mu.scc_state(prob)
    sols = {t: mu.solve_multipliers(prob, st, t) for t in TARGETS}
    return prob, st, sols


def test_stationarity_and_closed_forms(system):
    prob, st, sols = system
    assert abs(st["zeta"]) > 1e-3            # a genuinely constrained case
    for target, M in sols.items():
        assert M["residual"] < 1e-10, target
        g = mu.stationarity(prob, st, target, M)
        # R0 stationarity holds with lb0_k = gbar dO/dr0_k / omega_k
        assert abs(float(g["r0a"])) < 1e-10 and abs(float(g["r0b"])) < 1e-10
        # Lambda stationarity holds with Ebar_k = E_k (delta_kn - <Lbar_k|R_k>)
        gl = mu.lambda_stationarity(prob, st, target, M)
        assert float(gl[0].norm()) < 1e-10 and float(gl[1].norm()) < 1e-10
        # the remaining equations are exactly stationary too
        for k in ("t", "Ra", "Rb"):
            assert float(g[k].norm()) < 1e-10, (target, k)
        assert abs(float(g["zeta"])) < 1e-10


def test_gauge_direction_is_exactly_two_dimensional(system):
    """Lb_k -> Lb_k + alpha L_k leaves the equations unchanged (the bra
    K_k is invariant), so the system has exactly two null directions."""
    prob, st, sols = system
    s = np.linalg.svd(sols[("gradient", 0)]["matrix"].numpy(), compute_uv=False)
    assert s[-1] < 1e-12 and s[-2] < 1e-12 and s[-3] > 1e-6
    M = dict(sols[("gradient", 0)])
    M2 = mu.closed_forms(prob, st, ("gradient", 0), M["zbar"], M["Lba"] + 0.7 * st["La"],
                         M["Lbb"] - 0.3 * st["Lb"], M["gbar"])
    D1, G = mu.lagrangian_densities(prob, st, ("gradient", 0), M)
    D1b, Gb = mu.lagrangian_densities(prob, st, ("gradient", 0), M2)
    assert float((D1 - D1b).abs().max()) < 1e-12 and float((G - Gb).abs().max()) < 1e-12
    K = mu.gauge_free(st, ("gradient", 0), M2)
    for a, b in zip(K, M["K"]):
        assert float((a - b).abs().max()) < 1e-12


def test_lagrangian_derivatives_equal_finite_differences(system):
    prob, st, sols = system
    o, v, J, n = prob.o, prob.v, prob.J, prob.n
    rng = np.random.default_rng(5)
    h1 = rng.normal(0, 0.1, (n, n))
    h1 = h1 + h1.T
    L1 = rng.normal(0, 0.01, (J, n, n))
    L1 = L1 + L1.transpose(0, 2, 1)
    e = 1e-4
    sp = mu.scc_state(mu.perturbed_problem(prob, h1, L1, e), near=st)
    sm = mu.scc_state(mu.perturbed_problem(prob, h1, L1, -e), near=st)
    Ep, Op = mu.observables(sp, st)
    Em, Om = mu.observables(sm, st)
    E0, O0 = mu.observables(st, st)
    assert abs(O0[(0, 1)]) < 1e-12 and abs(O0[(1, 0)]) < 1e-12   # biorthonormal at x0
    for target in TARGETS:
        D1, G = mu.lagrangian_densities(prob, st, target, sols[target])
        analytic = float((D1 * torch.tensor(h1)).sum() + (G * torch.tensor(L1)).sum())
        if target[0] == "gradient":
            fd = (Ep[target[1]] - Em[target[1]]) / (2 * e)
        else:
            k = (target[1], target[2])
            fd = (Op[k] - Om[k]) / (2 * e)
        assert abs(analytic - fd) < 1e-7 * max(1.0, abs(fd)), (target, analytic, fd)
