"""Lagrangian multipliers of SCCSD gradients and couplings on the GPU
(Sec. 2.3.1-2.3.4): parity with the FP64 oracle, and mixed-precision solves
refined to the FP64 result."""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle import multipliers as mu
from paper_2403_01007_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

TARGETS = [("gradient", 0), ("gradient", 1), ("coupling", 0, 1), ("coupling", 1, 0)]


def _state_of(st):
    return {"t": st["t"].numpy(), "Ra": st["Ra"].numpy(), "Rb": st["Rb"].numpy(),
            "La": st["La"].numpy(), "Lb": st["Lb"].numpy(), "zeta": st["zeta"],
            "r0a": st["r0a"], "r0b": st["r0b"], "omega_a": st["omega"][0],
            "omega_b": st["omega"][1]}


def test_multipliers_match_oracle_tiny():
    """o=2, v=4 at the oracle's converged SCCSD state: every gauge-free
    multiplier and the Lagrangian densities, for both gradients and both
    couplings."""
    from paper_2403_01007_gb300 import binding as B
    o, v, J = 2, 4, 10
    eps, L = syn.system(o, v, J, 0.1, 1)
    prob = cc.Problem(eps, L, o)
    st = mu.scc_state(prob)
    state = _state_of(st)
    ctx = B.Context(o, v, J, eps, L)
    for target in TARGETS:
        res = ctx.solve_multipliers(state, target, tol=1e-11, maxit=800)
        M = mu.solve_multipliers(prob, st, target)
        D1, G = mu.lagrangian_densities(prob, st, target, M)
        assert abs(res["gbar"] - float(M["gbar"])) < 1e-9, target
        assert np.abs(res["zbar"] - M["zbar"].numpy()).max() < 1e-9, target
        for k in range(2):
            assert np.abs(res["K"][k] - M["K"][k].numpy()).max() < 1e-9, target
        assert np.abs(res["D1"] - D1.numpy()).max() < 1e-9, target
        assert np.abs(res["Gamma"] - G.numpy()).max() < 1e-9, target
    ctx.close()


@pytest.fixture(scope="module")
def small_state():
    """SCCSD state of the o=5, v=19, J=72 workload from the GPU's own FP64
    solvers (ground state, both states, zeta; left vectors)."""
    from paper_2403_01007_gb300 import binding as B
    w = syn.SMALL
    eps, L = syn.workload_system(w)
    ctx = B.Context(w.o, w.v, w.J, eps, L)
    state = ctx.scc_state(tol=1e-10, ground_tol=1e-11, eom_tol=1e-9, left_tol=1e-9)
    ctx.close()
    return w, eps, L, state


def test_multipliers_satisfy_oracle_equations_small(small_state):
    """The GPU multipliers of the o=5, v=19 workload make the oracle's
    stationarity residual vanish (the oracle evaluates its own equations at
    the GPU's solution), for a gradient and a coupling."""
    from paper_2403_01007_gb300 import binding as B
    w, eps, L, state = small_state
    prob = cc.Problem(eps, L, w.o)
    st = {"t": torch.tensor(state["t"]), "Ra": torch.tensor(state["Ra"]),
          "Rb": torch.tensor(state["Rb"]), "La": torch.tensor(state["La"]),
          "Lb": torch.tensor(state["Lb"]), "zeta": state["zeta"], "r0a": state["r0a"],
          "r0b": state["r0b"], "omega": (state["omega_a"], state["omega_b"])}
    Ehf = float(cc.energy_residual(torch.zeros(prob.dim, dtype=torch.float64), prob)[0])
    st["E0"] = Ehf + state["e_corr"]
    ctx = B.Context(w.o, w.v, w.J, eps, L)
    dim = prob.dim
    for target in [("gradient", 1), ("coupling", 0, 1)]:
        res = ctx.solve_multipliers(state, target, tol=1e-10, maxit=800, densities=False)
        # unknowns in the gauge Lbar_k . R_k = 0
        d = [1.0 if (target[0] == "gradient" and k == target[1]) else 0.0 for k in range(2)]
        r0 = [state["r0a"], state["r0b"]]
        lam = [state["La"], state["Lb"]]
        Lbar = [res["K"][k] - (d[k] - res["lb0"][k] * r0[k]) * lam[k] for k in range(2)]
        u = np.concatenate([res["zbar"], Lbar[0], Lbar[1], [res["gbar"]]])
        r = mu.residual_map(prob, st, target)(torch.tensor(u)).numpy()
        # relative to the size of the equations' constant part
        b = mu.residual_map(prob, st, target)(torch.zeros(3 * dim + 1, dtype=torch.float64))
        assert np.linalg.norm(r) < 1e-8 * max(1.0, float(torch.linalg.norm(b))), target
    ctx.close()


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_mixed_precision_multipliers_refine_to_fp64(small_state, prec):
    """Mixed-precision multiplier solves, refined by FP64 residuals, give the
    FP64 result: effective densities within 1e-7 max-abs."""
    from paper_2403_01007_gb300 import binding as B
    w, eps, L, state = small_state
    ref_ctx = B.Context(w.o, w.v, w.J, eps, L)
    ref = ref_ctx.solve_multipliers(state, ("gradient", 0), tol=1e-10, maxit=800)
    ref_ctx.close()
    ctx = B.Context(w.o, w.v, w.J, eps, L, precision=prec)
    res = ctx.solve_multipliers(state, ("gradient", 0), tol=1e-10, maxit=800, refine_tol=1e-6)
    assert np.abs(res["D1"] - ref["D1"]).max() < 1e-7
    assert np.abs(res["Gamma"] - ref["Gamma"]).max() < 1e-7
    assert abs(res["gbar"] - ref["gbar"]) < 1e-7
    ctx.close()
