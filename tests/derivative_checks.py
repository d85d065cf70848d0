"""Finite-difference check of gradients and couplings through the C ABI,
shared by the CPU test double (tests/test_host_logic.py) and the GPU library
(tests/test_gpu_derivatives.py).

Sec. 2.3.2: the gradient dE_a/dx and the coupling <psi_a|d psi_b/dx> at fixed
orbitals, along random perturbations x of eps and of L, assembled by
sccsd_integral_derivative from the effective densities of the multiplier
solves, must equal central differences of fully re-converged SCCSD energies
E_a = E_HF + E_corr + omega_a and bra-frozen overlaps O_ab (Sec. 2.3.4)."""
import numpy as np
import torch

from oracle import ccsd as cc
from oracle import multipliers as mu
from oracle import response as rp


def e_hf(eps, L, o):
    prob = cc.Problem(eps, L, o)
    return float(rp.residual(prob, np.zeros(prob.dim))[0])


def check(make_ctx, eps, L, o, v, J, projection, h=1e-5, rel=1e-7, seed=7, extra=None):
    """make_ctx(eps, L) -> context; extra(ctx, state), if given, runs on the
    unperturbed context before it closes. Returns the measured differences."""
    n = o + v

    def solve(e, l):
        ctx = make_ctx(e, l)
        ctx.set_projection(projection)
        st = ctx.scc_state(tol=1e-11, ground_tol=1e-12, eom_tol=1e-10, left_tol=1e-10)
        return ctx, st

    ctx, st = solve(eps, L)
    grad = ctx.solve_multipliers(st, ("gradient", 0), tol=1e-11, maxit=800)
    coup = ctx.solve_multipliers(st, ("coupling", 0, 1), tol=1e-11, maxit=800)
    t0, La0, Lb0 = (np.asarray(st[k]) for k in ("t", "La", "Lb"))

    def observables(e, l):
        c2, s2 = solve(e, l)
        c2.close()
        Rb = np.asarray(s2["Rb"])
        sc_ = 1.0 / float(Lb0 @ Rb)          # L_b(x0) . R_b(x) = 1
        O = float(mu.frozen_overlap(torch.tensor(s2["t"]), torch.tensor(t0), torch.tensor(La0),
                                    s2["r0b"] * sc_, torch.tensor(Rb * sc_), o, v))
        return e_hf(e, l, o) + s2["e_corr"] + s2["omega_a"], O

    rng = np.random.default_rng(seed)
    de = rng.normal(size=n)
    dL = rng.normal(size=(J, n, n))
    dL = 0.5 * (dL + dL.transpose(0, 2, 1))
    # h = diag(eps) - sum_k (2 g_pqkk - g_pkkq) changes with eps and, to first order, with L
    Lkk, dLkk = np.einsum("Jkk->J", L[:, :o, :o]), np.einsum("Jkk->J", dL[:, :o, :o])
    dh_L = -(2 * np.einsum("Jpq,J->pq", dL, Lkk) + 2 * np.einsum("Jpq,J->pq", L, dLkk)
             - np.einsum("Jpk,Jkq->pq", dL[:, :, :o], L[:, :o, :])
             - np.einsum("Jpk,Jkq->pq", L[:, :, :o], dL[:, :o, :]))
    out = {}
    for direction in ("eps", "L"):
        if direction == "eps":
            plus, minus = observables(eps + h * de, L), observables(eps - h * de, L)
            h1, L1, Gg, Gc = np.diag(de), None, None, None
        else:
            plus, minus = observables(eps, L + h * dL), observables(eps, L - h * dL)
            h1, L1, Gg, Gc = dh_L, dL, grad["Gamma"], coup["Gamma"]
        fd_E = (plus[0] - minus[0]) / (2 * h)
        fd_O = (plus[1] - minus[1]) / (2 * h)
        dE = ctx.integral_derivative(grad["D1"], Gg, h1, L1)
        dO = ctx.integral_derivative(coup["D1"], Gc, h1, L1)
        assert abs(dE - fd_E) < rel * max(1.0, abs(fd_E)), (direction, dE, fd_E)
        assert abs(dO - fd_O) < rel * max(1.0, abs(fd_O)), (direction, dO, fd_O)
        # the same through the inputs (eps, L), with h's change formed by the library
        d_eps = de if direction == "eps" else np.zeros(n)
        d_L = None if direction == "eps" else dL
        iE = ctx.input_derivative(grad["D1"], Gg, d_eps, d_L)
        iO = ctx.input_derivative(coup["D1"], Gc, d_eps, d_L)
        assert abs(iE - dE) < 1e-10 * max(1.0, abs(dE)), (direction, iE, dE)
        assert abs(iO - dO) < 1e-10 * max(1.0, abs(dO)), (direction, iO, dO)
        out[direction] = (abs(dE - fd_E), abs(dO - fd_O))
    if extra is not None:
        extra(ctx, st)
    ctx.close()
    return out
