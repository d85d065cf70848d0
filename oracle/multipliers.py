"""Lagrangian multipliers of SCCSD gradients and couplings (FP64 oracle).

This file is part of the oracle (test infrastructure). Only tests, the smoke
check and the benchmark's CPU-baseline leg may import it; the product path
never does.

K = {a, b} with the natural projection (Sec. 2.4.1), one constraint scalar
zeta and one orthogonality multiplier gamma_bar for O_ab. The orbitals are
held fixed (no kappa_bar F_ai term): the integral derivatives below are those
of the energy (or of the bra-frozen overlap) with respect to the integrals in
the fixed MO basis.

Lagrangian (Sec. 2.3.1, gradient of state n; coupling: first term O_mn):

  Lag = E_n + sum_k [ <Lbar_k|Hbar|R_k> - E_k <Lbar_k|R_k> ]
            + sum_k Ebar_k (1 - <Lambda_k|R_k>) + gbar O_ab + zbar . Omega

with full vectors Lbar_k = (lb0_k, Lb_k), R_k = (r0_k, R_k), Lambda_k = L_k
(the left EOM vectors, Sec. 2.3.3), E_k = <Lambda_k|Hbar|R_k>, and Hbar
depending on t, zeta, R_a, R_b through T + zeta X3 (Sec. 2.4.2). <L|Hbar|R>
is the transition element of oracle/response.py.

Stationarity (Sec. 2.3.3): with respect to Lambda_k it gives
Ebar_k = E_k (delta_kn - <Lbar_k|R_k>) (coupling: -E_k <Lbar_k|R_k>); with
respect to r0_k, lb0_k = gbar (dO_ab/dr0_k) / omega_k; with respect to t,
zeta, R_a, R_b a linear system in (zbar, Lb_a, Lb_b, gbar). That system is
singular along Lb_k -> Lb_k + alpha L_k (the Lagrangian depends on Lb_k only
through K_k = (delta_kn - <Lbar_k|R_k>) Lambda_k + Lb_k, the bra of Sec.
2.3.2); the gauge-free results are K_k, lb0_k, zbar, gbar and the densities.

The bra-frozen overlap O_mn = <psi_m(x0)|psi_n(x)> (Sec. 2.3.4), with fixed
orbitals and exp(-T0) exp(T) = exp(T - T0) (excitation operators commute),
keeps only the rank <= 2 part of exp(dT) R_n, dT = T - T0 (the X3 part cannot
reach a rank <= 2 bra):

  O_mn = L_m . [ r0_n (dt + dT1 dT1 / 2) + R_n + dT1 R1_n ]   (packed kets).
"""
from __future__ import annotations

import numpy as np
import torch
from torch.func import grad

from . import ccsd as cc
from . import response as rp
from . import scc as sc
from . import solvers as sv

DT = torch.float64


def _t(x):
    return torch.as_tensor(x, dtype=DT)


def singles_product(x, y, o, v):
    """Packed ket of X1 Y1|HF> (doubles only): amplitude x_P y_Q + x_Q y_P.
    The T1 T1 and T1 R1 doubles of exp(T - T0) in the bra-frozen overlap O_mn of Sec. 2.3.4."""
    x1 = _t(x)[: o * v].reshape(v, o)
    y1 = _t(y)[: o * v].reshape(v, o)
    p = torch.einsum("ai,bj->aibj", x1, y1)
    p = p + p.permute(2, 3, 0, 1)
    return cc.pack(torch.zeros(v, o, dtype=DT), p)


def frozen_overlap(t, t0, Lm, r0n, Rn, o, v):
    """O_mn = <psi_m(x0)|psi_n(x)> for fixed orbitals (Sec. 2.3.4)."""
    dt = _t(t) - _t(t0)
    ov = o * v
    dt1 = torch.cat([dt[:ov], torch.zeros_like(dt[ov:])])
    ket = (r0n * (dt + 0.5 * singles_product(dt1, dt1, o, v)) + _t(Rn)
           + singles_product(dt1, Rn, o, v))
    return torch.dot(_t(Lm), ket)


def _overlap_of(st):
    """O_ab of the state's projection: natural (default) or state (Sec. 2.4.1)."""
    return sc.overlap_states if st.get("projection", "natural") == "state" else sc.overlap


def scc_state(prob, tol=1e-12, ground_tol=1e-12, near=None, projection="natural"):
    """Converged SCCSD for K = {a, b} (small systems: roots from the explicit
    Jacobian): t, zeta, right vectors (r0, R), left vectors L (L_k . R_k = 1),
    omegas and E0. near: a state of a nearby system to start from.
    SCCSD of Sec. 2.2 and 2.4, the state the Lagrangian of Sec. 2.3.1 is taken at."""
    start = None if near is None else (near["zeta"], near["t"].numpy(), near["Ra"].numpy(),
                                       near["Rb"].numpy())
    s = sc.solve_scc(prob, tol=tol, ground_tol=ground_tol, dense=True, start=start,
                     projection=projection)
    scc = (s["zeta"], _t(s["Ra"]), _t(s["Rb"]))
    wl, XL = sv.eom_dense(prob, s["t"], 2, side="left", scc=scc)
    La = XL[0] / (XL[0] @ s["Ra"])
    Lb = XL[1] / (XL[1] @ s["Rb"])
    return {"t": _t(s["t"]), "zeta": float(s["zeta"]), "Ra": _t(s["Ra"]), "Rb": _t(s["Rb"]),
            "r0a": float(s["r0"][0]), "r0b": float(s["r0"][1]), "La": _t(La), "Lb": _t(Lb),
            "omega": (float(s["omega"][0]), float(s["omega"][1])), "E0": float(s["E0"]),
            "omega_left": (float(wl[0]), float(wl[1])), "o": prob.o, "v": prob.v,
            "projection": projection}


def _target(target):
    """('gradient', n) or ('coupling', m, n) with state indices 0 (a), 1 (b)."""
    if target[0] == "gradient":
        return "gradient", None, int(target[1])
    if target[0] == "coupling":
        return "coupling", int(target[1]), int(target[2])
    raise ValueError(target)


def lagrangian(prob, st, target, P, M, h=None, L=None, lam=None):
    """Value of the Lagrangian at parameters P and multipliers M.

    P: t, zeta, r0a, Ra, r0b, Rb.  M: zbar, lb0a, Lba, lb0b, Lbb, Ea, Eb, gbar.
    lam = (Lambda_a, Lambda_b), by default the left vectors of st; the frozen
    bra L_m and t0 of a coupling always come from st.
    The Lagrangian of Sec. 2.3.1, with the SCCSD terms of Sec. 2.4.2."""
    h = prob.h if h is None else h
    L = prob.L if L is None else L
    o, v = prob.o, prob.v
    kind, m, n = _target(target)
    t, zeta = P["t"], P["zeta"]
    scc = (zeta, P["Ra"], P["Rb"])
    kets = [(P["r0a"], P["Ra"]), (P["r0b"], P["Rb"])]
    lam = [st["La"], st["Lb"]] if lam is None else list(lam)
    bars = [(M["lb0a"], M["Lba"]), (M["lb0b"], M["Lbb"])]
    Ebar = [M["Ea"], M["Eb"]]

    def T(l0, Lv, k):
        r0, R = kets[k]
        return rp.transition_element(prob, t, l0, Lv, r0, R, h, L, scc=scc)

    zero = torch.zeros((), dtype=DT)
    E = [T(zero, lam[k], k) for k in range(2)]
    if kind == "gradient":
        val = E[n]
    else:
        Lm = [st["La"], st["Lb"]][m]
        r0n, Rn = kets[n]
        val = frozen_overlap(t, st["t"], Lm, r0n, Rn, o, v)
    for k in range(2):
        l0, Lb = bars[k]
        r0, R = kets[k]
        val = val + T(l0, Lb, k) - E[k] * (l0 * r0 + torch.dot(Lb, R))
        val = val + Ebar[k] * (1.0 - torch.dot(lam[k], R))
    val = val + M["gbar"] * _overlap_of(st)(t, P["r0a"], P["Ra"], P["r0b"], P["Rb"], o, v)
    _, Om = cc.energy_residual(t, prob, h=h, L=L, scc=scc)
    return val + torch.dot(M["zbar"], Om)


def params_of(st):
    """The parameters of the Lagrangian of Sec. 2.3.1 (t, zeta, r0 and R of both states) as tensors
    for differentiation."""
    return {"t": st["t"].clone(), "zeta": torch.tensor(st["zeta"], dtype=DT),
            "r0a": torch.tensor(st["r0a"], dtype=DT), "Ra": st["Ra"].clone(),
            "r0b": torch.tensor(st["r0b"], dtype=DT), "Rb": st["Rb"].clone()}


def overlap_r0_derivatives(prob, st):
    """(dO_ab/dr0_a, dO_ab/dr0_b) at the solution.
    The dO/dR0 terms of the stationarity equations (Sec. 2.3.3)."""
    P = params_of(st)
    f = lambda ra0, rb0: _overlap_of(st)(P["t"], ra0, P["Ra"], rb0, P["Rb"], prob.o, prob.v)
    g = grad(f, argnums=(0, 1))(P["r0a"], P["r0b"])
    return float(g[0]), float(g[1])


def closed_forms(prob, st, target, zbar, Lba, Lbb, gbar, dO_dr0=None):
    """Full multiplier set from the unknowns: lb0_k (R0 stationarity) and
    Ebar_k (Lambda stationarity), Sec. 2.3.3."""
    kind, _, n = _target(target)
    dO = overlap_r0_derivatives(prob, st) if dO_dr0 is None else dO_dr0
    lb0 = [gbar * dO[0] / st["omega"][0], gbar * dO[1] / st["omega"][1]]
    kets = [(st["r0a"], st["Ra"]), (st["r0b"], st["Rb"])]
    E = [st["E0"] + st["omega"][0], st["E0"] + st["omega"][1]]
    bars = [Lba, Lbb]
    Ebar = []
    for k in range(2):
        c = lb0[k] * kets[k][0] + torch.dot(_t(bars[k]), kets[k][1])
        d = 1.0 if (kind == "gradient" and k == n) else 0.0
        Ebar.append(E[k] * (d - c))
    return {"zbar": _t(zbar), "lb0a": _t(lb0[0]), "Lba": _t(Lba), "lb0b": _t(lb0[1]),
            "Lbb": _t(Lbb), "Ea": _t(Ebar[0]), "Eb": _t(Ebar[1]), "gbar": _t(gbar)}


def stationarity(prob, st, target, M):
    """Derivatives of the Lagrangian with respect to every parameter:
    dict t, zeta, r0a, Ra, r0b, Rb (all zero at the multipliers).
    The stationarity conditions of Sec. 2.3.3 (gradient) and Sec. 2.3.4 (coupling)."""
    P = params_of(st)
    names = ["t", "zeta", "r0a", "Ra", "r0b", "Rb"]
    f = lambda *xs: lagrangian(prob, st, target, dict(zip(names, xs)), M)
    g = grad(f, argnums=tuple(range(len(names))))(*[P[k] for k in names])
    return dict(zip(names, g))


def lambda_stationarity(prob, st, target, M):
    """Derivatives with respect to the bra vectors Lambda_a, Lambda_b.
    The bra conditions of Sec. 2.3.3, which give the closed forms for Ebar and L0bar."""
    P = params_of(st)
    f = lambda La, Lb: lagrangian(prob, st, target, P, M, lam=(La, Lb))
    return grad(f, argnums=(0, 1))(st["La"].clone(), st["Lb"].clone())


def unknowns_dim(prob):
    """Number of unknowns (zetabar, Lbar_a, Lbar_b, gammabar) of the multiplier equations of Sec.
    2.3.3."""
    return 3 * prob.dim + 1


def _split(u, dim):
    return u[:dim], u[dim:2 * dim], u[2 * dim:3 * dim], u[3 * dim]


def residual_map(prob, st, target, dO_dr0=None):
    """u = (zbar, Lb_a, Lb_b, gbar) -> stationarity residual (t, R_a, R_b, zeta)
    with the closed forms for lb0_k and Ebar_k substituted; affine in u.
    The linear system of Sec. 2.3.3 (gradient) or Sec. 2.3.4 (coupling)."""
    dim = prob.dim
    dO = overlap_r0_derivatives(prob, st) if dO_dr0 is None else dO_dr0

    def f(u):
        u = _t(u)
        zb, La_, Lb_, gb = _split(u, dim)
        M = closed_forms(prob, st, target, zb, La_, Lb_, gb, dO)
        g = stationarity(prob, st, target, M)
        return torch.cat([g["t"], g["Ra"], g["Rb"], g["zeta"].reshape(1)])
    return f


def solve_multipliers(prob, st, target):
    """Dense solve of the stationarity equations (small systems only).
    Returns the full multiplier dict plus the gauge-free bras K_a, K_b and the
    residual norm of the solved system.
    Sec. 2.3.3 solves this system iteratively (e.g. Davidson); here it is dense."""
    dim = prob.dim
    N = unknowns_dim(prob)
    dO = overlap_r0_derivatives(prob, st)
    f = residual_map(prob, st, target, dO)
    zero = torch.zeros(N, dtype=DT)
    b = f(zero)
    cols = torch.func.jacfwd(f)(zero)          # the map is affine: f(u) = cols u + b
    u = np.linalg.lstsq(cols.numpy(), -b.numpy(), rcond=1e-13)[0]
    zb, La_, Lb_, gb = _split(_t(u), dim)
    M = closed_forms(prob, st, target, zb, La_, Lb_, gb, dO)
    res = float(torch.linalg.norm(f(_t(u))))
    M["K"] = gauge_free(st, target, M)
    M["residual"] = res
    M["matrix"] = cols
    return M


def gauge_free(st, target, M):
    """K_k = (delta_kn - <Lbar_k|R_k>) Lambda_k + Lb_k (Sec. 2.3.2; coupling
    without delta_kn)."""
    kind, _, n = _target(target)
    out = []
    for k, (l0, Lb, r0, R, lam) in enumerate([(M["lb0a"], M["Lba"], st["r0a"], st["Ra"], st["La"]),
                                               (M["lb0b"], M["Lbb"], st["r0b"], st["Rb"], st["Lb"])]):
        c = l0 * r0 + torch.dot(Lb, R)
        d = 1.0 if (kind == "gradient" and k == n) else 0.0
        out.append((d - c) * lam + Lb)
    return out


def lagrangian_densities(prob, st, target, M):
    """(D1[n][n], Gamma[J][n][n]) = derivatives of the Lagrangian with respect
    to h_pq and L^J_pq at fixed parameters and multipliers (Sec. 2.3.2)."""
    P = params_of(st)
    g = grad(lambda h, L: lagrangian(prob, st, target, P, M, h=h, L=L),
             argnums=(0, 1))(prob.h, prob.L)
    return g[0], g[1]


def perturbed_problem(prob, h1, L1, e):
    """Copy of prob with integrals h + e h1, L + e L1 (fixed orbitals).
    The gradient and couplings are derivatives with respect to these integrals (Sec. 2.3.2)."""
    p = cc.Problem(prob.eps, prob.L, prob.o)
    p.h = prob.h + e * _t(h1)
    p.L = prob.L + e * _t(L1)
    return p


def observables(st, st0):
    """Energies E_a, E_b and bra-frozen overlaps O_ab, O_ba of the state st
    relative to the reference state st0 (Lambda_k = L_k of st0 fixes the
    normalisation of the kets of st, Sec. 2.3.1)."""
    E = (st["E0"] + st["omega"][0], st["E0"] + st["omega"][1])
    kets = []
    for r0, R, lam in [(st["r0a"], st["Ra"], st0["La"]), (st["r0b"], st["Rb"], st0["Lb"])]:
        s = 1.0 / float(torch.dot(lam, R))
        kets.append((r0 * s, R * s))
    o, v = st["o"], st["v"]
    O = {}
    for m, n in [(0, 1), (1, 0)]:
        Lm = [st0["La"], st0["Lb"]][m]
        O[(m, n)] = float(frozen_overlap(st["t"], st0["t"], Lm, kets[n][0], kets[n][1], o, v))
    return E, O
