"""Similarity-constraint pieces of SCCSD in the FP64 oracle (test infrastructure).

This file is part of the oracle. Only tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does.

SCCSD adds zeta X3 to the cluster operator, X3 = R1^a R2^b - R1^b R2^a
(Sec. 2.4.1), and the only surviving correction to the projected equations
is zeta <mu~|[Hhat, X3]|HF> = zeta <mu~|Hhat X3|HF> (Sec. 2.4.2; X3 Hhat|HF>
has rank >= 3). For a product R1 R2 of commuting excitation operators,

  <mu~|Hhat R1 R2|HF> = <mu~|[[Hhat,R1],R2]|HF>
                        + [mu single] r1_mu <HF|Hhat R2|HF>
                        + [mu double] ( (r1 (x) s1)_mu + r2_mu <HF|Hhat R1|HF> )

with s1_kappa = <kappa~|Hhat R2|HF> over singles and (r1 (x) s1) the doubles
amplitude r1_P s1_Q + s1_P r1_Q. This follows from Hhat R1 R2 =
[[Hhat,R1],R2] + R2 [Hhat,R1] + R1 Hhat R2 and a resolution of the identity
in the biorthonormal excitation basis. Each piece is a derivative of the
CCSD functions at T2 = 0 with the current T1 dressing:

  <mu~|[[Hhat,R1],R2]|HF> = d^2/ds du Omega(t1 + s r1, u r2),
  <kappa~|Hhat R2|HF>      = d/du Omega_1(t1, u r2),
  <HF|Hhat R2|HF>          = d/du E0(t1, u r2),
  <HF|Hhat R1|HF>          = d/ds E0(t1 + s r1, 0).

The orthogonality O_ab = <psi_a|P|psi_b> of the natural projection
(Sec. 2.4.1, 2.4.2) is the Hilbert-space inner product of the HF+S+D parts
of psi = exp(T)(R0 + R)|HF>, T without X3 (the triples part of the cluster
operator does not reach the projected space).
"""
from __future__ import annotations

import numpy as np
import torch
from torch.func import jvp

from . import ccsd as cc

DT = torch.float64


def _cc(t1, t2, h, L, o):
    E0, O1, O2 = cc.ccsd_energy_residual(t1, t2, h, L, o)
    return E0, cc.pack(O1, O2)


def xi(t1, Rx, Ry, h, L, o, v):
    """<mu~|Hhat R1(Rx) R2(Ry)|HF> in the packed layout.
    The SCC ground-state term of Sec. 2.4.2."""
    ov = o * v
    r1, r2 = cc.unpack(Rx, o, v)[0], cc.unpack(Ry, o, v)[1]
    z2 = torch.zeros(v, o, v, o, dtype=DT)

    def f_u(t1_, u):
        return _cc(t1_, u * r2, h, L, o)

    # d/du at u = 0 for a given t1
    def du(t1_):
        one = torch.ones((), dtype=DT)
        zero = torch.zeros((), dtype=DT)
        (_, _), (dE, dO) = jvp(lambda u: f_u(t1_, u), (zero,), (one,))
        return dE, dO

    # mixed derivative d/ds of du(t1 + s r1)
    zero = torch.zeros((), dtype=DT)
    one = torch.ones((), dtype=DT)
    (e2, s_all), (_, dd) = jvp(lambda s: du(t1 + s * r1), (zero,), (one,))
    (_, _), (e1, _) = jvp(lambda s: _cc(t1 + s * r1, z2, h, L, o), (zero,), (one,))
    s1 = s_all[:ov].reshape(v, o)
    out = dd.clone()
    out[:ov] = out[:ov] + r1.reshape(-1) * e2
    prod = torch.einsum("ai,bj->aibj", r1, s1)
    prod = prod + prod.permute(2, 3, 0, 1)
    extra2 = cc.pack(torch.zeros(v, o, dtype=DT), prod)[ov:] + r2_packed(Ry, ov) * e1
    out[ov:] = out[ov:] + extra2
    return out


def r2_packed(R, ov):
    """The packed doubles part of a packed vector."""
    return torch.as_tensor(R, dtype=DT)[ov:]


def projected_state(x_t, R0, R, o, v):
    """(c0, c1[a,i], c2[a,i,b,j]): HF+S+D part of exp(T)(R0 + R)|HF>.
    The natural projection of Sec. 2.4.1."""
    t1, t2 = cc.unpack(x_t, o, v)
    r1, r2 = cc.unpack(R, o, v)
    c0 = torch.as_tensor(R0, dtype=DT)
    c1 = r1 + c0 * t1
    tr = torch.einsum("ai,bj->aibj", t1, r1)
    tt = torch.einsum("ai,bj->aibj", t1, t1)
    c2 = r2 + tr + tr.permute(2, 3, 0, 1) + c0 * (t2 + tt)
    return c0, c1, c2


def metric_product(x, y):
    """Hilbert-space inner product of two HF+S+D kets given as (c0, c1, c2):
    <S|S'> = 2 sum c1 c1', <D|D'> = sum c2 (2 c2' - c2' exchanged).
    The inner product in O_kl of Sec. 2.2."""
    x0, x1, x2 = x
    y0, y1, y2 = y
    return (x0 * y0 + 2.0 * torch.sum(x1 * y1)
            + torch.sum(x2 * (2.0 * y2 - y2.permute(0, 3, 2, 1))))


def overlap(x_t, Ra0, Ra, Rb0, Rb, o, v):
    """O_ab of the natural projection (Sec. 2.4.2)."""
    return metric_product(projected_state(x_t, Ra0, Ra, o, v),
                          projected_state(x_t, Rb0, Rb, o, v))


def overlap_states(x_t, Ra0, Ra, Rb0, Rb, o, v):
    """O_ab of the state projection P = sum_kl |R_k> (S^-1)_kl <R_l| over
    K = {a, b} (Sec. 2.4.1), S_kl = <R_k|R_l>: <psi_a|R_k> needs only the
    HF+S+D part of psi_a = exp(T)|R_a>, since |R_k> lives there."""
    zero = torch.zeros(torch.as_tensor(x_t).shape, dtype=DT)
    ca, cb = projected_state(x_t, Ra0, Ra, o, v), projected_state(x_t, Rb0, Rb, o, v)
    ra, rb = projected_state(zero, Ra0, Ra, o, v), projected_state(zero, Rb0, Rb, o, v)
    S = torch.stack([torch.stack([metric_product(ra, ra), metric_product(ra, rb)]),
                     torch.stack([metric_product(rb, ra), metric_product(rb, rb)])])
    m = torch.stack([metric_product(ca, ra), metric_product(ca, rb)])
    n = torch.stack([metric_product(ra, cb), metric_product(rb, cb)])
    return m @ torch.linalg.solve(S, n)


def fix_sign(x):
    """Sign convention for state vectors: largest |component| positive.
    A convention of this code, not of the paper."""
    return -x if x[np.argmax(np.abs(x))] < 0 else x


def solve_scc(prob, tol=1e-10, maxit=40, ground_tol=1e-11, eom_tol=1e-9, dense=False,
              start=None, projection="natural"):
    """Self-consistent SCCSD for the two lowest states a, b (K = {a, b},
    Sec. 2.4.2): find zeta with O_ab(zeta) = 0, where at each zeta the ground
    state T(zeta) is converged with X3 built from the current R_a, R_b and the
    states are the two lowest right EOM roots of the SCC Jacobian; R0 = eta.R/omega
    (block form of the EOM matrix, Sec. 2.1). The root is followed from zeta = 0
    (plain CCSD) by the secant method on O_ab. dense=True takes the roots from
    the explicit Jacobian (small systems); start = (zeta, t, Ra, Rb) of a
    nearby solution replaces the zeta = 0 start. projection = "state" constrains
    O_ab of the state projection instead (SCCSD(K), Sec. 2.4.1). Returns a dict."""
    from . import solvers as sv
    from . import response as rp
    o, v = prob.o, prob.v
    zeta, Ra, Rb, x = (0.0, None, None, None) if start is None else start
    hist = []
    for it in range(1, maxit + 1):
        scc = None if Ra is None else (zeta, torch.tensor(Ra), torch.tensor(Rb))
        x, E0, _ = sv.ground_state(prob, tol=ground_tol, scc=scc, x0=x)
        if dense:
            w, X = sv.eom_dense(prob, x, 2, side="right", scc=scc)
        else:
            w, X = sv.eom(prob, x, 2, side="right", tol=eom_tol, scc=scc)
        Xa, Xb = fix_sign(X[0]), fix_sign(X[1])
        eta = rp.eta(prob, x, scc=scc).numpy()
        r0a, r0b = float(eta @ Xa / w[0]), float(eta @ Xb / w[1])
        ovl = overlap if projection == "natural" else overlap_states
        O = float(ovl(torch.tensor(x), r0a, torch.tensor(Xa), r0b, torch.tensor(Xb), o, v))
        hist.append((zeta, O))
        Ra, Rb = Xa, Xb
        if abs(O) < tol and len(hist) > 1 and abs(hist[-1][0] - hist[-2][0]) < 1e-8:
            return {"zeta": zeta, "O": O, "E0": E0, "omega": w, "t": x, "Ra": Xa, "Rb": Xb,
                    "r0": (r0a, r0b), "iterations": it}
        if len(hist) == 1:
            zeta = zeta - O
        else:
            (z1, o1), (z2, o2) = hist[-2], hist[-1]
            zeta = z2 - o2 * (z2 - z1) / (o2 - o1) if o2 != o1 else z2
    raise RuntimeError("SCC zeta iteration did not converge")


# ---------------------------------------------------- several constrained states

def overlaps(x_t, states, o, v, projection="natural"):
    """O_kl for every pair k < l of the states [(R0_k, R_k), ...] in K
    (Sec. 2.2): natural projection as in overlap(), or the state projection
    over all of K, P = sum_mn |R_m> (S^-1)_mn <R_n| (Sec. 2.4.1), so that
    O_kl = sum_mn <psi_k|R_m> (S^-1)_mn <R_n|psi_l>. Returns {(k, l): O_kl}."""
    K = len(states)
    if projection == "natural":
        return {(k, l): overlap(x_t, states[k][0], states[k][1], states[l][0], states[l][1], o, v)
                for k in range(K) for l in range(k + 1, K)}
    zero = torch.zeros(torch.as_tensor(x_t).shape, dtype=DT)
    c = [projected_state(x_t, r0, R, o, v) for r0, R in states]
    r = [projected_state(zero, r0, R, o, v) for r0, R in states]
    S = torch.stack([torch.stack([metric_product(r[m], r[n]) for n in range(K)]) for m in range(K)])
    M = torch.stack([torch.stack([metric_product(c[k], r[m]) for m in range(K)]) for k in range(K)])
    W = torch.linalg.solve(S, M.T)                 # S^-1 <R_n|psi_l>, column l
    return {(k, l): M[k] @ W[:, l] for k in range(K) for l in range(k + 1, K)}


def solve_scc_states(prob, nstates, tol=1e-10, maxit=60, ground_tol=1e-11, eom_tol=1e-9,
                     dense=True, projection="natural"):
    """Self-consistent SCCSD for the nstates lowest states, K = {1..nstates}
    (Sec. 2.2 with several states): one zeta_kl per pair k < l, with
    T + sum_kl zeta_kl X_kl, X_kl = R1^k R2^l - R1^l R2^k (Sec. 2.4.1); at every
    zeta the ground state and the nstates lowest right roots are re-converged,
    and zeta solves O_kl = 0 for all pairs by Broyden's method from zeta = 0
    (plain CCSD) with the unit matrix as the first Jacobian estimate (the
    two-state loop's first step). Returns a dict."""
    from . import solvers as sv
    from . import response as rp
    o, v = prob.o, prob.v
    pairs = [(k, l) for k in range(nstates) for l in range(k + 1, nstates)]
    zeta = np.zeros(len(pairs))
    Jb = np.eye(len(pairs))
    R, x, prev = None, None, None
    for it in range(1, maxit + 1):
        scc = None if R is None else [(float(zeta[p]), torch.tensor(R[k]), torch.tensor(R[l]))
                                      for p, (k, l) in enumerate(pairs)]
        x, E0, _ = sv.ground_state(prob, tol=ground_tol, scc=scc, x0=x)
        if dense:
            w, X = sv.eom_dense(prob, x, nstates, side="right", scc=scc)
        else:
            w, X = sv.eom(prob, x, nstates, side="right", tol=eom_tol, scc=scc)
        R = [fix_sign(X[k]) for k in range(nstates)]
        eta = rp.eta(prob, x, scc=scc).numpy()
        r0 = [float(eta @ R[k] / w[k]) for k in range(nstates)]
        states = [(r0[k], torch.tensor(R[k])) for k in range(nstates)]
        Od = overlaps(torch.tensor(x), states, o, v, projection)
        O = np.array([float(Od[p]) for p in pairs])
        if np.abs(O).max() < tol and prev is not None and np.abs(zeta - prev[0]).max() < 1e-8:
            return {"zeta": dict(zip(pairs, zeta.tolist())), "O": dict(zip(pairs, O.tolist())),
                    "E0": E0, "omega": w, "t": x, "R": R, "r0": r0, "iterations": it}
        if prev is not None:
            dz, dO = zeta - prev[0], O - prev[1]
            if dz @ dz > 0:
                Jb = Jb + np.outer(dO - Jb @ dz, dz) / (dz @ dz)
        prev = (zeta.copy(), O.copy())
        zeta = zeta - np.linalg.solve(Jb, O)
    raise RuntimeError("SCC zeta iteration did not converge")
