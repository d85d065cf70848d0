"""Jacobian transformations and densities in the FP64 oracle (test infrastructure).

This file is part of the oracle. Only tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does.

Each quantity is computed from its definition as a derivative of the
ground-state functions in oracle/ccsd.py (exact up to rounding):

* A R   = d/de Omega(t + e R)                     (A of Sec. 2.3.3)
* A^T L = grad_t (L . Omega(t))                   (left transformation)
* eta   = grad_t E0(t)                            (eta of Sec. 2.3.3)
* densities (Sec. 2.3.2) for a bra (L0, L) and a ket (R0, R):

  <L|Hbar|R> = L0 R0 E0 + L0 eta.R + R0 L.Omega + L.(A R) + E0 L.R
               + sum_mu L_mu (R1 (x) Omega1)_mu,

  which follows from <mu~|Hbar|nu> = A_mu,nu + <mu~|tau_nu Hbar|HF> and the
  rank of tau_nu; then d_pq = d<L|Hbar|R>/d h_pq and
  Gamma^J_pq = sum_rs d_pqrs L^J_rs = d<L|Hbar|R>/d L^J_pq.
"""
from __future__ import annotations

import torch
from torch.func import grad, jvp, vjp

from . import ccsd as cc

DT = torch.float64


def _t(x):
    return torch.as_tensor(x, dtype=DT)


def residual(prob, x, scc=None):
    """(E0, Omega) of Sec. 2.1 at packed amplitudes x (SCC term of Sec. 2.4.2 with scc)."""
    return cc.energy_residual(_t(x), prob, scc=scc)


def jacobian_right(prob, x, R, scc=None):
    """A R (packed) at amplitudes x.
    A_mu,nu = d Omega_mu / d t_nu of Sec. 2.1 and 2.3.3, as a forward derivative."""
    f = lambda y: cc.energy_residual(y, prob, scc=scc)[1]
    return jvp(f, (_t(x),), (_t(R),))[1]


def jacobian_left(prob, x, Lv, scc=None):
    """A^T L (packed) at amplitudes x.
    The left transformation of Sec. 2.1, as a reverse derivative."""
    f = lambda y: cc.energy_residual(y, prob, scc=scc)[1]
    _, pull = vjp(f, _t(x))
    return pull(_t(Lv))[0]


def eta(prob, x, scc=None):
    """eta_nu = <HF|[Hbar, tau_nu]|HF> = d E0 / d t_nu (Sec. 2.1 and 2.3.3), as a gradient."""
    return grad(lambda y: cc.energy_residual(y, prob, scc=scc)[0])(_t(x))


def _r1_omega1(R, Om, o, v):
    """Packed doubles of R1 (x) Omega1 (zero singles)."""
    r1 = _t(R)[: o * v].reshape(v, o)
    w1 = Om[: o * v].reshape(v, o)
    p = torch.einsum("ai,bj->aibj", r1, w1)
    p = p + p.permute(2, 3, 0, 1)
    return cc.pack(torch.zeros(v, o, dtype=DT), p)


def transition_element(prob, x, l0, Lv, r0, R, h, L, scc=None):
    """<L|Hbar|R> as a function of the integrals (h, L^J).
    Sec. 2.3.2."""
    o, v = prob.o, prob.v
    x, Lv, R = _t(x), _t(Lv), _t(R)
    f = lambda y: cc.energy_residual(y, prob, h=h, L=L, scc=scc)
    (E0, Om), (dE, dOm) = jvp(f, (x,), (R,))
    val = (l0 * r0 * E0 + l0 * dE + r0 * torch.dot(Lv, Om) + torch.dot(Lv, dOm)
           + E0 * torch.dot(Lv, R) + torch.dot(Lv, _r1_omega1(R, Om, o, v)))
    return val


def densities(prob, x, l0, Lv, r0, R, scc=None):
    """(d_pq[n][n], Gamma^J_pq[J][n][n]) for the bra (l0, L), ket (r0, R).
    The densities of Sec. 2.3.2 (with the Delta d of Sec. 2.4.2 for the SCC state), as derivatives
    of the transition element with respect to h and L^J."""
    g = grad(lambda h, L: transition_element(prob, x, l0, Lv, r0, R, h, L, scc),
             argnums=(0, 1))(prob.h, prob.L)
    return g[0], g[1]
