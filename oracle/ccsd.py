"""Plain closed-shell (S)CCSD oracle in FP64 on the CPU (test infrastructure).

This file is part of the oracle. Only tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does.

Everything is written with full tensors and torch.einsum in float64, in the
order of the defining expressions, with no blocking or fusion:

* the synthetic Hamiltonian (canonical HF reference: F = diag(eps), the
  Brillouin condition F_ai = 0 that the Lagrangian of Sec. 2.3.1 imposes);
* the T1-transformed Hamiltonian Hhat = exp(-T1) H exp(T1) (Sec. 2.4.2),
  which for a one-body similarity transform is the one-index transformation
  hhat = (1 - t1) h (1 + t1), Lhat^J = (1 - t1) L^J (1 + t1);
* the ground-state projections E0 = <HF|Hbar|HF>, Omega_mu = <mu~|Hbar|HF>
  (Sec. 2.1) with Hbar = exp(-T2) Hhat exp(T2) truncated where the rank of
  the projection makes the rest vanish.

The closed-shell working equations are not printed in the paper; they follow
from these definitions, and every term is checked against the brute-force
determinant engine in oracle/determinant.py.

Derived quantities are *defined* as derivatives of these functions, and the
oracle obtains them as such (torch.func forward/reverse differentiation,
exact up to rounding):

* A_mu,nu = d Omega_mu / d t_nu (Sec. 2.3.3), so A R is a directional
  derivative and A^T L a gradient of L . Omega;
* eta_nu = d E0 / d t_nu;
* one- and two-particle densities of Sec. 2.3.2: d_pq = d<L|Hbar|R>/d h_pq
  and Gamma^J_pq = sum_rs d_pqrs L^J_rs = d<L|Hbar|R>/d L^J_pq.

Layouts: singles t1[a, i]; full doubles t2[a, i, b, j] = t_ij^ab, symmetric
under (ai) <-> (bj); packed vectors as in oracle/determinant.py.
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64


# --------------------------------------------------------------------------
# layout helpers (oracle-private)
# --------------------------------------------------------------------------

def pack(t1: torch.Tensor, t2: torch.Tensor) -> torch.Tensor:
    """Packed layout of (t1[a][i], t2[a][i][b][j]): singles at a*o + i, then each doubles pair (ai)
    <= (bj) once (the singles and doubles manifold of Sec. 2.1, with t_ij^ab = t_ji^ba)."""
    v, o = t1.shape
    ov = o * v
    M = t2.reshape(ov, ov)
    Q, P = np.tril_indices(ov)
    return torch.cat([t1.reshape(-1), M[P, Q]])


def unpack(x, o: int, v: int):
    """Inverse of pack: (t1[a][i], t2[a][i][b][j]) from the packed layout (Sec. 2.1)."""
    x = torch.as_tensor(x, dtype=DT)
    ov = o * v
    t1 = x[:ov].reshape(v, o)
    Q, P = np.tril_indices(ov)
    M = torch.zeros(ov, ov, dtype=DT)
    M = M.index_put((torch.as_tensor(P), torch.as_tensor(Q)), x[ov:])
    M = M.index_put((torch.as_tensor(Q), torch.as_tensor(P)), x[ov:])
    return t1, M.reshape(v, o, v, o)


def bra_full(l2_packed_as_full: torch.Tensor) -> torch.Tensor:
    """Weights so that sum_packed L X = sum_full W X for symmetric X:
    off-diagonal pairs count 1/2 each (they appear twice), diagonal 1.
    Biorthonormal bras <mu~| of Sec. 2.1."""
    v, o = l2_packed_as_full.shape[0], l2_packed_as_full.shape[1]
    ov = o * v
    W = 0.5 * l2_packed_as_full.reshape(ov, ov).clone()
    idx = torch.arange(ov)
    W[idx, idx] = 2.0 * W[idx, idx]
    return W.reshape(v, o, v, o)


# --------------------------------------------------------------------------
# Hamiltonian
# --------------------------------------------------------------------------

def one_electron(eps: torch.Tensor, L: torch.Tensor, o: int) -> torch.Tensor:
    """h_pq = eps_p d_pq - sum_k (2 g_pqkk - g_pkkq), so that F = diag(eps).
    The Hamiltonian in h and g is that of Sec. 2.3.2; F = diag(eps) makes the reference canonical
    Hartree-Fock, as the orbital conditions of Sec. 2.3.1 assume."""
    h = torch.diag(eps).clone()
    Lkk = torch.einsum("Jkk->J", L[:, :o, :o])
    h = h - 2.0 * torch.einsum("Jpq,J->pq", L, Lkk)
    h = h + torch.einsum("Jpk,Jkq->pq", L[:, :, :o], L[:, :o, :])
    return h


def t1_matrix(t1: torch.Tensor, n: int) -> torch.Tensor:
    """The singles amplitudes as an n x n matrix X[o + a][i] = t_ai, so that the T1 dressing
    exp(-T1) H exp(T1) of Sec. 2.4.2 transforms the integrals as (1 - X) h (1 + X)."""
    v, o = t1.shape
    X = torch.zeros(n, n, dtype=DT)
    X = torch.cat([torch.zeros(o, n, dtype=DT),
                   torch.cat([t1, torch.zeros(v, v, dtype=DT)], dim=1)], dim=0)
    return X


def dress(h: torch.Tensor, L: torch.Tensor, t1: torch.Tensor):
    """One-index transformation by exp(-T1) ... exp(T1) (Sec. 2.4.2)."""
    n = h.shape[0]
    tm = t1_matrix(t1, n)
    I = torch.eye(n, dtype=DT)
    X, Y = I - tm, I + tm
    hh = X @ h @ Y
    Lh = torch.einsum("pr,Jrs,sq->Jpq", X, L, Y)
    return hh, Lh


def fock(hh: torch.Tensor, Lh: torch.Tensor, o: int) -> torch.Tensor:
    """F_pq = h_pq + sum_k (2 g_pqkk - g_pkkq) from (dressed) integrals.
    Integrals of Sec. 2.3.2, T1-dressed as in Sec. 2.4.2."""
    Lkk = torch.einsum("Jkk->J", Lh[:, :o, :o])
    return (hh + 2.0 * torch.einsum("Jpq,J->pq", Lh, Lkk)
            - torch.einsum("Jpk,Jkq->pq", Lh[:, :, :o], Lh[:, :o, :]))


class Blocks:
    """Dressed two-electron integral blocks g_xyzw = sum_J L_xy L_zw."""

    def __init__(self, Lh: torch.Tensor, o: int):
        self.Lh, self.o = Lh, o
        self.sl = {"o": slice(0, o), "v": slice(o, Lh.shape[1])}

    def __call__(self, spec: str) -> torch.Tensor:
        s = self.sl
        A = self.Lh[:, s[spec[0]], s[spec[1]]]
        B = self.Lh[:, s[spec[2]], s[spec[3]]]
        return torch.einsum("Jpq,Jrs->pqrs", A, B)


# --------------------------------------------------------------------------
# CCSD energy and residual (Sec. 2.1), T1-transformed form (Sec. 2.4.2)
# --------------------------------------------------------------------------

def ccsd_energy_residual(t1, t2, h, L, o):
    """Return (E0, Omega1[a,i], Omega2[a,i,b,j]) of closed-shell CCSD.
    E0 and Omega_mu = <mu~|Hbar|HF> of Sec. 2.1, in the T1-dressed closed-shell form (Sec. 2.4.2)."""
    hh, Lh = dress(h, L, t1)
    F = fock(hh, Lh, o)
    g = Blocks(Lh, o)
    nv = Lh.shape[1] - o
    Foo, Fov, Fvo, Fvv = F[:o, :o], F[:o, o:], F[o:, :o], F[o:, o:]
    u = 2.0 * t2 - t2.permute(0, 3, 2, 1)          # u[a,i,b,j] = 2t_ij^ab - t_ji^ab

    # energy: <HF|Hhat|HF> + sum (2 g_iajb - g_ibja) t_ij^ab
    goooo = g("oooo")
    e_ref = 2.0 * torch.einsum("ii->", hh[:o, :o]) + \
        torch.einsum("iijj->", 2.0 * goooo) - torch.einsum("ijji->", goooo)
    govov = g("ovov")
    E0 = e_ref + torch.einsum("aibj,iajb->", t2, 2.0 * govov) \
        - torch.einsum("aibj,ibja->", t2, govov)

    # singles residual
    gvvov = g("vvov")          # g[a,d,k,c]
    gooov = g("ooov")          # g[k,i,l,c]
    O1 = Fvo.clone()
    O1 = O1 + torch.einsum("ckdi,adkc->ai", u, gvvov)
    O1 = O1 - torch.einsum("akcl,kilc->ai", u, gooov)
    O1 = O1 + torch.einsum("aick,kc->ai", u, Fov)

    # doubles residual
    gvovo = g("vovo")          # g[a,i,b,j]
    gvvvv = g("vvvv")          # g[a,c,b,d]
    A2 = gvovo + torch.einsum("cidj,acbd->aibj", t2, gvvvv)
    B2 = torch.einsum("akbl,kilj->aibj", t2, goooo + torch.einsum("cidj,kcld->kilj", t2, govov))
    goovv = g("oovv")          # g[k,i,a,c]
    X = goovv - 0.5 * torch.einsum("aldi,kdlc->kiac", t2, govov)
    C2 = -0.5 * torch.einsum("bkcj,kiac->aibj", t2, X) - torch.einsum("bkci,kjac->aibj", t2, X)
    gvoov = g("voov")          # g[a,i,k,c]
    Lvoov = 2.0 * gvoov - g("vvoo").permute(0, 3, 2, 1)   # L_aikc = 2 g_aikc - g_acki
    Lovov = 2.0 * govov - govov.permute(0, 3, 2, 1)      # L_ldkc = 2 g_ldkc - g_lckd
    Y = Lvoov + 0.5 * torch.einsum("aidl,ldkc->aikc", u, Lovov)
    D2 = 0.5 * torch.einsum("bjck,aikc->aibj", u, Y)
    Fvv_i = Fvv - torch.einsum("bkdl,ldkc->bc", u, govov)
    Foo_i = Foo + torch.einsum("cldj,kdlc->kj", u, govov)
    E2 = torch.einsum("aicj,bc->aibj", t2, Fvv_i) - torch.einsum("aibk,kj->aibj", t2, Foo_i)
    Pp = C2 + D2 + E2
    O2 = A2 + B2 + Pp + Pp.permute(2, 3, 0, 1)
    return E0, O1, O2


# --------------------------------------------------------------------------
# packed-vector interface
# --------------------------------------------------------------------------

class Problem:
    """Integrals of one synthetic system in FP64 torch tensors."""

    def __init__(self, eps, L, o: int):
        self.eps = torch.as_tensor(eps, dtype=DT)
        self.L = torch.as_tensor(L, dtype=DT)
        self.o = o
        self.n = self.L.shape[1]
        self.v = self.n - o
        self.J = self.L.shape[0]
        self.h = one_electron(self.eps, self.L, o)

    @property
    def dim(self) -> int:
        """Size of the packed singles and doubles manifold (Sec. 2.1)."""
        ov = self.o * self.v
        return ov + ov * (ov + 1) // 2


def energy_residual(x, prob: Problem, h=None, L=None, scc=None):
    """(E0, Omega packed) at packed amplitudes x; scc = (zeta, Ra, Rb) adds
    the similarity-constraint term zeta <mu~|[Hhat, X3]|HF> (Sec. 2.4.2). A
    list of such triples, one per pair k < l of constrained states, adds one
    term per pair: T + sum_kl zeta_kl X_kl (Sec. 2.2 for several states)."""
    h = prob.h if h is None else h
    L = prob.L if L is None else L
    o, v = prob.o, prob.v
    t1, t2 = unpack(x, o, v)
    E0, O1, O2 = ccsd_energy_residual(t1, t2, h, L, o)
    Om = pack(O1, O2)
    if scc is not None:
        from .scc import xi
        pairs = scc if isinstance(scc, list) else [scc]
        for zeta, Ra, Rb in pairs:
            Om = Om + zeta * (xi(t1, Ra, Rb, h, L, o, v) - xi(t1, Rb, Ra, h, L, o, v))
    return E0, Om
