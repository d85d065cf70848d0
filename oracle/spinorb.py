"""Spin-orbital CCSD energy and residual: a second, independent FP64 oracle
(test infrastructure).

This file is part of the oracle. Only tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does.

oracle/ccsd.py writes the closed-shell residual in spin-adapted, T1-dressed
intermediates. This module evaluates the same projections of Sec. 2.1,
E0 = <HF|Hbar|HF> and Omega_mu = <mu|Hbar|HF> with Hbar = exp(-T) H exp(T),
in a different formulation that shares nothing with it:

* spin orbitals (each spatial orbital twice, alpha and beta) and
  antisymmetrised integrals <PQ||RS> = <PQ|RS> - <PQ|SR>, built here from the
  Cholesky vectors ((pq|rs) = sum_J L^J_pq L^J_rs, <pq|rs> = (pr|qs));
* the one-electron operator fixed by the canonical reference of the
  synthetic Hamiltonian, f = diag(eps): h_PQ = eps_P d_PQ - sum_K <PK||QK>;
* T1 kept explicitly (no T1 dressing) and the projected spin-orbital CCSD
  equations in the effective-operator arrangement of Stanton and Gauss
  (J. Chem. Phys. 94, 4334 (1991)), a textbook form of the same definition;
* its own map between the packed closed-shell layout and spin-orbital
  amplitudes, and back.

Closed-shell (singlet) amplitudes in spin orbitals, I = (i, s), A = (a, s):
  t_I^A   = d(s_I, s_A) t_ai
  t_IJ^AB = d(s_I, s_A) d(s_J, s_B) t_ij^ab - d(s_I, s_B) d(s_J, s_A) t_ij^ba.
The projected Hbar|HF> is sum_mu Omega_mu tau_mu |HF> in the biorthonormal
bras of Sec. 2.1 (T2 = 1/2 sum t_aibj E_ai E_bj), so a packed closed-shell
residual component is the coefficient of one determinant:
  Omega_ai   = r_{i alpha}^{a alpha},
  Omega_aibj = r_{i alpha, j beta}^{a alpha, b beta}.

A R is the derivative of this residual along R by a 7-point central stencil,
exact for the quartic residual up to rounding (Sec. 2.3.3: A = dOmega/dt).

The SCC term of Sec. 2.4.1-2.4.2 is written here with explicit triples: the
singlet X3 = R1^a R2^b - R1^b R2^a becomes the antisymmetric spin-orbital
triples amplitude
  x_IJK^ABC = P(I/JK) P(A/BC) [r^a_I^A r^b_JK^BC - r^b_I^A r^a_JK^BC],
P(I/JK) f(IJK) = f(IJK) - f(JIK) - f(KJI), and the part of
<mu|exp(-T) H exp(T)|HF> linear in X3 is <mu|(Hhat_N X3)_c|HF> with
Hhat = exp(-T1) H exp(T1): the triples terms of the CCSDT singles and doubles
equations, evaluated with the T1-transformed integrals. Those come from the
orbital transformation exp(-T1) a+_I exp(T1) = a+_I - sum_A t_I^A a+_A,
exp(-T1) a_A exp(T1) = a_A + sum_I t_I^A a_I (creators of virtual and
annihilators of occupied orbitals unchanged).
"""
from __future__ import annotations

import numpy as np


def _ein(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


class SpinSystem:
    """Spin-orbital Hamiltonian of the synthetic system (eps[n], L[J][n][n],
    o doubly occupied spatial orbitals, occupied first). Spin orbitals are
    ordered occ-alpha, occ-beta, vir-alpha, vir-beta."""

    def __init__(self, eps, L, o: int):
        eps = np.asarray(eps, dtype=np.float64)
        L = np.asarray(L, dtype=np.float64)
        n = eps.shape[0]
        v = n - o
        self.o, self.v, self.n = o, v, n
        self.no, self.nv = 2 * o, 2 * v
        spatial = np.concatenate([np.arange(o), np.arange(o), o + np.arange(v), o + np.arange(v)])
        spin = np.concatenate([np.zeros(o), np.ones(o), np.zeros(v), np.ones(v)]).astype(int)
        self.spatial, self.spin = spatial, spin
        # chemists' (pq|rs) over spatial orbitals, then <PQ|RS> = (PR|QS)
        g = _ein("Jpq,Jrs->pqrs", L, L)
        same = (spin[:, None] == spin[None, :]).astype(np.float64)
        G = g[np.ix_(spatial, spatial, spatial, spatial)]            # (PQ|RS) in spin orbitals
        G = G * same[:, :, None, None] * same[None, None, :, :]      # spin of P = Q, R = S
        phys = G.transpose(0, 2, 1, 3)                                # <PQ|RS> = (PR|QS)
        self.W = phys - phys.transpose(0, 1, 3, 2)                    # <PQ||RS>
        eps_s = eps[spatial]
        nocc = self.no
        occ_sum = _ein("pkqk->pq", self.W[:, :nocc, :, :nocc])
        self.h = np.diag(eps_s) - occ_sum
        self.f = self.h + occ_sum                                     # = diag(eps)
        self.e_ref = np.trace(self.h[:nocc, :nocc]) + 0.5 * _ein("ijij->", self.W[:nocc, :nocc, :nocc, :nocc])

    # ---------------------------------------------------------------- layout
    def packed_dim(self) -> int:
        ov = self.o * self.v
        return ov + ov * (ov + 1) // 2

    def closed_shell_from_packed(self, x):
        """(t1[a][i], t2[a][i][b][j]) of the packed layout: singles at a*o + i,
        then pair (P, Q), P = a o + i <= Q = b o + j, at ov + Q(Q+1)/2 + P."""
        o, v = self.o, self.v
        ov = o * v
        x = np.asarray(x, dtype=np.float64)
        t1 = x[:ov].reshape(v, o).copy()
        M = np.zeros((ov, ov))
        k = ov
        for Q in range(ov):
            M[:Q + 1, Q] = x[k:k + Q + 1]
            M[Q, :Q + 1] = x[k:k + Q + 1]
            k += Q + 1
        return t1, M.reshape(v, o, v, o)

    def packed_from_closed_shell(self, r1, r2):
        o, v = self.o, self.v
        ov = o * v
        M = r2.reshape(ov, ov)
        out = [r1.reshape(-1)]
        for Q in range(ov):
            out.append(M[:Q + 1, Q])
        return np.concatenate(out)

    def spin_amplitudes(self, x):
        """Spin-orbital t1[I][A] and antisymmetric t2[I][J][A][B] of packed x."""
        o, v = self.o, self.v
        c1, c2 = self.closed_shell_from_packed(x)
        so, sv = self.spin[:self.no], self.spin[self.no:]
        io, av = self.spatial[:self.no], self.spatial[self.no:] - o
        d_ia = (so[:, None] == sv[None, :]).astype(np.float64)       # [I][A]
        t1 = c1[av[None, :], io[:, None]] * d_ia
        # direct[I,J,A,B] = t_ij^ab = c2[a, i, b, j]; exchange = t_ij^ba = c2[b, i, a, j]
        I, J, A, B = np.ix_(io, io, av, av)
        direct = c2[A, I, B, J]
        exch = c2[B, I, A, J]
        d1 = d_ia[:, None, :, None] * d_ia[None, :, None, :]          # s_I = s_A, s_J = s_B
        d2 = d_ia[:, None, None, :] * d_ia[None, :, :, None]          # s_I = s_B, s_J = s_A
        t2 = d1 * direct - d2 * exch
        return t1, t2

    # ------------------------------------------------------------ equations
    def energy_residual_spin(self, t1, t2):
        """(E0, r1[I][A], r2[I][J][A][B]) with r the projections <Phi|Hbar|HF>."""
        no = self.no
        o, v = slice(0, no), slice(no, None)
        W, f = self.W, self.f
        fov, foo, fvv = f[o, v], f[o, o], f[v, v]
        Woooo, Wooov, Woovv = W[o, o, o, o], W[o, o, o, v], W[o, o, v, v]
        Wovvv, Wvovv, Wovov = W[o, v, v, v], W[v, o, v, v], W[o, v, o, v]
        Wovvo, Woovo = W[o, v, v, o], W[o, o, v, o]
        Wvvvv, Wvvvo, Wovoo = W[v, v, v, v], W[v, v, v, o], W[o, v, o, o]

        tt = _ein("ia,jb->ijab", t1, t1)
        tau_t = t2 + 0.5 * (tt - tt.transpose(0, 1, 3, 2))
        tau = t2 + tt - tt.transpose(0, 1, 3, 2)

        E0 = (self.e_ref + _ein("ia,ia->", fov, t1) + 0.25 * _ein("ijab,ijab->", Woovv, t2)
              + 0.5 * _ein("ijab,ia,jb->", Woovv, t1, t1))

        Fae = (fvv - 0.5 * _ein("me,ma->ae", fov, t1) + _ein("mf,mafe->ae", t1, Wovvv)
               - 0.5 * _ein("mnaf,mnef->ae", tau_t, Woovv))
        Fmi = (foo + 0.5 * _ein("ie,me->mi", t1, fov) + _ein("ne,mnie->mi", t1, Wooov)
               + 0.5 * _ein("inef,mnef->mi", tau_t, Woovv))
        Fme = fov + _ein("nf,mnef->me", t1, Woovv)

        x = _ein("je,mnie->mnij", t1, Wooov)
        Wmnij = Woooo + x - x.transpose(0, 1, 3, 2) + 0.25 * _ein("ijef,mnef->mnij", tau, Woovv)
        y = _ein("mb,amef->abef", t1, Wvovv)
        Wabef = Wvvvv - (y - y.transpose(1, 0, 2, 3)) + 0.25 * _ein("mnab,mnef->abef", tau, Woovv)
        Z = 0.5 * t2 + _ein("jf,nb->jnfb", t1, t1)
        Wmbej = (Wovvo + _ein("jf,mbef->mbej", t1, Wovvv) - _ein("nb,mnej->mbej", t1, Woovo)
                 - _ein("jnfb,mnef->mbej", Z, Woovv))

        r1 = (fov + _ein("ie,ae->ia", t1, Fae) - _ein("ma,mi->ia", t1, Fmi)
              + _ein("imae,me->ia", t2, Fme) - _ein("nf,naif->ia", t1, Wovov)
              - 0.5 * _ein("imef,maef->ia", t2, Wovvv) - 0.5 * _ein("mnae,nmei->ia", t2, Woovo))

        def Pab(z):
            return z - z.transpose(0, 1, 3, 2)

        def Pij(z):
            return z - z.transpose(1, 0, 2, 3)

        r2 = Woovv.copy()
        r2 = r2 + Pab(_ein("ijae,be->ijab", t2, Fae - 0.5 * _ein("mb,me->be", t1, Fme)))
        r2 = r2 - Pij(_ein("imab,mj->ijab", t2, Fmi + 0.5 * _ein("je,me->mj", t1, Fme)))
        r2 = r2 + 0.5 * _ein("mnab,mnij->ijab", tau, Wmnij)
        r2 = r2 + 0.5 * _ein("ijef,abef->ijab", tau, Wabef)
        ring = _ein("imae,mbej->ijab", t2, Wmbej) - _ein("ie,ma,mbej->ijab", t1, t1, Wovvo)
        r2 = r2 + Pij(Pab(ring))
        r2 = r2 + Pij(_ein("ie,abej->ijab", t1, Wvvvo))
        r2 = r2 - Pab(_ein("ma,mbij->ijab", t1, Wovoo))
        return E0, r1, r2

    def energy_residual(self, x):
        """(E0, packed closed-shell Omega) at packed closed-shell amplitudes x."""
        t1, t2 = self.spin_amplitudes(x)
        E0, r1, r2 = self.energy_residual_spin(t1, t2)
        return E0, self.closed_shell_residual(r1, r2)

    def closed_shell_residual(self, r1, r2):
        """Packed Omega from the spin-orbital projections: singles from the
        alpha -> alpha block, doubles from the (alpha, beta) -> (alpha, beta)
        block (the determinant coefficients of sum_mu Omega_mu tau_mu |HF>)."""
        o, v = self.o, self.v
        R1 = r1[:o, :v].T                                 # [a][i] = r_{i alpha}^{a alpha}
        blk = r2[:o, o:2 * o, :v, v:2 * v]                # [i][j][a][b] = r_{i a, j b}^{a a, b b}
        R2 = blk.transpose(2, 0, 3, 1)                    # [a][i][b][j]
        return self.packed_from_closed_shell(R1, R2)

    # ----------------------------------------------------------- SCC term
    def dressed(self, t1):
        """(f^, W^): Fock-like one-body part (normal order with respect to HF)
        and antisymmetrised two-body integrals of exp(-T1) H exp(T1)."""
        no, N = self.no, self.no + self.nv
        Lm = np.eye(N)
        Rm = np.eye(N)
        Lm[no:, :no] = -t1.T          # a+_I -> a+_I - sum_A t_I^A a+_A
        Rm[no:, :no] = t1.T           # a_A -> a_A + sum_I t_I^A a_I
        h = Lm @ self.h @ Rm
        W = _ein("aP,bQ,PQRS,Rc,Sd->abcd", Lm, Lm, self.W, Rm, Rm)
        f = h + _ein("pkqk->pq", W[:, :no, :, :no])
        return f, W

    def triples_of(self, Ra, Rb):
        """x_IJK^ABC of X3 = R1^a R2^b - R1^b R2^a (packed closed-shell kets)."""
        r1a, r2a = self.spin_amplitudes(Ra)
        r1b, r2b = self.spin_amplitudes(Rb)
        c = _ein("ia,jkbc->ijkabc", r1a, r2b) - _ein("ia,jkbc->ijkabc", r1b, r2a)

        def p_occ(z):   # P(I/JK)
            return z - z.transpose(1, 0, 2, 3, 4, 5) - z.transpose(2, 1, 0, 3, 4, 5)

        def p_vir(z):   # P(A/BC)
            return z - z.transpose(0, 1, 2, 4, 3, 5) - z.transpose(0, 1, 2, 5, 4, 3)

        return p_vir(p_occ(c))

    def x3_term_spin(self, t1, x3):
        """(s1[I][A], s2[I][J][A][B]): <mu|(Hhat_N X3)_c|HF> for singles and
        doubles, X3 given by its triples amplitude x3[I][J][K][A][B][C]."""
        no = self.no
        o, v = slice(0, no), slice(no, None)
        f, W = self.dressed(t1)
        s1 = 0.25 * _ein("mnef,imnaef->ia", W[o, o, v, v], x3)
        s2 = _ein("me,ijmabe->ijab", f[o, v], x3)
        y = 0.5 * _ein("bmef,ijmaef->ijab", W[v, o, v, v], x3)
        s2 = s2 + y - y.transpose(0, 1, 3, 2)
        z = 0.5 * _ein("mnje,imnabe->ijab", W[o, o, o, v], x3)
        s2 = s2 - (z - z.transpose(1, 0, 2, 3))
        return s1, s2

    def energy_residual_scc(self, x, zeta, Ra, Rb):
        """(E0, packed Omega) with the cluster operator T + zeta X3 (Sec. 2.4.1):
        the CCSD projections plus zeta <mu|(Hhat_N X3)_c|HF> (Sec. 2.4.2)."""
        t1, t2 = self.spin_amplitudes(x)
        E0, r1, r2 = self.energy_residual_spin(t1, t2)
        s1, s2 = self.x3_term_spin(t1, self.triples_of(Ra, Rb))
        return E0, self.closed_shell_residual(r1 + zeta * s1, r2 + zeta * s2)

    def jacobian_right_scc(self, x, R, zeta, Ra, Rb, h: float = 1.0):
        """A R of the SCC residual at fixed (zeta, Ra, Rb), by the exact 7-point
        stencil (the residual is a polynomial of degree <= 6 in t)."""
        x = np.asarray(x, dtype=np.float64)
        R = np.asarray(R, dtype=np.float64)
        w = {1: 45.0, 2: -9.0, 3: 1.0}
        acc = np.zeros_like(x)
        for k, c in w.items():
            acc += c * (self.energy_residual_scc(x + k * h * R, zeta, Ra, Rb)[1]
                        - self.energy_residual_scc(x - k * h * R, zeta, Ra, Rb)[1])
        return acc / (60.0 * h)

    # ------------------------------------------------------- SCC overlap
    def projected_state(self, x, r0, R):
        """Determinant coefficients (c0, c1[I][A], c2[I][J][A][B]) of
        exp(T)(r0 + R)|HF> on HF, singles and doubles (T from packed x,
        without X3): c1 = r1 + r0 t1, c2 = r2 + P(IJ)P(AB) t1 r1 + r0 (t2 + t1^t1)."""
        t1, t2 = self.spin_amplitudes(x)
        r1, r2 = self.spin_amplitudes(R)
        tr = _ein("ia,jb->ijab", t1, r1)
        ptr = tr - tr.transpose(1, 0, 2, 3) - tr.transpose(0, 1, 3, 2) + tr.transpose(1, 0, 3, 2)
        tt = _ein("ia,jb->ijab", t1, t1)
        return r0, r1 + r0 * t1, r2 + ptr + r0 * (t2 + tt - tt.transpose(0, 1, 3, 2))

    def overlap(self, x, ra0, Ra, rb0, Rb):
        """O_ab = <psi_a|P|psi_b> of the natural projection (Sec. 2.4.2): the
        plain sum over HF, singles and doubles determinants (each doubles
        determinant once: 1/4 of the sum over all four-index amplitudes)."""
        a0, a1, a2 = self.projected_state(x, ra0, Ra)
        b0, b1, b2 = self.projected_state(x, rb0, Rb)
        return float(a0 * b0 + np.sum(a1 * b1) + 0.25 * np.sum(a2 * b2))

    def jacobian_right(self, x, R, h: float = 1.0):
        """A R by the exact 7-point central stencil of Omega(x + e R)."""
        x = np.asarray(x, dtype=np.float64)
        R = np.asarray(R, dtype=np.float64)
        w = {1: 45.0, 2: -9.0, 3: 1.0}
        acc = np.zeros_like(x)
        for k, c in w.items():
            acc += c * (self.energy_residual(x + k * h * R)[1] - self.energy_residual(x - k * h * R)[1])
        return acc / (60.0 * h)
