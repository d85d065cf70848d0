"""Brute-force determinant-space engine (test infrastructure, FP64, CPU).

This file is part of the oracle. Only tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does.

It evaluates every quantity of the closed-shell (S)CCSD hot path from its
defining expression, with explicit second quantisation over all N-electron,
S_z = 0 Slater determinants of n spatial orbitals. Nothing is spin-adapted or
simplified: operators are sparse matrices, exp(T) is its (terminating) power
series, projections are least-squares solves onto the excitation kets. It is
meant for tiny systems (o <= 3, v <= 5) and serves as the authority against
which the closed-shell oracle is pinned.

Definitions used (paper Sec. 2.1, 2.2, 2.3.2, 2.4):

* H = sum_pq h_pq E_pq + 1/2 sum_pqrs g_pqrs e_pqrs,  e_pqrs = E_pq E_rs - d_qr E_ps
  (the density expansion of Sec. 2.3.2; the nuclear term is dropped).
* cluster operator T = sum_ai t_ai E_ai + 1/2 sum_{ai,bj} t_aibj E_ai E_bj
  (+ zeta X3 for SCC, Sec. 2.4.1), Hbar = exp(-T) H exp(T) (Sec. 2.1).
* excitation kets |mu> = tau_mu |HF>: tau_ai = E_ai, tau_aibj = E_ai E_bj for
  ai < bj and tau_aiai = 1/2 E_ai E_ai, so that T = sum_mu t_mu tau_mu with
  the packed amplitudes t_mu.
* bras <mu~| are the biorthonormal partners of the kets inside the span of
  {|HF>, |mu>}: Omega_mu = <mu~|Hbar|HF> is the coefficient of |mu> in the
  expansion of the singles-and-doubles part of Hbar|HF> (Sec. 2.1).

Packed layout (shared convention of the whole project, stated in the C
header too): singles index P = a*o + i; doubles over unique compound pairs
P <= Q stored at ov + Q*(Q+1)/2 + P.
"""
from __future__ import annotations

from itertools import combinations

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# packed layout helpers (oracle-private copies)
# --------------------------------------------------------------------------

def packed_pairs(ov: int):
    """List of (P, Q) with P <= Q in packed order.
    The doubles of Sec. 2.1, each pair once."""
    out = []
    for Q in range(ov):
        for P in range(Q + 1):
            out.append((P, Q))
    return out


class Space:
    """All N-electron, S_z = 0 determinants of n spatial orbitals."""

    def __init__(self, o: int, v: int):
        self.o, self.v, self.n = o, v, o + v
        n = self.n
        self.strings = [sum(1 << k for k in c) for c in combinations(range(n), o)]
        self.str_index = {s: k for k, s in enumerate(self.strings)}
        ns = len(self.strings)
        self.dim = ns * ns
        hf_str = (1 << o) - 1
        self.hf = self.str_index[hf_str] * ns + self.str_index[hf_str]
        vir_mask = ((1 << n) - 1) ^ hf_str
        lev = np.array([bin(s & vir_mask).count("1") for s in self.strings])
        self.level = (lev[:, None] + lev[None, :]).reshape(-1)
        self._E = {}
        self._build_excitation_kets()

    # ---- one-body operators -------------------------------------------------
    def _string_excite(self, s: int, p: int, q: int):
        """a_p^+ a_q on an occupation string; returns (sign, new) or None."""
        if not (s >> q) & 1:
            return None
        sign = -1 if bin(s & ((1 << q) - 1)).count("1") % 2 else 1
        s2 = s ^ (1 << q)
        if (s2 >> p) & 1:
            return None
        if bin(s2 & ((1 << p) - 1)).count("1") % 2:
            sign = -sign
        return sign, s2 | (1 << p)

    def E(self, p: int, q: int) -> sp.csr_matrix:
        """Singlet excitation operator E_pq = a+_pa a_qa + a+_pb a_qb.
        The operators of the Hamiltonian of Sec. 2.3.2 and of the excitations of Sec. 2.1."""
        key = (p, q)
        if key in self._E:
            return self._E[key]
        ns = len(self.strings)
        rows, cols, vals = [], [], []
        for ka, sa in enumerate(self.strings):
            r = self._string_excite(sa, p, q)
            if r is None:
                continue
            sign, sa2 = r
            ka2 = self.str_index[sa2]
            for kb in range(ns):
                rows.append(ka2 * ns + kb)
                cols.append(ka * ns + kb)
                vals.append(sign)
        for kb, sb in enumerate(self.strings):
            r = self._string_excite(sb, p, q)
            if r is None:
                continue
            sign, sb2 = r
            kb2 = self.str_index[sb2]
            for ka in range(ns):
                rows.append(ka * ns + kb2)
                cols.append(ka * ns + kb)
                vals.append(sign)
        M = sp.csr_matrix((np.array(vals, dtype=np.float64), (rows, cols)),
                          shape=(self.dim, self.dim))
        M.sum_duplicates()
        self._E[key] = M
        return M

    # ---- excitation manifold ---------------------------------------------
    def _build_excitation_kets(self):
        o, v = self.o, self.v
        ov = o * v
        hf = np.zeros(self.dim)
        hf[self.hf] = 1.0
        self.hf_vec = hf
        singles = []
        for a in range(v):
            for i in range(o):
                singles.append(self.E(o + a, i) @ hf)
        self.single_kets = singles
        doubles = []
        for (P, Q) in packed_pairs(ov):
            a, i = divmod(P, o)
            b, j = divmod(Q, o)
            k = self.E(o + a, i) @ (self.E(o + b, j) @ hf)
            if P == Q:
                k = 0.5 * k
            doubles.append(k)
        kets = [hf] + singles + doubles
        self.kets = np.array(kets).T            # dim x (1 + packed)
        self.rows = np.where(self.level <= 2)[0]  # determinants inside span
        B = self.kets[self.rows, :]
        # dual (biorthonormal) bras restricted to the <=2 rows
        self.B = B
        self.Bpinv = np.linalg.pinv(B)
        if np.linalg.matrix_rank(B) != B.shape[1]:
            raise RuntimeError("excitation kets are not linearly independent")

    @property
    def packed_dim(self):
        """Size of the packed singles and doubles manifold (Sec. 2.1)."""
        ov = self.o * self.v
        return ov + ov * (ov + 1) // 2

    def ket(self, c0: float, c: np.ndarray) -> np.ndarray:
        """Determinant vector of c0 |HF> + sum_mu c_mu |mu>.
        Kets |mu> = tau_mu |HF> of Sec. 2.1."""
        return self.kets @ np.concatenate([[c0], c])

    def bra(self, c0: float, c: np.ndarray) -> np.ndarray:
        """Determinant vector of the bra c0 <HF| + sum_mu c_mu <mu~|.
        Bras <mu~| biorthonormal to the kets (Sec. 2.1)."""
        x = np.zeros(self.dim)
        x[self.rows] = np.concatenate([[c0], c]) @ self.Bpinv
        return x

    def project(self, psi: np.ndarray, check: bool = True) -> np.ndarray:
        """Coefficients (c0, c_mu) of the <= doubles part of psi in the kets.
        The natural projection onto HF and the singles and doubles (Sec. 2.4.1)."""
        y = psi[self.rows]
        c = self.Bpinv @ y
        if check:
            res = np.linalg.norm(self.B @ c - y)
            if res > 1e-9 * max(1.0, np.linalg.norm(y)):
                raise RuntimeError(f"projection left a residual {res:.3e}")
        return c

    # ---- operators built from amplitudes ----------------------------------
    def op_singles(self, r1: np.ndarray) -> sp.csr_matrix:
        """sum_ai r_ai E_ai, r1 indexed a*o + i.
        T1 of Sec. 2.1."""
        o, v = self.o, self.v
        M = sp.csr_matrix((self.dim, self.dim))
        for a in range(v):
            for i in range(o):
                if r1[a * o + i] != 0.0:
                    M = M + r1[a * o + i] * self.E(o + a, i)
        return M

    def op_doubles(self, r2: np.ndarray) -> sp.csr_matrix:
        """sum over packed mu of r_mu tau_mu (1/2 on the diagonal pairs).
        T2 of Sec. 2.1."""
        o, v = self.o, self.v
        ov = o * v
        M = sp.csr_matrix((self.dim, self.dim))
        for k, (P, Q) in enumerate(packed_pairs(ov)):
            if r2[k] == 0.0:
                continue
            a, i = divmod(P, o)
            b, j = divmod(Q, o)
            f = 0.5 if P == Q else 1.0
            M = M + (f * r2[k]) * (self.E(o + a, i) @ self.E(o + b, j))
        return M

    def op_cluster(self, t: np.ndarray) -> sp.csr_matrix:
        """The cluster operator T = sum_mu t_mu tau_mu of Sec. 2.1 (singles and doubles) as a sparse
        matrix."""
        ov = self.o * self.v
        return self.op_singles(t[:ov]) + self.op_doubles(t[ov:])

    def hamiltonian(self, h: np.ndarray, g: np.ndarray) -> sp.csr_matrix:
        """H = sum h_pq E_pq + 1/2 sum g_pqrs (E_pq E_rs - d_qr E_ps).
        Sec. 2.3.2."""
        n = self.n
        H = sp.csr_matrix((self.dim, self.dim))
        for p in range(n):
            for q in range(n):
                Gpq = sp.csr_matrix((self.dim, self.dim))
                for r in range(n):
                    for s in range(n):
                        if g[p, q, r, s] != 0.0:
                            Gpq = Gpq + g[p, q, r, s] * self.E(r, s)
                H = H + h[p, q] * self.E(p, q) + 0.5 * (self.E(p, q) @ Gpq)
                # - 1/2 sum_r g_prrq E_pq
                H = H - 0.5 * np.einsum("rr->", g[p, :, :, q]) * self.E(p, q)
        return H.tocsr()


def expm_apply(T: sp.spmatrix, x: np.ndarray, sign: float = 1.0) -> np.ndarray:
    """exp(sign*T) x by the power series; T is nilpotent on this space.
    exp(T) of Sec. 2.1 applied to a determinant vector."""
    out = x.copy()
    term = x.copy()
    for k in range(1, 64):
        term = (sign / k) * (T @ term)
        nrm = np.linalg.norm(term)
        out += term
        if nrm == 0.0 or nrm < 1e-300:
            break
    return out


class System:
    """A Hamiltonian on a Space plus the brute-force (S)CCSD quantities."""

    def __init__(self, space: Space, h: np.ndarray, g: np.ndarray):
        self.S = space
        self.h, self.g = h, g
        self.H = space.hamiltonian(h, g)

    # Hbar acting on a vector: exp(-T) H exp(T) x
    def hbar_apply(self, T, x):
        """Hbar x = exp(-T) H exp(T) x, the similarity-transformed Hamiltonian of Sec. 2.1."""
        return expm_apply(T, self.H @ expm_apply(T, x, +1.0), -1.0)

    def omega(self, t: np.ndarray, extra=None):
        """(E0, Omega) with T = op_cluster(t) (+ extra operator, e.g. zeta X3).
        E0 = <HF|Hbar|HF> and Omega_mu = <mu~|Hbar|HF> of Sec. 2.1; with zeta X3 the SCC cluster
        operator of Sec. 2.4.1."""
        T = self.S.op_cluster(t)
        if extra is not None:
            T = T + extra
        c = self.S.project(self.hbar_apply(T, self.S.hf_vec))
        return c[0], c[1:]

    def jacobian(self, t: np.ndarray, extra=None) -> np.ndarray:
        """A_mu,nu = <mu~|[Hbar, tau_nu]|HF>, explicit (Sec. 2.3.3)."""
        T = self.S.op_cluster(t)
        if extra is not None:
            T = T + extra
        hbar_hf = self.hbar_apply(T, self.S.hf_vec)
        m = self.S.packed_dim
        A = np.zeros((m, m))
        eta = np.zeros(m)
        for nu in range(m):
            e = np.zeros(m)
            e[nu] = 1.0
            tau = self.S.op_cluster(e)
            c = self.S.project(self.hbar_apply(T, tau @ self.S.hf_vec) - tau @ hbar_hf)
            A[:, nu] = c[1:]
            eta[nu] = c[0]
        return A, eta

    def hbar_matrix(self, t: np.ndarray, extra=None) -> np.ndarray:
        """<mu~|Hbar|nu> over the full manifold incl. HF (Sec. 2.1)."""
        T = self.S.op_cluster(t)
        if extra is not None:
            T = T + extra
        m = self.S.packed_dim + 1
        M = np.zeros((m, m))
        for nu in range(m):
            M[:, nu] = self.S.project(self.hbar_apply(T, self.S.kets[:, nu]))
        return M

    def densities(self, t, l0, l, r0, r, extra=None):
        """d_pq and d_pqrs of Sec. 2.3.2 for bra (l0, l) and ket (r0, r)."""
        S = self.S
        T = S.op_cluster(t)
        if extra is not None:
            T = T + extra
        ket = expm_apply(T, S.ket(r0, r), +1.0)
        bra = expm_apply(T.T.tocsr(), S.bra(l0, l), -1.0)   # (<L| exp(-T))^T
        n = S.n
        d1 = np.zeros((n, n))
        Ek = {}
        for p in range(n):
            for q in range(n):
                Ek[p, q] = S.E(p, q) @ ket
                d1[p, q] = bra @ Ek[p, q]
        d2 = np.zeros((n, n, n, n))
        braE = {}
        for p in range(n):
            for q in range(n):
                braE[p, q] = S.E(p, q).T @ bra
        for p in range(n):
            for q in range(n):
                for r in range(n):
                    for s in range(n):
                        val = braE[p, q] @ Ek[r, s]
                        if q == r:
                            val -= d1[p, s]
                        d2[p, q, r, s] = val
        return d1, d2

    def overlap(self, t, ra0, ra, rb0, rb):
        """SCC orthogonality O_ab = <psi_a|P|psi_b> with P onto HF+S+D
        determinants and psi = exp(T)(R0|HF> + R), T without X3 (Sec. 2.4.2)."""
        S = self.S
        T = S.op_cluster(t)
        pa = expm_apply(T, S.ket(ra0, ra), +1.0)
        pb = expm_apply(T, S.ket(rb0, rb), +1.0)
        rows = S.rows
        return float(pa[rows] @ pb[rows])

    def overlap_states(self, t, ra0, ra, rb0, rb):
        """SCC orthogonality with the state projection (Sec. 2.4.1):
        O_ab = sum_kl <psi_a|R_k> (S^-1)_kl <R_l|psi_b>, S_kl = <R_k|R_l>, for
        K = {a, b}, with |R_k> = R0_k|HF> + R_k and psi = exp(T)|R>, T without X3;
        every inner product over full determinant vectors."""
        S = self.S
        T = S.op_cluster(t)
        ka, kb = S.ket(ra0, ra), S.ket(rb0, rb)
        pa, pb = expm_apply(T, ka, +1.0), expm_apply(T, kb, +1.0)
        Smat = np.array([[ka @ ka, ka @ kb], [kb @ ka, kb @ kb]])
        m = np.array([pa @ ka, pa @ kb])
        nvec = np.array([ka @ pb, kb @ pb])
        return float(m @ np.linalg.solve(Smat, nvec))


def overlaps_states(system, t, states):
    """O_kl of the state projection over all of K = {(R0_k, R_k)} (Sec. 2.4.1)
    for every pair k < l, over full determinant vectors: O_kl = sum_mn
    <psi_k|R_m> (S^-1)_mn <R_n|psi_l>, psi = exp(T)|R>, T without X."""
    S = system.S
    T = S.op_cluster(t)
    kets = [S.ket(r0, r) for r0, r in states]
    psis = [expm_apply(T, k, +1.0) for k in kets]
    K = len(states)
    Smat = np.array([[kets[m] @ kets[n] for n in range(K)] for m in range(K)])
    M = np.array([[psis[k] @ kets[m] for m in range(K)] for k in range(K)])
    W = np.linalg.solve(Smat, M.T)
    return {(k, l): float(M[k] @ W[:, l]) for k in range(K) for l in range(k + 1, K)}


def x3_operator(space: Space, ra: np.ndarray, rb: np.ndarray) -> sp.csr_matrix:
    """X3 = R1^a R2^b - R1^b R2^a (Sec. 2.4.1) as a determinant-space matrix."""
    ov = space.o * space.v
    R1a, R2a = space.op_singles(ra[:ov]), space.op_doubles(ra[ov:])
    R1b, R2b = space.op_singles(rb[:ov]), space.op_doubles(rb[ov:])
    return (R1a @ R2b - R1b @ R2a).tocsr()


def full_g(L: np.ndarray) -> np.ndarray:
    """g_pqrs = sum_J L^J_pq L^J_rs.
    The two-electron integrals of the Hamiltonian of Sec. 2.3.2, from their Cholesky vectors."""
    return np.einsum("Jpq,Jrs->pqrs", L, L)


def synthetic_h(eps: np.ndarray, g: np.ndarray, o: int) -> np.ndarray:
    """One-electron integrals that make F = diag(eps) exactly:
    h_pq = eps_p d_pq - sum_k (2 g_pqkk - g_pkkq) (canonical HF reference).
    Canonical Hartree-Fock reference for the Hamiltonian of Sec. 2.3.2."""
    h = np.diag(eps).astype(np.float64)
    for k in range(o):
        h -= 2.0 * g[:, :, k, k] - g[:, k, k, :]
    return h
