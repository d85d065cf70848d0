"""Iterative solvers of the FP64 oracle (test infrastructure).

This file is part of the oracle. Only tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does.

* ground_state: Omega(t) = 0 (Sec. 2.1) by the orbital-energy-preconditioned
  fixed point t <- t - Omega/D with DIIS extrapolation (Pulay), the standard
  way CC amplitude equations are solved; D_ai = eps_a - eps_i and
  D_aibj = eps_a + eps_b - eps_i - eps_j.
* eom_right / eom_left: lowest roots of A R = omega R, L^T A = omega L^T
  (Sec. 2.1, block form of the EOM matrix) by the Davidson method
  (Davidson 1975, cited in Sec. 2.3.3) with the same diagonal preconditioner.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ccsd as cc
from . import response as rp


def denominators(prob) -> np.ndarray:
    """Orbital-energy denominators D_ai = e_a - e_i and D_ai + D_bj in the packed layout. These are
    the standard Jacobi preconditioner; the paper does not specify one."""
    o, v = prob.o, prob.v
    e = prob.eps.numpy()
    eo, ev = e[:o], e[o:]
    d1 = (ev[:, None] - eo[None, :]).reshape(-1)          # [a*o + i]
    ov = o * v
    Q, P = np.tril_indices(ov)
    return np.concatenate([d1, d1[P] + d1[Q]])


def ground_state(prob, tol=1e-10, maxit=200, scc=None, x0=None, diis=8):
    """Converge Omega(t) = 0; returns (t, E0, iterations).
    Solves Omega(t) = 0 of Sec. 2.1 by Jacobi steps with DIIS, a standard method the paper does not
    specify."""
    D = denominators(prob)
    x = np.zeros(prob.dim) if x0 is None else np.array(x0, dtype=np.float64)
    xs, rs = [], []
    for it in range(1, maxit + 1):
        E0, Om = rp.residual(prob, x, scc=scc)
        Om = Om.numpy()
        nrm = np.linalg.norm(Om)
        if nrm < tol:
            return x, float(E0), it
        xn = x - Om / D
        xs.append(xn)
        rs.append(xn - x)
        if len(xs) > diis:
            xs.pop(0)
            rs.pop(0)
        if len(xs) >= 2:
            m = len(xs)
            B = -np.ones((m + 1, m + 1))
            B[m, m] = 0.0
            for p in range(m):
                for q in range(m):
                    B[p, q] = rs[p] @ rs[q]
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            try:
                c = np.linalg.solve(B, rhs)[:m]
                xn = sum(c[k] * xs[k] for k in range(m))
            except np.linalg.LinAlgError:
                pass
        x = xn
    raise RuntimeError(f"ground state did not converge: |Omega| = {nrm:.3e}")


def jacobian_matrix(prob, x, scc=None):
    """Explicit A (columns A e_nu) for small systems.
    A of Sec. 2.3.3."""
    f = lambda y: rp.jacobian_right(prob, x, y, scc=scc)
    return torch.func.vmap(f)(torch.eye(prob.dim, dtype=torch.float64)).T.numpy()


def eom_dense(prob, x, nroots, side="right", scc=None):
    """Lowest-Re roots from a dense eigendecomposition of the explicit
    Jacobian (small systems; same conventions as eom).
    The EOM eigenproblem of Sec. 2.1."""
    A = jacobian_matrix(prob, x, scc=scc)
    w, V = np.linalg.eig(A if side == "right" else A.T)
    order = np.argsort(w.real)[:nroots]
    w, V = w[order], V[:, order]
    if np.max(np.abs(w.imag)) > 1e-10:
        raise RuntimeError("complex EOM roots")
    X = V.real.T
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    return w.real, X


def eom(prob, x, nroots, side="right", tol=1e-8, maxit=200, scc=None,
        max_space=None, seed_vectors=None):
    """Lowest-Re roots of the EOM Jacobian; returns (omega[nroots], V[nroots][dim]).
    The EOM eigenproblem of Sec. 2.1, by Davidson (the method Sec. 2.3.3 names)."""
    D = denominators(prob)
    dim = prob.dim
    op = (lambda r: rp.jacobian_right(prob, x, r, scc=scc).numpy()) if side == "right" \
        else (lambda l: rp.jacobian_left(prob, x, l, scc=scc).numpy())
    max_space = max_space or max(8 * nroots, 40)
    if seed_vectors is None:
        order = np.argsort(D)[:max(2 * nroots, nroots + 2)]
        V = np.zeros((len(order), dim))
        for k, idx in enumerate(order):
            V[k, idx] = 1.0
    else:
        V = np.array(seed_vectors, dtype=np.float64)
    V, _ = np.linalg.qr(V.T)
    V = V.T
    AV = np.array([op(v) for v in V])
    for it in range(maxit):
        Hs = V @ AV.T                      # Hs[p,q] = v_p . (A v_q)
        w, Y = np.linalg.eig(Hs)
        order = np.argsort(w.real)[:nroots]
        w, Y = w[order], Y[:, order]
        if np.max(np.abs(w.imag)) > 1e-8:
            raise RuntimeError("complex Davidson roots")
        w, Y = w.real, Y.real
        X = Y.T @ V
        AX = Y.T @ AV
        Rres = AX - w[:, None] * X
        norms = np.linalg.norm(Rres, axis=1) / np.linalg.norm(X, axis=1)
        if np.all(norms < tol):
            X /= np.linalg.norm(X, axis=1, keepdims=True)
            return w, X
        new = []
        for k in range(nroots):
            if norms[k] >= tol:
                den = w[k] - D
                den[np.abs(den) < 1e-6] = 1e-6
                new.append(Rres[k] / den)
        if V.shape[0] + len(new) > max_space:
            # restart from the Ritz vectors
            Q, _ = np.linalg.qr(X.T)
            V = Q.T
            AV = np.array([op(v) for v in V])
        for nv in new:
            for _ in range(2):
                nv = nv - V.T @ (V @ nv)
            nn = np.linalg.norm(nv)
            if nn > 1e-10:
                nv = nv / nn
                V = np.vstack([V, nv])
                AV = np.vstack([AV, op(nv)])
    raise RuntimeError("Davidson did not converge")
