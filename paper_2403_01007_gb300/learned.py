"""Learned initial guess and preconditioner for the ground-state solver.

The plain solver generates the data: converged amplitudes of seeded synthetic
systems. A per-amplitude MLP (3 hidden layers of 256, BF16 weights, FP32
accumulation) is trained on the GPU with the library's forward, backward and
Adam kernels to map MP2-level features of each doubles amplitude to its
converged value and to the dressed denominator D' (the Jacobian diagonal seen
through the intermediates). The solver then starts from the proposed
amplitudes and uses the proposed denominators as its update preconditioner;
when the proposal starts from a larger residual than the MP2 first iterate,
or does not converge, the plain MP2 guess with the orbital-energy
denominators is used instead. The converged result is the plain solver's in
every case. (An extension of the method; the paper has no learned part.)
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import binding as B
from . import synthetic as syn

N_FEATURES, N_TARGETS = 10, 2
LEARN_CONFIG = 5


def system(o, v, instance, sd=0.03):
    J = 3 * (o + v)
    eps, L = syn.system(o, v, J, sd, syn.seed_of(LEARN_CONFIG, instance))
    return o, v, J, eps, L


def generate(instances, samples_per_instance=20000, tol=1e-8, device="cuda:0", seed=0):
    """Training rows from the plain solver: (X [S][10], Y [S][2]) on the device."""
    g = torch.Generator(device=device).manual_seed(seed)
    Xs, Ys = [], []
    for (o, v, J, eps, L) in instances:
        ctx = B.Context(o, v, J, eps, L, precision="bf16")
        _, t, _ = ctx.solve_ground(tol=tol, maxit=1000, refine_tol=1e-5)
        n = o * o * v * v
        X = torch.empty((n, N_FEATURES), dtype=torch.float32, device=device)
        Y = torch.empty((n, N_TARGETS), dtype=torch.float32, device=device)
        sc = ctx.learned_features(X)
        ctx.learned_targets(t, sc[0], Y)
        k = min(samples_per_instance, n)
        idx = torch.randperm(n, generator=g, device=device)[:k]
        Xs.append(X[idx])
        Ys.append(Y[idx])
        ctx.close()
    return torch.cat(Xs).contiguous(), torch.cat(Ys).contiguous()


def train(net, X, Y, epochs=20, batch=4096, lr=1e-3, seed=0):
    """Minibatch Adam on the device; returns the loss history per epoch."""
    g = torch.Generator(device=X.device).manual_seed(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(X.shape[0], generator=g, device=X.device)
        tot, nb = 0.0, 0
        for s in range(0, X.shape[0] - batch + 1, batch):
            idx = perm[s:s + batch]
            tot += net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr)
            nb += 1
        hist.append(tot / max(nb, 1))
    return hist


def solve_with(ctx, net=None, tol=1e-8, maxit=1000):
    """Ground state from the network's proposal (or the plain method when net is
    None or the proposal starts worse); returns (e_corr, iterations, seconds, used_net)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    used = False
    if net is not None:
        tg, D = ctx.learned_guess(net)
        # compare the starting residuals of the proposal and of the MP2 first iterate
        zero = np.zeros(ctx.dim)
        _, om0 = ctx.residual(zero)
        r_plain = np.linalg.norm(om0)          # |Omega(0)| ~ residual before the MP2 step
        _, omg = ctx.residual(tg)
        if np.all(np.isfinite(D)) and np.all(D > 0) and np.linalg.norm(omg) < r_plain:
            ctx.set_preconditioner(D)
            try:
                e, _, it = ctx.solve_ground(t0=tg, tol=tol, maxit=maxit, refine_tol=1e-5)
                used = True
            except B.SccsdError:
                used = False
            ctx.set_preconditioner(None)
    if not used:
        e, _, it = ctx.solve_ground(tol=tol, maxit=maxit, refine_tol=1e-5)
    torch.cuda.synchronize()
    return e, it, time.perf_counter() - t0, used


def evaluate(net, instances, tol=1e-8):
    """Per instance: plain and learned iterations, seconds and energies."""
    rows = []
    for (o, v, J, eps, L) in instances:
        ctx = B.Context(o, v, J, eps, L, precision="bf16")
        e0, it0, s0, _ = solve_with(ctx, None, tol)
        e1, it1, s1, used = solve_with(ctx, net, tol)
        rows.append({"o": o, "v": v, "plain_iters": it0, "plain_s": s0, "learned_iters": it1,
                     "learned_s": s1, "used_net": used, "de": e1 - e0})
        ctx.close()
    return rows
