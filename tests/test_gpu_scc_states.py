"""More than two constrained states on the GPU (Sec. 2.2 with K of n states;
X_kl of Sec. 2.4.1 for every pair) against the FP64 oracle at o=5 v=19 J=72.

* The residual with T + sum_kl zeta_kl X_kl for three states, A R with eta.R,
  A^T L and the densities, element by element (FP64 path), and the split
  BF16 path within its error.
* n = 2 through the several-states call equals the two-state call.
* The ground solve with the three-state X3 terms in the split BF16 precision
  with FP64 refinement: the oracle's residual vanishes at the GPU amplitudes.
* O_kl of every pair, natural and state projection over all three states.
"""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle import response as rp
from paper_2403_01007_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

PAIRS = [(0, 1), (0, 2), (1, 2)]


@pytest.fixture(scope="module")
def small():
    from paper_2403_01007_gb300 import binding as B
    w = syn.SMALL
    eps, L = syn.workload_system(w)
    prob = cc.Problem(eps, L, w.o)
    t = syn.random_vectors(w.o, w.v, 1, syn.seed_of(w.config, 51), scale=0.05)[0]
    R3 = syn.random_vectors(w.o, w.v, 3, syn.seed_of(w.config, 61), normalise=True)
    zeta = np.array([0.31, -0.17, 0.12])
    scct = [(float(z), torch.tensor(R3[k]), torch.tensor(R3[l])) for z, (k, l) in zip(zeta, PAIRS)]
    return B, w, eps, L, prob, t, R3, zeta, scct


def test_three_states_fp64_against_oracle(small):
    B, w, eps, L, prob, t, R3, zeta, scct = small
    Rt = syn.random_vectors(w.o, w.v, 2, syn.seed_of(w.config, 62), normalise=True)
    ctx = B.Context(w.o, w.v, w.J, eps, L, precision="fp64")
    e, om = ctx.residual_states(t, zeta, R3)
    E0, Om = rp.residual(prob, t, scc=scct)
    Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    ref = Om.numpy()
    assert abs(e - (float(E0) - Ehf)) < 1e-11 * abs(e)
    assert np.abs(om - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(om - rp.residual(prob, t)[1].numpy()).max() > 1e-4 * np.abs(ref).max()
    s, eta = ctx.jacobian_right(Rt, with_eta=True)
    sl = ctx.jacobian_left(Rt)
    for k in range(2):
        r = rp.jacobian_right(prob, t, Rt[k], scc=scct).numpy()
        assert np.abs(s[k] - r).max() < 1e-12 * np.abs(r).max()
        assert abs(eta[k] - float(rp.eta(prob, t, scc=scct) @ torch.tensor(Rt[k]))) < 1e-11
        r = rp.jacobian_left(prob, t, Rt[k], scc=scct).numpy()
        assert np.abs(sl[k] - r).max() < 1e-12 * np.abs(r).max()
    D1, G = ctx.densities(0.5, Rt[0], -0.2, Rt[1])
    D1r, Gr = rp.densities(prob, t, 0.5, Rt[0], -0.2, Rt[1], scc=scct)
    assert np.abs(D1 - D1r.numpy()).max() < 1e-10
    assert np.abs(G - Gr.numpy()).max() < 1e-10
    # n = 2 equals the two-state call
    e2, om2 = ctx.residual_states(t, [0.4], R3[:2])
    e2p, om2p = ctx.residual(t, scc=(0.4, R3[0], R3[1]))
    assert abs(e2 - e2p) < 1e-12 * abs(e2)
    assert np.abs(om2 - om2p).max() < 1e-13 * np.abs(om2p).max()
    ctx.close()


def test_three_states_split_bf16_against_oracle(small):
    B, w, eps, L, prob, t, R3, zeta, scct = small
    ctx = B.Context(w.o, w.v, w.J, eps, L, precision="bf16x3")
    _, om = ctx.residual_states(t, zeta, R3)
    ref = rp.residual(prob, t, scc=scct)[1].numpy()
    assert np.abs(om - ref).max() < 2e-4 * np.abs(ref).max()
    Rt = syn.random_vectors(w.o, w.v, 1, syn.seed_of(w.config, 63), normalise=True)
    s = ctx.jacobian_right(Rt)
    r = rp.jacobian_right(prob, t, Rt[0], scc=scct).numpy()
    assert np.abs(s[0] - r).max() < 2e-4 * np.abs(r).max()
    # refined ground solve with the three-state terms: the oracle's residual vanishes
    z = 0.1 * zeta
    e, tg, _ = ctx.solve_ground_states(z, R3, tol=1e-9, maxit=400, refine_tol=1e-5)
    sccg = [(0.1 * zz, x, y) for zz, x, y in scct]
    E0, Om = rp.residual(prob, tg, scc=sccg)
    Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    assert np.linalg.norm(Om.numpy()) < 1e-8
    assert abs(e - (float(E0) - Ehf)) < 1e-9
    ctx.close()


def test_overlaps_of_every_pair_against_oracle(small):
    """O_kl of the three pairs at the fixed (CCSD) state, natural projection
    and state projection over all three states (Sec. 2.2, 2.4.1), against the
    oracle; with two states the pair calls."""
    from oracle import scc as sc
    B, w, eps, L, prob, t, R3, zeta, scct = small
    ctx = B.Context(w.o, w.v, w.J, eps, L, precision="fp64")
    ctx.residual(t)
    r0 = np.array([0.3, -0.2, 0.1])
    states = [(float(r0[k]), torch.tensor(R3[k])) for k in range(3)]
    for proj in ("natural", "state"):
        got = ctx.overlaps(r0, R3, proj)
        ref = sc.overlaps(torch.tensor(t), states, w.o, w.v, proj)
        for kl, val in ref.items():
            assert abs(got[kl] - float(val)) < 1e-11 * max(1.0, abs(float(val))), (proj, kl)
    two = ctx.overlaps(r0[:2], R3[:2], "state")
    assert abs(two[(0, 1)] - ctx.overlap_states(r0[0], R3[0], r0[1], R3[1])) < 1e-12
    ctx.close()
