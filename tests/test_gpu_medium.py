"""The o=10 v=90 J=300 workload on the GPU against the FP64 oracle.

* A R and A^T L of the FP64 path element by element (Sec. 2.1, 2.3.3), two
  vectors each, at amplitudes of MP2 size.
* The ground state and the four lowest right and left roots solved in the
  split BF16 precision with FP64 refinement: the oracle's own residual at the
  GPU amplitudes vanishes to the solve tolerance and gives the GPU's E_corr;
  the oracle's A R - omega R and L^T A - omega L^T vanish for every GPU root
  (the oracle's solvers themselves would take minutes at this size).
* The transition densities d_pq and Gamma^J_pq between the left vector of
  root 0 and the right vector of root 1 (Sec. 2.3.2) to 1e-7 max-abs.
"""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle import response as rp
from paper_2403_01007_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def medium():
    from paper_2403_01007_gb300 import binding as B
    w = syn.MEDIUM
    eps, L = syn.workload_system(w)
    prob = cc.Problem(eps, L, w.o)
    return B, w, eps, L, prob


def test_fp64_transforms_medium_against_oracle(medium):
    B, w, eps, L, prob = medium
    t = syn.random_vectors(w.o, w.v, 1, syn.seed_of(w.config, 50), scale=1e-3)[0]
    R = syn.random_vectors(w.o, w.v, 2, syn.seed_of(w.config, 60), normalise=True)
    Lb = syn.random_vectors(w.o, w.v, 2, syn.seed_of(w.config, 70), normalise=True)
    ctx = B.Context(w.o, w.v, w.J, eps, L, precision="fp64")
    e, om = ctx.residual(t, omega=np.empty(ctx.dim))
    E0, Om = rp.residual(prob, t)
    Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    assert abs(e - (float(E0) - Ehf)) < 1e-11 * abs(e)
    assert np.abs(om - Om.numpy()).max() < 1e-12 * np.abs(Om.numpy()).max()
    sr = ctx.jacobian_right(R)
    sl = ctx.jacobian_left(Lb)
    for k in range(2):
        ref = rp.jacobian_right(prob, t, R[k]).numpy()
        assert np.abs(sr[k] - ref).max() < 1e-12 * np.abs(ref).max()
        ref = rp.jacobian_left(prob, t, Lb[k]).numpy()
        assert np.abs(sl[k] - ref).max() < 1e-12 * np.abs(ref).max()
    ctx.close()


def test_refined_solves_medium_satisfy_oracle_equations(medium):
    B, w, eps, L, prob = medium
    ctx = B.Context(w.o, w.v, w.J, eps, L, precision="bf16x3")
    e, t, _ = ctx.solve_ground(tol=1e-8, maxit=400, refine_tol=1e-5)
    E0, Om = rp.residual(prob, t)
    Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    assert abs(e - (float(E0) - Ehf)) < 1e-8
    assert float(np.linalg.norm(Om.numpy())) < 1e-7
    wR, VR, _ = ctx.solve_states(4, "right", tol=1e-7, maxit=600, refine_tol=1e-4)
    wL, VL, _ = ctx.solve_states(4, "left", tol=1e-7, maxit=600, refine_tol=1e-4)
    assert np.abs(wR - wL).max() < 1e-8
    for k in range(4):
        r = rp.jacobian_right(prob, t, VR[k]).numpy() - wR[k] * VR[k]
        assert np.linalg.norm(r) < 1e-6, (k, np.linalg.norm(r))
        l = rp.jacobian_left(prob, t, VL[k]).numpy() - wL[k] * VL[k]
        assert np.linalg.norm(l) < 1e-6, (k, np.linalg.norm(l))
    # transition densities <L_0| ... |R_1> in FP64 at the converged state
    ctx.set_precision("fp64")
    ctx.residual(t)
    VLn = ctx.normalize_left(VR[:2].copy(), VL[:2].copy())
    D1, G = ctx.densities(0.0, np.ascontiguousarray(VLn[0]), 0.0, np.ascontiguousarray(VR[1]))
    d1, g = rp.densities(prob, t, 0.0, VLn[0], 0.0, VR[1])
    assert np.abs(D1 - d1.numpy()).max() < 1e-7
    assert np.abs(G - g.numpy()).max() < 1e-7
    ctx.close()
