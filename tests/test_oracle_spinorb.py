"""The closed-shell oracle against an independent spin-orbital CCSD oracle.

oracle/ccsd.py (spin-adapted, T1-dressed closed-shell intermediates) and
oracle/spinorb.py (spin orbitals, antisymmetrised integrals, explicit T1, the
Stanton-Gauss arrangement of the projected equations, its own Hamiltonian and
packed-layout map) share no code and no intermediates. Both compute the
projections E0 = <HF|Hbar|HF> and Omega_mu = <mu~|Hbar|HF> of Sec. 2.1.

* At tiny sizes both are pinned by the determinant engine (brute force in the
  full determinant space).
* At the o=5, v=19, J=72 workload, where the determinant engine cannot run,
  they must agree with each other: E0, Omega, A R along the three seeded unit
  vectors of that workload (A from the spin-orbital side by an exact 7-point
  stencil, Sec. 2.3.3), and A^T L through <L|A R> = <A^T L|R> with A^T L from
  the closed-shell side, plus single components (A^T L)_nu = L . (A e_nu).
* The SCC overlap O_ab of the natural projection (Sec. 2.4.2): determinant
  coefficients of exp(T)(r0 + R)|HF> in spin orbitals and the plain
  determinant inner product, against the closed-shell metric at o=5 v=19.
* The SCC term of Sec. 2.4.2, zeta <mu~|[Hhat, X3]|HF>: the spin-orbital side
  writes X3 as explicit triples and uses the triples terms of the CCSDT
  equations with T1-transformed integrals, pinned by the determinant engine at
  tiny sizes; at o=5 v=19 the closed-shell SCC residual and its A R equal it.
A mistake made in one factorisation (a dropped term, a wrong sign or index,
a transposed operand) cannot appear identically in the other.
"""
import numpy as np
import pytest

from oracle import ccsd as cc
from oracle import determinant as det
from oracle import response as rp
from oracle import spinorb as so
from paper_2403_01007_gb300 import synthetic as syn


@pytest.mark.parametrize("size", [(1, 4, 5), (2, 3, 6), (3, 3, 8)], ids=lambda s: "o%d_v%d" % s[:2])
def test_spin_orbital_oracle_equals_determinant_engine(size):
    o, v, J = size
    eps, L = syn.system(o, v, J, 0.3, 1)
    g = det.full_g(L)
    S = det.System(det.Space(o, v), det.synthetic_h(eps, g, o), g)
    sys_ = so.SpinSystem(eps, L, o)
    for seed in (7, 8):
        x = syn.random_vectors(o, v, 1, seed, scale=0.1)[0]
        E_d, Om_d = S.omega(x)
        E_s, Om_s = sys_.energy_residual(x)
        assert abs(E_d - E_s) < 1e-12 * max(1.0, abs(E_d))
        assert np.abs(Om_d - Om_s).max() < 1e-12 * max(1.0, np.abs(Om_d).max())


def test_spin_blocks_of_a_singlet():
    """For singlet amplitudes the spin-orbital projections have the singlet
    structure: beta blocks equal alpha blocks, spin-flip blocks vanish, and
    the same-spin doubles are the antisymmetrised (alpha, beta) block."""
    o, v, J = 2, 4, 7
    eps, L = syn.system(o, v, J, 0.3, 2)
    sys_ = so.SpinSystem(eps, L, o)
    x = syn.random_vectors(o, v, 1, 9, scale=0.1)[0]
    t1, t2 = sys_.spin_amplitudes(x)
    _, r1, r2 = sys_.energy_residual_spin(t1, t2)
    a, b = slice(0, o), slice(o, 2 * o)
    va, vb = slice(0, v), slice(v, 2 * v)
    scale = np.abs(r2).max()
    assert np.abs(r1[a, va] - r1[b, vb]).max() < 1e-13
    assert np.abs(r1[a, vb]).max() == 0.0 and np.abs(r1[b, va]).max() == 0.0
    ab = r2[a, b, va, vb]                                 # r_{i a, j b}^{a a, b b}
    same = r2[a, a, va, va]
    assert np.abs(same - (ab - ab.transpose(0, 1, 3, 2))).max() < 1e-13 * scale
    assert np.abs(r2[b, b, vb, vb] - same).max() < 1e-13 * scale
    assert np.abs(r2[a, a, va, vb]).max() < 1e-14 * scale
    assert np.abs(r2[a, b, vb, va] + ab.transpose(0, 1, 3, 2)).max() < 1e-13 * scale


@pytest.fixture(scope="module")
def c1():
    w = syn.SMALL
    eps, L = syn.workload_system(w)
    prob = cc.Problem(eps, L, w.o)
    sys_ = so.SpinSystem(eps, L, w.o)
    x = syn.random_vectors(w.o, w.v, 1, syn.seed_of(w.config, 50), scale=0.05)[0]
    R = syn.random_vectors(w.o, w.v, 3, syn.seed_of(w.config, 60), normalise=True)
    Lb = syn.random_vectors(w.o, w.v, 1, syn.seed_of(w.config, 70), normalise=True)[0]
    return w, prob, sys_, x, R, Lb


def test_closed_shell_oracle_equals_spin_orbital_oracle_at_o5_v19(c1):
    w, prob, sys_, x, R, Lb = c1
    E_c, Om_c = rp.residual(prob, x)
    E_s, Om_s = sys_.energy_residual(x)
    assert abs(float(E_c) - E_s) < 1e-12 * abs(E_s)
    assert np.abs(Om_c.numpy() - Om_s).max() < 1e-12 * np.abs(Om_s).max()
    # the MP2 amplitudes of the converged-state neighbourhood are not special:
    # also at t = 0 (Omega = the doubles integrals, singles F_ai = 0)
    E0c, O0c = rp.residual(prob, np.zeros(prob.dim))
    E0s, O0s = sys_.energy_residual(np.zeros(prob.dim))
    assert abs(float(E0c) - E0s) < 1e-12 * abs(E0s)
    assert np.abs(O0c.numpy() - O0s).max() < 1e-13 * np.abs(O0s).max()


def test_jacobians_equal_spin_orbital_stencil_at_o5_v19(c1):
    w, prob, sys_, x, R, Lb = c1
    ATL = rp.jacobian_left(prob, x, Lb).numpy()
    for k in range(3):
        ar_s = sys_.jacobian_right(x, R[k])
        ar_c = rp.jacobian_right(prob, x, R[k]).numpy()
        assert np.abs(ar_c - ar_s).max() < 1e-11 * np.abs(ar_s).max()
        # <L|A R> with A from the spin-orbital side = <A^T L|R> from the closed shell
        lhs, rhs = float(Lb @ ar_s), float(ATL @ R[k])
        assert abs(lhs - rhs) < 1e-11 * np.abs(Lb).max() * np.abs(ar_s).sum()
    # single components (A^T L)_nu = L . (A e_nu): two singles, two doubles
    ov = w.o * w.v
    for nu in (3, ov - 1, ov + 17, prob.dim - 5):
        e = np.zeros(prob.dim)
        e[nu] = 1.0
        col = sys_.jacobian_right(x, e)
        assert abs(float(Lb @ col) - ATL[nu]) < 1e-11 * max(1.0, np.abs(col).max())


@pytest.mark.parametrize("size", [(2, 3, 6), (2, 4, 7), (3, 3, 8)], ids=lambda s: "o%d_v%d" % s[:2])
def test_spin_orbital_x3_term_equals_determinant_engine(size):
    """T + zeta X3 (Sec. 2.4.1): the spin-orbital residual with explicit triples
    equals the determinant engine's projections with the X3 operator added."""
    o, v, J = size
    eps, L = syn.system(o, v, J, 0.3, 11)
    g = det.full_g(L)
    S = det.System(det.Space(o, v), det.synthetic_h(eps, g, o), g)
    sys_ = so.SpinSystem(eps, L, o)
    x = syn.random_vectors(o, v, 1, 12, scale=0.1)[0]
    Ra, Rb = syn.random_vectors(o, v, 2, 13, normalise=True)
    zeta = 0.37
    E_d, Om_d = S.omega(x, extra=zeta * det.x3_operator(S.S, Ra, Rb))
    E_s, Om_s = sys_.energy_residual_scc(x, zeta, Ra, Rb)
    assert abs(E_d - E_s) < 1e-12 * max(1.0, abs(E_d))
    assert np.abs(Om_d - Om_s).max() < 1e-12 * max(1.0, np.abs(Om_d).max())
    # the term is present
    assert np.abs(Om_s - sys_.energy_residual(x)[1]).max() > 1e-3


def test_closed_shell_scc_residual_and_jacobian_equal_spin_orbital_at_o5_v19(c1):
    """At o=5 v=19 J=72 the closed-shell SCC residual (T1-dressed X3 terms), its
    A R and (through <L|A R> = <A^T L|R>) its A^T L equal the spin-orbital
    formulation with explicit triples."""
    import torch
    w, prob, sys_, x, R, Lb = c1
    Ra, Rb = syn.random_vectors(w.o, w.v, 2, syn.seed_of(w.config, 80), normalise=True)
    zeta = 0.3
    scc = (zeta, torch.tensor(Ra), torch.tensor(Rb))
    E_s, Om_s = sys_.energy_residual_scc(x, zeta, Ra, Rb)
    E_c, Om_c = rp.residual(prob, x, scc=scc)
    assert abs(float(E_c) - E_s) < 1e-12 * abs(E_s)
    assert np.abs(Om_c.numpy() - Om_s).max() < 1e-12 * np.abs(Om_s).max()
    assert np.abs(Om_s - sys_.energy_residual(x)[1]).max() > 1e-3
    ar_s = sys_.jacobian_right_scc(x, R[0], zeta, Ra, Rb)
    ar_c = rp.jacobian_right(prob, x, R[0], scc=scc).numpy()
    assert np.abs(ar_c - ar_s).max() < 1e-11 * np.abs(ar_s).max()
    # A^T L of the closed-shell SCC residual through <L|A R> with A from the spin side
    atl = rp.jacobian_left(prob, x, Lb, scc=scc).numpy()
    assert abs(float(Lb @ ar_s) - float(atl @ R[0])) < 1e-11 * np.abs(Lb).max() * np.abs(ar_s).sum()


@pytest.mark.parametrize("size", [(1, 4, 5), (2, 3, 6), (3, 3, 8)], ids=lambda s: "o%d_v%d" % s[:2])
def test_spin_orbital_overlap_equals_determinant_engine(size):
    o, v, J = size
    eps, L = syn.system(o, v, J, 0.3, 21)
    g = det.full_g(L)
    S = det.System(det.Space(o, v), det.synthetic_h(eps, g, o), g)
    sys_ = so.SpinSystem(eps, L, o)
    x = syn.random_vectors(o, v, 1, 22, scale=0.1)[0]
    Ra, Rb = syn.random_vectors(o, v, 2, 23, normalise=True)
    ref = S.overlap(x, 0.3, Ra, -0.2, Rb)
    assert abs(sys_.overlap(x, 0.3, Ra, -0.2, Rb) - ref) < 1e-13 * max(1.0, abs(ref))


def test_closed_shell_overlap_equals_spin_orbital_at_o5_v19(c1):
    """O_ab with the closed-shell doubles metric (sum c2 (2 c2' - c2' with
    i <-> j)) equals the plain determinant inner product in spin orbitals."""
    import torch
    from oracle import scc as sc
    w, prob, sys_, x, R, Lb = c1
    Ra, Rb = syn.random_vectors(w.o, w.v, 2, syn.seed_of(w.config, 81), normalise=True)
    a = sys_.overlap(x, 0.3, Ra, -0.2, Rb)
    b = float(sc.overlap(torch.tensor(x), 0.3, torch.tensor(Ra), -0.2, torch.tensor(Rb), w.o, w.v))
    assert abs(a - b) < 1e-12 * max(1.0, abs(a))
