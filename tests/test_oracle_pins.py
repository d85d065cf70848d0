"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

* brute force: every closed-shell quantity against the determinant-space
  engine, which applies the defining second-quantised expressions directly;
* exactness: for two electrons CCSD and EOM-CCSD equal full CI;
* closed forms: the MP2 first iterate and energy, the HF energy, the
  commutation relations of the singlet excitation operators;
* exact identities: a 7-point central stencil is exact for the quartic
  polynomial Omega(t + e R); <L|A R> = <A^T L|R>; density sum rules;
* symmetry: with two states of different symmetry the similarity constraint
  holds at zeta = 0 and SCCSD is CCSD (Sec. 3.1.1).
"""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle import determinant as det
from oracle import response as rp
from oracle import scc as sc
from oracle import solvers as sv
from paper_2403_01007_gb300 import synthetic as syn

TINY = [(2, 3, 6), (3, 3, 8), (2, 4, 7), (1, 4, 5)]


def tiny_system(o, v, J, seed=1, sd=0.3):
    eps, L = syn.system(o, v, J, sd, seed)
    g = det.full_g(L)
    h = det.synthetic_h(eps, g, o)
    S = det.Space(o, v)
    return eps, L, det.System(S, h, g), cc.Problem(eps, L, o)


@pytest.fixture(scope="module", params=TINY, ids=lambda p: "o%d_v%d" % p[:2])
def tiny(request):
    o, v, J = request.param
    return (o, v) + tiny_system(o, v, J)


# ---------------------------------------------------------------- engine pins

def test_excitation_operator_algebra():
    """[E_pq, E_rs] = d_qr E_ps - d_ps E_rq on the determinant space."""
    S = det.Space(2, 2)
    n = S.n
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for s in range(n):
                    lhs = (S.E(p, q) @ S.E(r, s) - S.E(r, s) @ S.E(p, q)).toarray()
                    rhs = np.zeros_like(lhs)
                    if q == r:
                        rhs += S.E(p, s).toarray()
                    if p == s:
                        rhs -= S.E(r, q).toarray()
                    assert np.abs(lhs - rhs).max() == 0.0


def test_engine_reference_energy(tiny):
    o, v, eps, L, system, prob = tiny
    g = det.full_g(L)
    h = system.h
    E_hf = 2 * np.trace(h[:o, :o]) + sum(2 * g[i, i, j, j] - g[i, j, j, i]
                                         for i in range(o) for j in range(o))
    e0, om = system.omega(np.zeros(system.S.packed_dim))
    assert abs(e0 - E_hf) < 1e-12
    # canonical reference: F_ai = 0, so the singles vanish at t = 0, and the
    # doubles equal g_aibj (the MP2 driving term)
    ov = o * v
    assert np.abs(om[:ov]).max() < 1e-13
    gd = np.array([g[o + P // o, P % o, o + Q // o, Q % o] for P, Q in det.packed_pairs(ov)])
    assert np.abs(om[ov:] - gd).max() < 1e-13


def test_doubles_metric_closed_form():
    """<D|D'> for D = 1/2 sum x E E|HF> is sum x (2 y - y exchanged)."""
    o, v = 2, 3
    S = det.Space(o, v)
    x = syn.random_vectors(o, v, 2, 3)
    kx, ky = S.ket(0.4, x[0]), S.ket(-0.7, x[1])
    ref = float(kx @ ky)
    got = sc.metric_product(sc.projected_state(torch.zeros(S.packed_dim), 0.4, x[0], o, v),
                            sc.projected_state(torch.zeros(S.packed_dim), -0.7, x[1], o, v))
    assert abs(float(got) - ref) < 1e-13


# ------------------------------------------------------- oracle vs brute force

def test_energy_residual_vs_brute_force(tiny):
    o, v, eps, L, system, prob = tiny
    for seed in (7, 8):
        t = syn.random_vectors(o, v, 1, seed, scale=0.1)[0]
        E0, om = system.omega(t)
        e, O = rp.residual(prob, t)
        assert abs(float(e) - E0) < 1e-12
        assert np.abs(O.numpy() - om).max() < 1e-12


def test_jacobians_vs_brute_force(tiny):
    o, v, eps, L, system, prob = tiny
    t = syn.random_vectors(o, v, 1, 7, scale=0.1)[0]
    A, eta = system.jacobian(t)
    R, Lv = syn.random_vectors(o, v, 2, 9, normalise=True)
    assert np.abs(rp.jacobian_right(prob, t, R).numpy() - A @ R).max() < 1e-12
    assert np.abs(rp.jacobian_left(prob, t, Lv).numpy() - A.T @ Lv).max() < 1e-12
    assert np.abs(rp.eta(prob, t).numpy() - eta).max() < 1e-12


def test_scc_terms_vs_brute_force(tiny):
    o, v, eps, L, system, prob = tiny
    t = syn.random_vectors(o, v, 1, 7, scale=0.1)[0]
    Ra, Rb, R, Lv = syn.random_vectors(o, v, 4, 11, normalise=True)
    zeta = 0.37
    X3 = zeta * det.x3_operator(system.S, Ra, Rb)
    scc = (zeta, torch.tensor(Ra), torch.tensor(Rb))
    E0, om = system.omega(t, extra=X3)
    _, om0 = system.omega(t)
    e, O = rp.residual(prob, t, scc=scc)
    assert abs(float(e) - E0) < 1e-12
    assert np.abs(O.numpy() - om).max() < 1e-12
    if o * v > 4:     # the term is non-trivial
        assert np.abs(om - om0).max() > 1e-3
    A, _ = system.jacobian(t, extra=X3)
    assert np.abs(rp.jacobian_right(prob, t, R, scc=scc).numpy() - A @ R).max() < 1e-12
    assert np.abs(rp.jacobian_left(prob, t, Lv, scc=scc).numpy() - A.T @ Lv).max() < 1e-12


def test_several_constrained_pairs_vs_brute_force(tiny):
    """K of three states (Sec. 2.2): T + sum_kl zeta_kl X_kl over the pairs
    k < l; the residual and both Jacobians against the determinant engine with
    the summed operators, and the overlaps of both projections against full
    determinant vectors; with two states they are the two-state functions."""
    o, v, eps, L, system, prob = tiny
    t = syn.random_vectors(o, v, 1, 7, scale=0.1)[0]
    Ra, Rb, Rc, R, Lv = syn.random_vectors(o, v, 5, 13, normalise=True)
    pairs = [(0.37, Ra, Rb), (-0.21, Ra, Rc), (0.15, Rb, Rc)]
    X = sum(z * det.x3_operator(system.S, x, y) for z, x, y in pairs)
    scc = [(z, torch.tensor(x), torch.tensor(y)) for z, x, y in pairs]
    E0, om = system.omega(t, extra=X)
    e, O = rp.residual(prob, t, scc=scc)
    assert abs(float(e) - E0) < 1e-12
    assert np.abs(O.numpy() - om).max() < 1e-12
    A, _ = system.jacobian(t, extra=X)
    assert np.abs(rp.jacobian_right(prob, t, R, scc=scc).numpy() - A @ R).max() < 1e-12
    assert np.abs(rp.jacobian_left(prob, t, Lv, scc=scc).numpy() - A.T @ Lv).max() < 1e-12
    states = [(0.3, Ra), (-0.2, Rb), (0.1, Rc)]
    tt = torch.tensor(t)
    ts = [(r0, torch.tensor(r)) for r0, r in states]
    ref = det.overlaps_states(system, t, states)
    got = sc.overlaps(tt, ts, o, v, "state")
    for kl in ref:
        assert abs(float(got[kl]) - ref[kl]) < 1e-12 * max(1.0, abs(ref[kl]))
    nat = sc.overlaps(tt, ts, o, v, "natural")
    for (k, l), val in nat.items():
        assert abs(float(val) - system.overlap(t, *states[k], *states[l])) < 1e-12
    two = sc.overlaps(tt, ts[:2], o, v, "state")
    assert abs(float(two[(0, 1)]) - float(sc.overlap_states(tt, *ts[0], *ts[1], o, v))) < 1e-13


def test_several_states_loop_reduces_to_two_states():
    """With two states Broyden's update is the secant step, so the loop for
    several constrained states is the two-state loop; on the symmetric system
    whose two lowest states differ in symmetry both stop at zeta = 0 with the
    CCSD energies (Sec. 3.1.1)."""
    o, v, J = 3, 6, 18
    eps, L, _, _ = syn.symmetric_system(o, v, J, 0.2, 1007, SYM_OCC, SYM_VIR)
    prob = cc.Problem(eps, L, o)
    two = sc.solve_scc(prob, tol=1e-12, ground_tol=1e-12, dense=True)
    gen = sc.solve_scc_states(prob, 2, tol=1e-12, ground_tol=1e-12, dense=True)
    assert abs(gen["zeta"][(0, 1)]) < 1e-12 and abs(two["zeta"]) < 1e-12
    assert np.allclose(gen["omega"], two["omega"], rtol=0, atol=1e-12)
    assert abs(gen["E0"] - two["E0"]) < 1e-12


@pytest.mark.parametrize("with_scc", [False, True])
def test_densities_vs_brute_force(tiny, with_scc):
    o, v, eps, L, system, prob = tiny
    t = syn.random_vectors(o, v, 1, 7, scale=0.1)[0]
    Ra, Rb, R, Lv = syn.random_vectors(o, v, 4, 13, normalise=True)
    extra, scc = None, None
    if with_scc:
        extra = 0.25 * det.x3_operator(system.S, Ra, Rb)
        scc = (0.25, torch.tensor(Ra), torch.tensor(Rb))
    l0, r0 = 0.7, -0.4
    d1, d2 = system.densities(t, l0, Lv, r0, R, extra=extra)
    D1, G = rp.densities(prob, t, l0, Lv, r0, R, scc=scc)
    assert np.abs(D1.numpy() - d1).max() < 1e-12
    assert np.abs(G.numpy() - np.einsum("pqrs,Jrs->Jpq", d2, L)).max() < 1e-12
    # sum rules of the two-particle density: sum_r d_pqrr = (N - 1) d_pq
    N = 2 * o
    assert np.abs(np.einsum("pqrr->pq", d2) - (N - 1) * d1).max() < 1e-11


def test_overlap_vs_brute_force(tiny):
    o, v, eps, L, system, prob = tiny
    t = syn.random_vectors(o, v, 1, 7, scale=0.1)[0]
    Ra, Rb = syn.random_vectors(o, v, 2, 17, normalise=True)
    ref = system.overlap(t, 0.3, Ra, -0.2, Rb)
    got = sc.overlap(torch.tensor(t), 0.3, torch.tensor(Ra), -0.2, torch.tensor(Rb), o, v)
    assert abs(float(got) - ref) < 1e-12


def test_state_projection_overlap_vs_brute_force(tiny):
    """O_ab with the state projection of Sec. 2.4.1 against full determinant
    vectors; at T = 0 the projector reproduces its own span, so O_ab is the
    plain Hilbert overlap <R_a|R_b>."""
    o, v, eps, L, system, prob = tiny
    t = syn.random_vectors(o, v, 1, 7, scale=0.1)[0]
    Ra, Rb = syn.random_vectors(o, v, 2, 17, normalise=True)
    ref = system.overlap_states(t, 0.3, Ra, -0.2, Rb)
    got = sc.overlap_states(torch.tensor(t), 0.3, torch.tensor(Ra), -0.2, torch.tensor(Rb), o, v)
    assert abs(float(got) - ref) < 1e-12 * max(1.0, abs(ref))
    z = np.zeros_like(t)
    S = system.S
    plain = float(S.ket(0.3, Ra) @ S.ket(-0.2, Rb))
    assert abs(system.overlap_states(z, 0.3, Ra, -0.2, Rb) - plain) < 1e-12
    got0 = sc.overlap_states(torch.tensor(z), 0.3, torch.tensor(Ra), -0.2, torch.tensor(Rb), o, v)
    assert abs(float(got0) - plain) < 1e-12


# --------------------------------------------------------- exactness for N = 2

def test_two_electron_ccsd_is_full_ci():
    """With two electrons CCSD is exact: E0 and E0 + omega_k are FCI singlets."""
    o, v, J = 1, 5, 6
    eps, L, system, prob = tiny_system(o, v, J, seed=3, sd=0.25)
    x, E0, _ = sv.ground_state(prob, tol=1e-12)
    M = system.hbar_matrix(np.zeros(system.S.packed_dim))   # <mu~|H|nu> at T = 0
    fci = np.sort(np.linalg.eigvals(M).real)
    assert abs(E0 - fci[0]) < 1e-10
    A = torch.func.jacfwd(lambda y: cc.energy_residual(y, prob)[1])(torch.tensor(x)).numpy()
    w = np.sort(np.linalg.eigvals(A).real)
    assert np.abs((E0 + w) - fci[1:]).max() < 1e-9


# ------------------------------------------------------------ closed forms

def test_mp2_first_iterate():
    """From t = 0 one Jacobi step gives t_ij^ab = -g_aibj/D and E = E_MP2."""
    w = syn.SMALL
    eps, L = syn.workload_system(w)
    o, v = w.o, w.v
    prob = cc.Problem(eps, L, o)
    E_hf, om = rp.residual(prob, np.zeros(prob.dim))
    om = om.numpy()
    D = sv.denominators(prob)
    t = -om / D
    ov = o * v
    assert np.abs(om[:ov]).max() < 1e-13
    # closed form written out from the Cholesky vectors directly
    g_ovov = np.einsum("Jia,Jjb->iajb", L[:, :o, o:], L[:, :o, o:])
    e_o, e_v = eps[:o], eps[o:]
    Dijab = (e_v[None, :, None, None] + e_v[None, None, None, :]
             - e_o[:, None, None, None] - e_o[None, None, :, None])  # [i,a,j,b]
    t_ref = -g_ovov / Dijab
    t1, t2 = cc.unpack(t, o, v)
    assert np.abs(t2.numpy().transpose(1, 0, 3, 2) - t_ref).max() < 1e-14
    e_mp2 = -np.sum(g_ovov * (2 * g_ovov - g_ovov.transpose(0, 3, 2, 1)) / Dijab)
    E1, _ = rp.residual(prob, t)
    assert abs((float(E1) - float(E_hf)) - e_mp2) < 1e-12


# ----------------------------------------------------------- exact identities

@pytest.fixture(scope="module")
def small():
    w = syn.SMALL
    eps, L = syn.workload_system(w)
    prob = cc.Problem(eps, L, w.o)
    t = syn.random_vectors(w.o, w.v, 1, 21, scale=0.02)[0]
    return prob, t


def test_jacobian_right_is_exact_stencil(small):
    """Omega(t + e R) is a polynomial of degree <= 4 in e, so the 7-point
    central difference is exact up to rounding."""
    prob, t = small
    R = syn.random_vectors(prob.o, prob.v, 1, 23, normalise=True)[0]
    h = 0.05
    c = {1: 3 / 4, 2: -3 / 20, 3: 1 / 60}
    fd = np.zeros(prob.dim)
    for k, ck in c.items():
        fd += ck * (rp.residual(prob, t + k * h * R)[1].numpy()
                    - rp.residual(prob, t - k * h * R)[1].numpy())
    fd /= h
    AR = rp.jacobian_right(prob, t, R).numpy()
    assert np.abs(fd - AR).max() < 1e-9 * max(1.0, np.abs(AR).max())


def test_left_right_adjoint(small):
    prob, t = small
    R, Lv = syn.random_vectors(prob.o, prob.v, 2, 25, normalise=True)
    a = float(torch.dot(torch.tensor(Lv), rp.jacobian_right(prob, t, R)))
    b = float(torch.dot(rp.jacobian_left(prob, t, Lv), torch.tensor(R)))
    assert abs(a - b) < 1e-12 * max(1.0, abs(a))


def test_residual_symmetry(small):
    """t_ij^ab = t_ji^ba is kept by Omega."""
    prob, t = small
    t1, t2 = cc.unpack(t, prob.o, prob.v)
    _, O1, O2 = cc.ccsd_energy_residual(t1, t2, prob.h, prob.L, prob.o)
    assert torch.abs(O2 - O2.permute(2, 3, 0, 1)).max() < 1e-14


def test_density_sum_rules(small):
    """trace d = N <L|R>;  sum h d + 1/2 sum L Gamma = <L|Hbar|R> (Euler's
    relation for a functional linear in h and quadratic in L)."""
    prob, t = small
    R, Lv = syn.random_vectors(prob.o, prob.v, 2, 27, normalise=True)
    l0, r0 = 0.3, 0.8
    D1, G = rp.densities(prob, t, l0, Lv, r0, R)
    N = 2 * prob.o
    lr = l0 * r0 + float(np.dot(Lv, R))
    assert abs(float(torch.trace(D1)) - N * lr) < 1e-11
    F = rp.transition_element(prob, t, l0, Lv, r0, R, prob.h, prob.L)
    euler = torch.sum(prob.h * D1) + 0.5 * torch.sum(prob.L * G)
    assert abs(float(euler - F)) < 1e-10 * max(1.0, abs(float(F)))


def test_zeta_zero_is_ccsd(small):
    prob, t = small
    Ra, Rb = syn.random_vectors(prob.o, prob.v, 2, 29, normalise=True)
    _, O = rp.residual(prob, t)
    _, Oz = rp.residual(prob, t, scc=(0.0, torch.tensor(Ra), torch.tensor(Rb)))
    assert torch.abs(O - Oz).max() == 0.0


# ------------------------------------------------------------------ symmetry

SYM_OCC, SYM_VIR = [0, 1, 0], [0, 1, 0, 1, 0, 1]


def irrep_weights(x, o, v):
    """Fraction of |x|^2 on the components of each irrep (0, 1): a singles
    component a<-i has irrep s_a XOR s_i, a doubles component the XOR of its
    two pairs."""
    t1, t2 = cc.unpack(x, o, v)
    so, sv_ = np.array(SYM_OCC), np.array(SYM_VIR)
    g1 = sv_[:, None] ^ so[None, :]
    g2 = g1[:, :, None, None] ^ g1[None, None, :, :]
    a1, a2 = t1.numpy(), t2.numpy()
    w = np.array([(a1[g1 == k] ** 2).sum() + (a2[g2 == k] ** 2).sum() for k in (0, 1)])
    return w / w.sum()


def test_states_of_different_symmetry_need_no_constraint():
    """Where the two intersecting states differ in symmetry, the SCC correction
    vanishes and the method reduces to CCSD (Sec. 3.1.1, the planar
    intersection of formaldimine). In a two-irrep system: the ground state is
    totally symmetric, the two lowest roots lie in different irreps, O_ab
    vanishes at zeta = 0, and the SCC loop returns zeta = 0 with the CCSD
    energies. Contrast: in the same construction with a seed whose two lowest
    roots share an irrep, O_ab(0) is far from zero, so the loop must move zeta."""
    o, v, J = 3, 6, 18

    def ccsd_pair(seed):
        eps, L, _, _ = syn.symmetric_system(o, v, J, 0.2, seed, SYM_OCC, SYM_VIR)
        prob = cc.Problem(eps, L, o)
        x, E0, _ = sv.ground_state(prob, tol=1e-12)
        w, X = sv.eom_dense(prob, x, 2, side="right")
        Xa, Xb = sc.fix_sign(X[0]), sc.fix_sign(X[1])
        eta = rp.eta(prob, x).numpy()
        r0a, r0b = float(eta @ Xa / w[0]), float(eta @ Xb / w[1])
        O = float(sc.overlap(torch.tensor(x), r0a, torch.tensor(Xa), r0b, torch.tensor(Xb), o, v))
        return prob, x, E0, w, (Xa, Xb), O

    prob, x, E0, w, (Xa, Xb), O = ccsd_pair(1007)
    assert irrep_weights(x, o, v)[1] < 1e-24
    wa, wb = irrep_weights(Xa, o, v), irrep_weights(Xb, o, v)
    assert {int(np.argmax(wa)), int(np.argmax(wb))} == {0, 1}
    assert max(wa.min(), wb.min()) < 1e-24
    assert abs(O) < 1e-13
    s = sc.solve_scc(prob, tol=1e-12, ground_tol=1e-12, dense=True)
    assert abs(s["zeta"]) < 1e-12
    assert np.allclose(s["omega"], w, rtol=0, atol=1e-11)
    assert abs(s["E0"] - E0) < 1e-11

    _, _, _, _, (Ya, Yb), O_same = ccsd_pair(1000)
    assert np.argmax(irrep_weights(Ya, o, v)) == np.argmax(irrep_weights(Yb, o, v))
    assert abs(O_same) > 1e-3


# -------------------------------------------------------------- eigensolvers

def test_dense_roots_are_full_ci_for_two_electrons():
    """The dense EOM roots (explicit Jacobian assembled column by column,
    then a library eigendecomposition) are all the FCI excitation energies
    for two electrons."""
    o, v, J = 1, 4, 5
    eps, L, system, prob = tiny_system(o, v, J, seed=4, sd=0.25)
    x, E0, _ = sv.ground_state(prob, tol=1e-12)
    M = system.hbar_matrix(np.zeros(system.S.packed_dim))
    fci = np.sort(np.linalg.eigvals(M).real)
    w, _ = sv.eom_dense(prob, x, prob.dim, side="right")
    assert np.abs(w - (fci[1:] - fci[0])).max() < 1e-9
    wl, _ = sv.eom_dense(prob, x, prob.dim, side="left")
    assert np.abs(wl - w).max() < 1e-9


@pytest.mark.parametrize("side", ["right", "left"])
def test_davidson_finds_the_lowest_dense_roots(side):
    """The oracle's Davidson returns the nroots lowest eigenvalues of the
    explicit Jacobian, with vectors that satisfy A X = w X (right) or
    A^T X = w X (left) to the requested tolerance."""
    o, v, J = 3, 4, 9
    eps, L = syn.system(o, v, J, 0.2, 55)
    prob = cc.Problem(eps, L, o)
    x, _, _ = sv.ground_state(prob, tol=1e-12)
    wd, _ = sv.eom_dense(prob, x, 4, side=side)
    w, X = sv.eom(prob, x, 4, side=side, tol=1e-9)
    assert np.abs(w - wd).max() < 1e-8
    op = rp.jacobian_right if side == "right" else rp.jacobian_left
    for k in range(4):
        r = op(prob, x, X[k]).numpy() - w[k] * X[k]
        assert np.linalg.norm(r) < 1e-8
