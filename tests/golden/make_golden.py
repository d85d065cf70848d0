"""Writes the stored expected values under tests/golden/.

Test infrastructure: it calls only the FP64 CPU oracle (oracle/) and the
seeded input generators, never the CUDA path. The paper prints no value that
can be reproduced without its molecular integrals (its examples are
formaldimine, thymine and LiH), so every fixture here is a value of the
oracle on a seeded synthetic system, stored with the passage that defines it.

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SYM_OCC, SYM_VIR = [0, 1, 0], [0, 1, 0, 1, 0, 1]


def fci_two_electron():
    """Two electrons (o=1, v=5): full CI by brute force in the determinant
    space. CCSD is exact for two electrons (the cluster operator of Sec. 2.1
    truncated at doubles spans every excitation), so the CCSD correlation
    energy and the EOM-CCSD excitation energies are these FCI values."""
    from oracle import ccsd as cc
    from oracle import determinant as det
    from oracle import response as rp
    from paper_2403_01007_gb300 import synthetic as syn
    o, v, J, sd, seed = 1, 5, 6, 0.25, 3
    eps, L = syn.system(o, v, J, sd, seed)
    g = det.full_g(L)
    h = det.synthetic_h(eps, g, o)
    system = det.System(det.Space(o, v), h, g)
    M = system.hbar_matrix(np.zeros(system.S.packed_dim))
    fci = np.sort(np.linalg.eigvals(M).real)
    prob = cc.Problem(eps, L, o)
    e_hf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    return {
        "citation": "Sec. 2.1 (CCSD ground and EOM states); exact for two electrons",
        "produced_by": "tests/golden/make_golden.py: oracle.determinant (full CI matrix)",
        "inputs": {"generator": "synthetic.system", "o": o, "v": v, "J": J, "sd": sd,
                   "seed": seed},
        "values": {"e_corr": float(fci[0] - e_hf),
                   "excitation_energies": [float(x) for x in fci[1:] - fci[0]]},
    }


def scc_symmetric():
    """Two-irrep system whose two lowest states differ in symmetry: the
    similarity constraint holds at zeta = 0 and SCCSD equals CCSD
    (Sec. 3.1.1, the planar intersection of formaldimine)."""
    import torch
    from oracle import ccsd as cc
    from oracle import response as rp
    from oracle import scc as sc
    from oracle import solvers as sv
    from paper_2403_01007_gb300 import synthetic as syn
    o, v, J, sd, seed = 3, 6, 18, 0.2, 1007
    eps, L, _, _ = syn.symmetric_system(o, v, J, sd, seed, SYM_OCC, SYM_VIR)
    prob = cc.Problem(eps, L, o)
    s = sc.solve_scc(prob, tol=1e-12, ground_tol=1e-12, dense=True)
    e_hf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    return {
        "citation": "Sec. 3.1.1 (states of different symmetry: SCCSD reduces to CCSD); "
                    "Sec. 2.2 (the constraint O_ab = 0) with the natural projection of "
                    "Sec. 2.4.1",
        "produced_by": "tests/golden/make_golden.py: oracle.scc.solve_scc (dense roots)",
        "inputs": {"generator": "synthetic.symmetric_system", "o": o, "v": v, "J": J, "sd": sd,
                   "seed": seed, "irrep_occ": SYM_OCC, "irrep_vir": SYM_VIR},
        "values": {"zeta": 0.0, "e_corr": float(s["E0"] - e_hf),
                   "omega": [float(x) for x in s["omega"]], "O_ab": 0.0},
    }


SCC_ACTIVE = dict(o=3, v=8, J=14, sd=0.1, seed=123)


def _scc_active_values(s, prob):
    from oracle import response as rp
    e_hf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    return {"zeta": float(s["zeta"]), "e_corr": float(s["E0"] - e_hf),
            "omega": [float(x) for x in s["omega"]]}


def scc_active(projection="natural"):
    """A system where the constraint is active (zeta far from 0): the
    self-consistent SCCSD solution of Sec. 2.2 and 2.4 for the two lowest
    states, from the oracle's loop (ground state and Davidson roots
    re-converged at each zeta, secant on O_ab). The converged t, R_a, R_b are
    stored too, so that a check can evaluate the defining equations there."""
    from oracle import ccsd as cc
    from oracle import scc as sc
    from paper_2403_01007_gb300 import synthetic as syn
    p = SCC_ACTIVE
    eps, L = syn.system(p["o"], p["v"], p["J"], p["sd"], p["seed"])
    prob = cc.Problem(eps, L, p["o"])
    s = sc.solve_scc(prob, tol=1e-10, projection=projection)
    return {
        "citation": "Sec. 2.2 (O_ab = 0 enforced by zeta) and Sec. 2.4.1-2.4.2 (SCCSD with "
                    "X3 = R1^a R2^b - R1^b R2^a, %s projection)" % projection,
        "produced_by": "tests/golden/make_golden.py: oracle.scc.solve_scc (Davidson roots)",
        "inputs": {"generator": "synthetic.system", **p, "projection": projection},
        "values": _scc_active_values(s, prob),
        "state": {"t": [float(x) for x in s["t"]], "Ra": [float(x) for x in s["Ra"]],
                  "Rb": [float(x) for x in s["Rb"]]},
    }


def scc_active_verify(stored):
    """The defining equations of the stored solution, evaluated by the oracle
    (instead of re-running the two-minute loop): the SCC ground residual
    Omega(t; zeta, R_a, R_b), the right eigen-equations A R_k = omega_k R_k of
    the SCC Jacobian (Sec. 2.1), the constraint O_ab with r0_k = eta.R_k /
    omega_k (Sec. 2.2, 2.4.1), and E_corr. Returns {name: (value, bound)}."""
    import torch
    from oracle import ccsd as cc
    from oracle import response as rp
    from oracle import scc as sc
    from paper_2403_01007_gb300 import synthetic as syn
    p = SCC_ACTIVE
    eps, L = syn.system(p["o"], p["v"], p["J"], p["sd"], p["seed"])
    prob = cc.Problem(eps, L, p["o"])
    val, st = stored["values"], stored["state"]
    t, Ra, Rb = (np.array(st[k]) for k in ("t", "Ra", "Rb"))
    zeta = val["zeta"]
    scc = (zeta, torch.tensor(Ra), torch.tensor(Rb))
    E0, Om = rp.residual(prob, t, scc=scc)
    e_hf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    out = {"ground residual": (float(torch.linalg.norm(Om)), 1e-8),
           "e_corr": (abs(float(E0) - e_hf - val["e_corr"]), 1e-10)}
    eta = rp.eta(prob, t, scc=scc).numpy()
    r0 = []
    for name, R, w in (("a", Ra, val["omega"][0]), ("b", Rb, val["omega"][1])):
        AR = rp.jacobian_right(prob, t, R, scc=scc).numpy()
        out["eigen-equation " + name] = (float(np.linalg.norm(AR - w * R)), 1e-7)
        r0.append(float(eta @ R / w))
    ovl = sc.overlap_states if stored["inputs"].get("projection") == "state" else sc.overlap
    O = float(ovl(torch.tensor(t), r0[0], torch.tensor(Ra), r0[1], torch.tensor(Rb),
                  prob.o, prob.v))
    out["O_ab"] = (abs(O), 1e-9)
    return out


SCC_THREE = dict(o=3, v=6, J=18, sd=0.2, seed=1007)


def scc_three_states(projection="natural"):
    """Three constrained states (Sec. 2.2 with K = {1, 2, 3}; X_kl of Sec.
    2.4.1 for every pair) on the two-irrep system: the oracle's loop (ground
    state and three Davidson roots re-converged at each zeta, Broyden on the
    three O_kl from zeta = 0), with the natural projection or the state
    projection over all three states. Two pairs join states of different
    symmetry, whose zeta stays 0 (Sec. 3.1.1); the pair of equal symmetry is
    active. The converged t and R_k are stored for the check of the defining
    equations (the loop takes about twenty minutes)."""
    from oracle import ccsd as cc
    from oracle import response as rp
    from oracle import scc as sc
    from paper_2403_01007_gb300 import synthetic as syn
    p = SCC_THREE
    eps, L, _, _ = syn.symmetric_system(p["o"], p["v"], p["J"], p["sd"], p["seed"], SYM_OCC,
                                        SYM_VIR)
    prob = cc.Problem(eps, L, p["o"])
    s = sc.solve_scc_states(prob, 3, tol=1e-10, ground_tol=1e-11, dense=False, maxit=40,
                            projection=projection)
    e_hf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    pairs = [(0, 1), (0, 2), (1, 2)]
    return {
        "citation": "Sec. 2.2 (O_kl = 0 for every pair of K, here three states) and "
                    "Sec. 2.4.1 (X_kl = R1^k R2^l - R1^l R2^k, %s projection); "
                    "Sec. 3.1.1 (states of different symmetry need no constraint)" % projection,
        "produced_by": "tests/golden/make_golden.py: oracle.scc.solve_scc_states "
                       "(Davidson roots)",
        "inputs": {"generator": "synthetic.symmetric_system", **p, "irrep_occ": SYM_OCC,
                   "irrep_vir": SYM_VIR, "nstates": 3, "projection": projection},
        "values": {"zeta": [float(s["zeta"][kl]) for kl in pairs],
                   "e_corr": float(s["E0"] - e_hf),
                   "omega": [float(x) for x in s["omega"][:3]]},
        "state": {"t": [float(x) for x in s["t"]],
                  "R": [[float(x) for x in s["R"][k]] for k in range(3)]},
    }


def scc_three_states_verify(stored):
    """The defining equations at the stored three-state solution, evaluated by
    the oracle: the ground residual with sum_kl zeta_kl X_kl, the three right
    eigen-equations, every O_kl with r0_k = eta.R_k / omega_k, and E_corr."""
    import torch
    from oracle import ccsd as cc
    from oracle import response as rp
    from oracle import scc as sc
    from paper_2403_01007_gb300 import synthetic as syn
    p = SCC_THREE
    eps, L, _, _ = syn.symmetric_system(p["o"], p["v"], p["J"], p["sd"], p["seed"], SYM_OCC,
                                        SYM_VIR)
    prob = cc.Problem(eps, L, p["o"])
    val, st = stored["values"], stored["state"]
    t = np.array(st["t"])
    R = [np.array(r) for r in st["R"]]
    pairs = [(0, 1), (0, 2), (1, 2)]
    scc = [(z, torch.tensor(R[k]), torch.tensor(R[l])) for z, (k, l) in zip(val["zeta"], pairs)]
    E0, Om = rp.residual(prob, t, scc=scc)
    e_hf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    out = {"ground residual": (float(torch.linalg.norm(Om)), 1e-8),
           "e_corr": (abs(float(E0) - e_hf - val["e_corr"]), 1e-10)}
    eta = rp.eta(prob, t, scc=scc).numpy()
    r0 = []
    for k in range(3):
        AR = rp.jacobian_right(prob, t, R[k], scc=scc).numpy()
        out["eigen-equation %d" % k] = (float(np.linalg.norm(AR - val["omega"][k] * R[k])), 1e-7)
        r0.append(float(eta @ R[k] / val["omega"][k]))
    O = sc.overlaps(torch.tensor(t), [(r0[k], torch.tensor(R[k])) for k in range(3)],
                    prob.o, prob.v, stored["inputs"]["projection"])
    for kl in pairs:
        out["O_%d%d" % kl] = (abs(float(O[kl])), 1e-9)
    out["constraint active"] = (1.0 / max(abs(val["zeta"][1]), 1e-300), 1.0 / 0.3)
    return out


FIXTURES = {"fci_two_electron_o1_v5.json": fci_two_electron,
            "scc_symmetric_o3_v6.json": scc_symmetric,
            "scc_active_o3_v8.json": scc_active,
            "scc_state_projection_o3_v8.json": lambda: scc_active("state"),
            "scc_three_states_o3_v6.json": scc_three_states,
            "scc_three_states_state_projection_o3_v6.json": lambda: scc_three_states("state")}
# fixtures whose full regeneration is slow: checked through their defining
# equations instead
VERIFY = {"scc_active_o3_v8.json": scc_active_verify,
          "scc_state_projection_o3_v8.json": scc_active_verify,
          "scc_three_states_o3_v6.json": scc_three_states_verify,
          "scc_three_states_state_projection_o3_v6.json": scc_three_states_verify}


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def main(names=None):
    for name, fn in FIXTURES.items():
        if names and name not in names:
            continue
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(fn(), f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
