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


FIXTURES = {"fci_two_electron_o1_v5.json": fci_two_electron,
            "scc_symmetric_o3_v6.json": scc_symmetric}


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def main():
    for name, fn in FIXTURES.items():
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(fn(), f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main()
