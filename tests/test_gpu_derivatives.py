"""Gradients and couplings along perturbations of the integrals, and SCCSD(K)
(the state projection of Sec. 2.4.1), on the GPU library through the C ABI:
the same checks as the CPU test double's, against the oracle, stored oracle
solutions and finite differences of re-converged states."""
import json
import os

import numpy as np
import pytest
import torch

import derivative_checks as dc
from oracle import scc as sc
from paper_2403_01007_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _golden(name):
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        return json.load(f)


@pytest.mark.parametrize("projection", ["natural", "state"])
def test_gradient_and_coupling_by_finite_differences(projection):
    """Sec. 2.3.2: sum D1 h1 + sum Gamma L1 of the GPU multipliers equals
    central differences of GPU-re-converged SCCSD(E) / SCCSD(K) energies and
    bra-frozen overlaps along random perturbations of eps and L."""
    from paper_2403_01007_gb300 import binding as B
    p = _golden("scc_active_o3_v8.json")["inputs"]
    o, v, J = p["o"], p["v"], p["J"]
    eps, L = syn.system(o, v, J, p["sd"], p["seed"])
    dc.check(lambda e, l: B.Context(o, v, J, e, l), eps, L, o, v, J, projection)


def test_state_projection_overlap():
    """O_ab of the state projection on the device equals the oracle's (pinned
    against determinant vectors), at o=5 v=19 with an SCC state."""
    from paper_2403_01007_gb300 import binding as B
    w = syn.SMALL
    eps, L = syn.workload_system(w)
    t = syn.random_vectors(w.o, w.v, 1, 301, scale=0.02)[0]
    Ra, Rb = syn.random_vectors(w.o, w.v, 2, 302, normalise=True)
    ctx = B.Context(w.o, w.v, w.J, eps, L)
    ctx.residual(t, scc=(0.2, Ra, Rb))
    O = ctx.overlap_states(0.3, Ra, -0.2, Rb)
    ref = float(sc.overlap_states(torch.tensor(t), 0.3, torch.tensor(Ra), -0.2, torch.tensor(Rb),
                                  w.o, w.v))
    assert abs(O - ref) < 1e-12 * max(1.0, abs(ref))
    ctx.close()


def test_state_projection_scc_loop():
    """SCCSD(K) on the device reaches the stored oracle solution."""
    from paper_2403_01007_gb300 import binding as B
    g = _golden("scc_state_projection_o3_v8.json")
    p = g["inputs"]
    eps, L = syn.system(p["o"], p["v"], p["J"], p["sd"], p["seed"])
    ctx = B.Context(p["o"], p["v"], p["J"], eps, L)
    ctx.set_projection("state")
    r = ctx.solve_scc(tol=1e-10)
    ctx.close()
    assert abs(r["zeta"] - g["values"]["zeta"]) < 1e-7
    assert np.abs(r["omega"] - np.array(g["values"]["omega"])).max() < 1e-8
    assert abs(r["e_corr"] - g["values"]["e_corr"]) < 1e-9
