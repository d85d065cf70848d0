"""Host logic on the CPU: the C ABI exports, and the tensor-operation graph
with its forward/reverse differentiation run through the same C ABI code
with a loop-based test double of the device backend (tests/host_executor),
against the FP64 oracle. The product library itself always needs the GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle import response as rp
from paper_2403_01007_gb300 import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2403_01007_gb300", "csrc")
HEADER = os.path.join(ROOT, "include", "sccsd.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sccsd_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    from paper_2403_01007_gb300 import binding
    lib_path = binding.LIB_PATH
    if not os.path.exists(lib_path):
        from paper_2403_01007_gb300 import build
        build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    exported = set(l.split()[-1] for l in out.stdout.splitlines() if l.strip())
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # the library loads without a GPU (CUDA is only touched by calls)
    ctypes.CDLL(lib_path)


@pytest.fixture(scope="module")
def host_lib():
    from paper_2403_01007_gb300 import binding
    tmp = tempfile.mkdtemp()
    so = os.path.join(tmp, "libsccsd_hostexec.so")
    srcs = [os.path.join(CSRC, f) for f in ("graph.cpp", "ccsd_graph.cpp", "api.cpp", "model.cpp",
                                            "solvers.cpp", "multipliers.cpp", "learned_api.cpp",
                                            "capture.cpp")]
    srcs.append(os.path.join(ROOT, "tests", "host_executor", "host_backend.cpp"))
    # SCCSD_HOST_SANITIZE=1 builds the executor with AddressSanitizer (run the
    # tests with the sanitizer runtime preloaded) to catch out-of-range buffer use
    san = ["-g", "-fsanitize=address", "-fno-omit-frame-pointer"] \
        if os.environ.get("SCCSD_HOST_SANITIZE") else []
    cmd = ["g++", "-O1", "-std=c++17", "-fPIC", "-shared", *san, "-I/usr/local/cuda/include",
           *srcs, "-L/usr/local/cuda/lib64", "-lcudart", "-o", so]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("host toolchain unavailable: " + r.stderr[-300:])
    return binding, binding.load(so)


@pytest.mark.parametrize("size", [(1, 2, 3), (2, 3, 6), (3, 4, 7)], ids=lambda s: "o%d_v%d" % s[:2])
@pytest.mark.parametrize("with_scc", [False, True], ids=["ccsd", "sccsd"])
def test_graph_differentiation_matches_oracle(host_lib, size, with_scc):
    B, lib = host_lib
    o, v, J = size
    eps, L = syn.system(o, v, J, 0.3, 77 + o + v)
    prob = cc.Problem(eps, L, o)
    t = syn.random_vectors(o, v, 1, 78, scale=0.1)[0]
    R = syn.random_vectors(o, v, 3, 79, normalise=True)
    Ra, Rb = syn.random_vectors(o, v, 2, 80, normalise=True)
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    scc = (0.4, Ra, Rb) if with_scc else None
    scct = (0.4, torch.tensor(Ra), torch.tensor(Rb)) if with_scc else None
    e, om = ctx.residual(t, scc=scc)
    E0, Om = rp.residual(prob, t, scc=scct)
    Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    assert abs(e - (float(E0) - Ehf)) < 1e-12
    assert np.abs(om - Om.numpy()).max() < 1e-12
    s, eta = ctx.jacobian_right(R, with_eta=True)
    sl = ctx.jacobian_left(R)
    for k in range(3):
        assert np.abs(s[k] - rp.jacobian_right(prob, t, R[k], scc=scct).numpy()).max() < 1e-12
        assert abs(eta[k] - float(rp.eta(prob, t, scc=scct) @ torch.tensor(R[k]))) < 1e-12
        assert np.abs(sl[k] - rp.jacobian_left(prob, t, R[k], scc=scct).numpy()).max() < 1e-12
    D1, G = ctx.densities(0.5, R[0], -0.2, R[1])
    D1r, Gr = rp.densities(prob, t, 0.5, R[0], -0.2, R[1], scc=scct)
    assert np.abs(D1 - D1r.numpy()).max() < 1e-12
    assert np.abs(G - Gr.numpy()).max() < 1e-12
    ctx.close()


def test_abi_argument_checks(host_lib):
    B, lib = host_lib
    h = ctypes.c_void_p()
    eps = np.linspace(-1, 1, 4)
    L = np.zeros((2, 4, 4))
    assert lib.sccsd_init(ctypes.byref(h), 0, 4, 2, eps.ctypes.data, L.ctypes.data, 0, None) == -1
    assert lib.sccsd_init(ctypes.byref(h), 2, 2, 2, None, L.ctypes.data, 0, None) == -1
    bad = np.array([-1.0, -2.0, 0.5, 1.0])
    assert lib.sccsd_init(ctypes.byref(h), 2, 2, 2, bad.ctypes.data, L.ctypes.data, 0, None) == -1
    ctx = B.Context(2, 2, 2, eps, L, lib=lib)
    with pytest.raises(B.SccsdError) as ei:
        ctx.jacobian_right(np.zeros(B.dim(2, 2)))
    assert ei.value.code == -4          # call order
    with pytest.raises(B.SccsdError) as ei:
        ctx.residual(np.zeros(B.dim(2, 2)), scc=(float("nan"), np.zeros(B.dim(2, 2)), np.zeros(B.dim(2, 2))))
    assert ei.value.code == -1
    ctx.close()


@pytest.fixture(scope="module")
def mult_system():
    from oracle import multipliers as mu
    o, v, J = 2, 4, 10
    eps, L = syn.system(o, v, J, 0.1, 1)
    prob = cc.Problem(eps, L, o)
    st = mu.scc_state(prob)
    state = {"t": st["t"].numpy(), "Ra": st["Ra"].numpy(), "Rb": st["Rb"].numpy(),
             "La": st["La"].numpy(), "Lb": st["Lb"].numpy(), "zeta": st["zeta"],
             "r0a": st["r0a"], "r0b": st["r0b"], "omega_a": st["omega"][0],
             "omega_b": st["omega"][1]}
    return (o, v, J, eps, L), prob, st, state


@pytest.mark.parametrize("target", [("gradient", 0), ("coupling", 1, 0)], ids=str)
def test_multiplier_solve_matches_oracle(host_lib, mult_system, target):
    """The C-ABI multiplier solver (GMRES over the graph's reverse-over-forward
    Lagrangian gradient), run by the host test double of the device backend,
    against the oracle's dense solve: every gauge-free quantity and the
    Lagrangian densities."""
    from oracle import multipliers as mu
    B, lib = host_lib
    (o, v, J, eps, L), prob, st, state = mult_system
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    res = ctx.solve_multipliers(state, target, tol=1e-11, maxit=600)
    M = mu.solve_multipliers(prob, st, target)
    D1, G = mu.lagrangian_densities(prob, st, target, M)
    assert abs(res["gbar"] - float(M["gbar"])) < 1e-9
    assert np.abs(res["lb0"] - np.array([float(M["lb0a"]), float(M["lb0b"])])).max() < 1e-9
    # Ebar in the gauge Lbar_k . R_k = 0
    E = np.array([st["E0"] + st["omega"][0], st["E0"] + st["omega"][1]])
    d = np.array([1.0 if (target[0] == "gradient" and k == target[1]) else 0.0 for k in range(2)])
    lb0 = np.array([float(M["lb0a"]), float(M["lb0b"])])
    Eb = E * (d - lb0 * np.array([st["r0a"], st["r0b"]]))
    assert np.abs(res["Ebar"] - Eb).max() < 1e-8
    assert np.abs(res["zbar"] - M["zbar"].numpy()).max() < 1e-9
    for k in range(2):
        assert np.abs(res["K"][k] - M["K"][k].numpy()).max() < 1e-9
    assert np.abs(res["D1"] - D1.numpy()).max() < 1e-9
    assert np.abs(res["Gamma"] - G.numpy()).max() < 1e-9
    ctx.close()


def test_multiplier_residual_map_matches_oracle(host_lib, mult_system):
    """The stationarity map through the C ABI equals the oracle's at random
    unknowns (both the affine constant and the linear part)."""
    from oracle import multipliers as mu
    B, lib = host_lib
    (o, v, J, eps, L), prob, st, state = mult_system
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    for target in [("gradient", 1), ("coupling", 0, 1)]:
        f = mu.residual_map(prob, st, target)
        for seed in (0, 1):
            u = np.zeros(3 * prob.dim + 1) if seed == 0 else \
                np.random.default_rng(seed).normal(size=3 * prob.dim + 1)
            r = ctx.multiplier_residual(state, target, u)
            ro = f(torch.tensor(u)).numpy()
            assert np.abs(r - ro).max() < 1e-11 * max(1.0, np.abs(ro).max()), target
    ctx.close()
