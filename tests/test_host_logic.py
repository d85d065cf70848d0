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
    srcs = [os.path.join(CSRC, f) for f in ("graph.cpp", "ccsd_graph.cpp", "api.cpp")]
    srcs.append(os.path.join(ROOT, "tests", "host_executor", "host_backend.cpp"))
    cmd = ["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-I/usr/local/cuda/include",
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
