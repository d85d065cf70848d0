"""Host logic on the CPU: the C ABI exports, and the tensor-operation graph
with its forward/reverse differentiation, the solvers (ground state, Davidson,
the SCC loop, multipliers) and the argument checks run through the same C ABI
code with a loop-based test double of the device backend (tests/host_executor),
against the FP64 oracle and the stored values of tests/golden. The product
library itself always needs the GPU."""
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


def test_noalloc_size_checks_come_before_any_cuda_call():
    """sccsd_gemm_tn_noalloc rejects M*N above its fixed array, negative sizes
    and NULL pointers before it touches CUDA (so this runs without a GPU),
    including products M*N that overflow a 64-bit integer; empty outputs return
    OK at once."""
    from paper_2403_01007_gb300 import binding
    lib_path = binding.LIB_PATH
    if not os.path.exists(lib_path):
        from paper_2403_01007_gb300 import build
        build.build()
    lib = binding.load()
    cap = lib.sccsd_gemm_tn_noalloc_capacity()
    buf = (ctypes.c_double * 4)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    f = lib.sccsd_gemm_tn_noalloc
    # M * N = 2^64 wraps to 0; 2^20 * (2^44 + 1) wraps to exactly the capacity
    for (M, N) in [(1 << 21, 1 << 43), (1 << 20, (1 << 44) + 1), (cap, 2), (2, cap),
                   (1 << 62, 1 << 62)]:
        assert f(M, N, 16, 1.0, p, p, p, None) == -1, (M, N)
    assert f(-1, 2, 2, 1.0, p, p, p, None) == -1
    assert f(2, 2, -1, 1.0, p, p, p, None) == -1
    assert f(2, 2, 2, 1.0, None, p, p, None) == -1
    assert f(0, 5, 5, 1.0, p, p, p, None) == 0
    assert f(5, 0, 5, 1.0, p, p, p, None) == 0


@pytest.fixture(scope="module")
def host_lib():
    from paper_2403_01007_gb300 import binding
    tmp = tempfile.mkdtemp()
    so = os.path.join(tmp, "libsccsd_hostexec.so")
    srcs = [os.path.join(CSRC, f) for f in ("graph.cpp", "ccsd_graph.cpp", "api.cpp", "model.cpp",
                                            "solvers.cpp", "multipliers.cpp", "learned_api.cpp",
                                            "capture.cpp", "tc_tune.cpp")]
    srcs.append(os.path.join(ROOT, "tests", "host_executor", "host_backend.cpp"))
    # SCCSD_HOST_SANITIZE=1 builds the executor with AddressSanitizer to catch
    # out-of-range buffer use; run the tests with the sanitizer runtime and the
    # C++ runtime preloaded (LD_PRELOAD="$(gcc -print-file-name=libasan.so)
    # $(gcc -print-file-name=libstdc++.so)", ASAN_OPTIONS=detect_leaks=0), or
    # the first C++ exception trips the sanitizer's own interceptor
    san = ["-g", "-fsanitize=address", "-fno-omit-frame-pointer"] \
        if os.environ.get("SCCSD_HOST_SANITIZE") else []
    # -Bsymbolic: the double's own cudaMemcpyAsync (host memory only) must win
    # over a CUDA runtime that another library already loaded globally
    cmd = ["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-Wl,-Bsymbolic", *san,
           "-I/usr/local/cuda/include",
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


@pytest.mark.parametrize("size", [(2, 3, 6), (3, 4, 7)], ids=lambda s: "o%d_v%d" % s[:2])
def test_several_constrained_states_match_oracle(host_lib, size):
    """K of three states (Sec. 2.2; X_kl of Sec. 2.4.1 for every pair): the
    residual, A R with eta.R, A^T L and the densities through the C ABI with
    T + sum_kl zeta_kl X_kl against the oracle's sum over the pairs (which the
    determinant engine pins); with two states the call equals the two-state
    (zeta, Ra, Rb) call. The overlaps O_kl of every pair, natural and state
    projection over all three states, equal the oracle's (pinned against full
    determinant vectors). Bad arguments are refused."""
    from oracle import scc as sc
    B, lib = host_lib
    o, v, J = size
    eps, L = syn.system(o, v, J, 0.3, 91 + o + v)
    prob = cc.Problem(eps, L, o)
    t = syn.random_vectors(o, v, 1, 92, scale=0.1)[0]
    R3 = syn.random_vectors(o, v, 3, 93, normalise=True)
    Rt = syn.random_vectors(o, v, 2, 94, normalise=True)
    zeta = np.array([0.37, -0.21, 0.15])
    pairs = [(0, 1), (0, 2), (1, 2)]
    scct = [(float(z), torch.tensor(R3[k]), torch.tensor(R3[l])) for z, (k, l) in zip(zeta, pairs)]
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    e, om = ctx.residual_states(t, zeta, R3)
    E0, Om = rp.residual(prob, t, scc=scct)
    Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    assert abs(e - (float(E0) - Ehf)) < 1e-12
    assert np.abs(om - Om.numpy()).max() < 1e-12
    # the X3 terms are active: they move omega
    assert np.abs(om - rp.residual(prob, t)[1].numpy()).max() > 1e-3
    s, eta = ctx.jacobian_right(Rt, with_eta=True)
    sl = ctx.jacobian_left(Rt)
    for k in range(2):
        assert np.abs(s[k] - rp.jacobian_right(prob, t, Rt[k], scc=scct).numpy()).max() < 1e-12
        assert abs(eta[k] - float(rp.eta(prob, t, scc=scct) @ torch.tensor(Rt[k]))) < 1e-12
        assert np.abs(sl[k] - rp.jacobian_left(prob, t, Rt[k], scc=scct).numpy()).max() < 1e-12
    D1, G = ctx.densities(0.5, Rt[0], -0.2, Rt[1])
    D1r, Gr = rp.densities(prob, t, 0.5, Rt[0], -0.2, Rt[1], scc=scct)
    assert np.abs(D1 - D1r.numpy()).max() < 1e-12
    assert np.abs(G - Gr.numpy()).max() < 1e-12
    # n = 2 is the two-state call
    e2, om2 = ctx.residual_states(t, [0.4], R3[:2])
    e2p, om2p = ctx.residual(t, scc=(0.4, R3[0], R3[1]))
    assert abs(e2 - e2p) < 1e-13
    assert np.abs(om2 - om2p).max() < 1e-13
    # back to three states after the model for two was used
    e3, om3 = ctx.residual_states(t, zeta, R3)
    assert np.abs(om3 - om).max() < 1e-13
    # the ground solve with the three-state terms reaches Omega = 0 of the oracle's residual
    eg, tg, _ = ctx.solve_ground_states(0.1 * zeta, R3, tol=1e-11, maxit=300)
    sccg = [(0.1 * z, x, y) for z, x, y in scct]
    assert np.abs(rp.residual(prob, tg, scc=sccg)[1].numpy()).max() < 1e-10
    # bad arguments: one state, NULL vectors, non-finite zeta
    d = prob.dim
    buf = np.zeros(3 * d)
    z3 = np.zeros(3)
    assert lib.sccsd_residual_states(ctx.h, buf.ctypes.data, 1, z3.ctypes.data, buf.ctypes.data,
                                     None, None) == -1
    assert lib.sccsd_residual_states(ctx.h, buf.ctypes.data, 3, z3.ctypes.data, None, None,
                                     None) == -1
    z3[1] = np.nan
    assert lib.sccsd_residual_states(ctx.h, buf.ctypes.data, 3, z3.ctypes.data, buf.ctypes.data,
                                     None, None) == -1
    # the overlaps of every pair, both projections, against the oracle
    r0 = np.array([0.3, -0.2, 0.1])
    ctx.residual(t)
    states = [(float(r0[k]), torch.tensor(R3[k])) for k in range(3)]
    for proj in ("natural", "state"):
        got = ctx.overlaps(r0, R3, proj)
        ref = sc.overlaps(torch.tensor(t), states, o, v, proj)
        for kl, val in ref.items():
            assert abs(got[kl] - float(val)) < 1e-12 * max(1.0, abs(float(val))), (proj, kl)
    # two states: the pair calls
    two = ctx.overlaps(r0[:2], R3[:2], "state")
    assert abs(two[(0, 1)] - ctx.overlap_states(r0[0], R3[0], r0[1], R3[1])) < 1e-13
    assert abs(ctx.overlaps(r0[:2], R3[:2])[(0, 1)] - ctx.overlap(r0[0], R3[0], r0[1], R3[1])) < 1e-13
    # linearly dependent states are refused under the state projection
    Rd = np.stack([R3[0], R3[1], 2.0 * R3[0]])
    assert lib.sccsd_overlaps(ctx.h, 3, np.array([0.3, -0.2, 0.6]).ctypes.data, Rd.ctypes.data, 1,
                              np.zeros(3).ctypes.data) == -1
    assert lib.sccsd_overlaps(ctx.h, 1, r0.ctypes.data, R3.ctypes.data, 0,
                              np.zeros(3).ctypes.data) == -1
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


# ------------------------------------------- launch-shape tuning (host part)

def _default_rule(M, n_pad, nk, sm, ab, bb):
    """The fixed launch rule of the tensor-core contraction, written out: K is
    split only when the output tiles (128 x 256) cannot fill the SMs and there
    are at least 8 K blocks, into ranges of at least 4 blocks, and only when
    the split grid's waves per unit of work are at most 0.85 of the unsplit
    grid's; N tiles are walked fastest when A is more than four times larger
    than B; the eight-warp variant serves items of at most 16 K blocks."""
    mt, nt = -(-M // 128), n_pad // 256
    tiles = mt * nt
    want = min(-(-2 * sm // tiles), nk // 4) if (tiles < sm and nk >= 8) else 1
    if want > 1 and (-(-want * tiles // sm)) / want > 0.85 * (-(-tiles // sm)):
        want = 1
    if want <= 1:
        splits, kbs = 1, nk
    else:
        kbs = -(-nk // want)
        splits = -(-nk // kbs)
    return (1 if kbs <= 16 else 0, 1 if (nt > 1 and ab > 4 * bb) else 0, splits, kbs)


TUNE_SHAPES = [
    (2646, 40192, 625, 152, 2688 * 40000, 40192 * 40000),   # ladder, 6 vectors, o=21 v=200
    (100000, 256, 1, 152, 100096 * 64, 256 * 64),           # skinny, K = o
    (126, 256, 1313, 152, 128 * 84032, 256 * 84032),        # one output tile, long K
    (5000, 768, 11, 152, 5120 * 704, 768 * 704),            # few tiles, short K
    (40000, 512, 2, 152, 40064 * 128, 512 * 128),           # A much larger than B
    (1386, 3328, 315, 152, 1408 * 20160, 3328 * 20160),     # ladder chunk: 143 tiles, one wave
    (1200, 2560, 300, 152, 1280 * 19200, 2560 * 19200),     # 100 tiles: a split of 4 pays
]


def test_autotune_candidates_follow_the_launch_rules():
    tmp = tempfile.mkdtemp()
    exe = os.path.join(tmp, "tc_tune_main")
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, os.path.join(CSRC, "tc_tune.cpp"),
                        os.path.join(ROOT, "tests", "host_executor", "tc_tune_main.cpp"), "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("host toolchain unavailable: " + r.stderr[-300:])
    args = [str(x) for s in TUNE_SHAPES for x in s]
    out = subprocess.run([exe, *args], capture_output=True, text=True, check=True).stdout
    blocks = out.split("\n\n")
    for shape, block in zip(TUNE_SHAPES, blocks):
        M, n_pad, nk = shape[:3]
        nt = n_pad // 256
        cands = [tuple(int(x) for x in line.split()) for line in block.strip().splitlines()]
        assert cands[0][:4] == _default_rule(*shape), shape
        assert all(c[4] == 1 for c in cands), shape
        assert len(set(c[:4] for c in cands)) == len(cands), shape
        assert any(c[2] == 1 and c[3] == nk for c in cands), shape
        for variant, nfast, splits, kbs, _ in cands:
            assert variant in (0, 1)
            assert nfast == 0 or nt > 1
            if splits > 1:
                assert kbs >= 4 and splits == -(-nk // kbs) and nk >= 8
            else:
                assert kbs == nk
    # one output tile over 1313 K blocks: no split, half the default number of
    # ranges (120 ranges of 11 blocks) and the default (263 ranges of 5, which
    # is also the finest split with at least 4 blocks per range), each with
    # either kernel form
    cands = [tuple(int(x) for x in l.split()) for l in blocks[2].strip().splitlines()]
    assert {(c[2], c[3]) for c in cands} == {(1, 1313), (120, 11), (263, 5)}
    assert {(c[0], c[2]) for c in cands} == {(v, s) for v in (0, 1) for s in (1, 120, 263)}


def test_autotune_table_text(host_lib):
    B, lib = host_lib
    B.autotune_clear(lib)
    assert B.autotune_entries(lib) == 0
    good = ("2646 40192 625 1 0 152 12345 0 0 1 625 5100.000\n"
            "126 256 1313 1 1 152 99 0 0 263 5 80.500\n")
    B.autotune_import(good, lib)
    assert B.autotune_entries(lib) == 2
    text = B.autotune_export(lib)
    rows = sorted(tuple(l.split()[:11]) for l in text.strip().splitlines())
    assert rows == sorted(tuple(l.split()[:11]) for l in good.strip().splitlines())
    B.autotune_import(text, lib)                      # re-import is idempotent
    assert B.autotune_entries(lib) == 2
    B.autotune_import("126 256 1313 1 1 152 99 1 0 263 5 1.0", lib)   # eight-warp form, 5 blocks
    assert B.autotune_entries(lib) == 2                                 # replaces the entry
    B.autotune_import(good, lib)
    bad = [
        "126 256 1313 1 1 152 99 2 0 263 5 1.0",      # no third kernel form
        "126 256 1313 1 1 152 99 0 0 200 5 1.0",      # split count does not cover K
        "126 256 1313 1 1 152 99 0 1 263 5 1.0",      # N-fastest with one N tile
        "2646 40192 625 1 0 152 1 0 0 1 600 1.0",     # unsplit but K range != K
        "2646 40000 625 1 0 152 1 0 0 1 625 1.0",     # N not padded to 256
        "2646 40192 625 3 0 152 1 0 0 1 625 1.0",     # three slices
        "1 2 3",
        "2646 40192 625 1 0 152 1 0 0 1 625 1.0 extra",
        "9999 256 1 1 0 152 7 1 0 1 1 2.0\n126 256 1313 1 1 152 99 0 0 200 5 1.0",
    ]
    for b in bad:
        with pytest.raises(B.SccsdError) as ei:
            B.autotune_import(b, lib)
        assert ei.value.code == -1, b
        assert B.autotune_entries(lib) == 2, b        # all or nothing
    assert lib.sccsd_autotune_import(None) == -1
    n = ctypes.c_longlong()
    small = ctypes.create_string_buffer(3)
    assert lib.sccsd_autotune_export(small, 3, ctypes.byref(n)) == -1
    assert n.value == len(text) + 1
    B.autotune_clear(lib)
    assert B.autotune_entries(lib) == 0


def test_set_autotune_arguments(host_lib):
    B, lib = host_lib
    eps = np.linspace(-1, 1, 4)
    L = np.zeros((2, 4, 4))
    ctx = B.Context(2, 2, 2, eps, L, lib=lib)
    ctx.set_autotune(True)
    ctx.set_autotune(False)
    assert lib.sccsd_set_autotune(ctx.h, 2) == -1
    assert lib.sccsd_set_autotune(None, 1) == -1
    ctx.close()


def test_transform_edge_cases(host_lib):
    """Empty batches, zero vectors and linearity of the Jacobian transforms
    through the C ABI (A R is linear in R, Sec. 2.1)."""
    B, lib = host_lib
    o, v, J = 2, 3, 6
    eps, L = syn.system(o, v, J, 0.3, 91)
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    t = syn.random_vectors(o, v, 1, 92, scale=0.1)[0]
    ctx.residual(t)
    assert lib.sccsd_jacobian_right(ctx.h, 0, None, None, None) == 0
    assert lib.sccsd_jacobian_left(ctx.h, 0, None, None) == 0
    assert lib.sccsd_jacobian_right(ctx.h, -1, None, None, None) == -1
    assert lib.sccsd_jacobian_left(ctx.h, -1, None, None) == -1
    Z = np.zeros((2, ctx.dim))
    s, eta = ctx.jacobian_right(Z, with_eta=True)
    assert not s.any() and not np.any(eta)
    assert not ctx.jacobian_left(Z).any()
    R1, R2 = syn.random_vectors(o, v, 2, 93, normalise=True)
    a, b = 0.7, -1.9
    s = ctx.jacobian_right(np.stack([R1, R2, a * R1 + b * R2]))
    assert np.abs(s[2] - (a * s[0] + b * s[1])).max() < 1e-13
    sl = ctx.jacobian_left(np.stack([R1, R2, a * R1 + b * R2]))
    assert np.abs(sl[2] - (a * sl[0] + b * sl[1])).max() < 1e-13
    ctx.close()


def test_autotune_candidates_random_shapes():
    """The candidate rules on 300 seeded random shapes (M up to 10^6, N up to
    64 tiles, 1 to 2000 K blocks, operands of any relative size)."""
    tmp = tempfile.mkdtemp()
    exe = os.path.join(tmp, "tc_tune_main")
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, os.path.join(CSRC, "tc_tune.cpp"),
                        os.path.join(ROOT, "tests", "host_executor", "tc_tune_main.cpp"), "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("host toolchain unavailable: " + r.stderr[-300:])
    rng = np.random.default_rng(2024)
    shapes = []
    for _ in range(300):
        M = int(rng.integers(1, 10 ** int(rng.integers(1, 7)) + 1))
        n_pad = 256 * int(rng.integers(1, 65))
        nk = int(rng.integers(1, 2001))
        ab = float((-(-M // 128) * 128) * nk * 64)
        bb = float(n_pad * nk * 64)
        shapes.append((M, n_pad, nk, 152, ab, bb))
    args = [str(x) for s in shapes for x in s]
    out = subprocess.run([exe, *args], capture_output=True, text=True, check=True).stdout
    blocks = out.split("\n\n")
    for shape, block in zip(shapes, blocks):
        M, n_pad, nk = shape[:3]
        nt = n_pad // 256
        cands = [tuple(int(x) for x in line.split()) for line in block.strip().splitlines()]
        assert cands and cands[0][:4] == _default_rule(*shape), shape
        assert all(c[4] == 1 for c in cands), shape
        assert len(set(c[:4] for c in cands)) == len(cands), shape
        assert any(c[2] == 1 and c[3] == nk for c in cands), shape
        assert all(c[1] == 0 for c in cands) if nt == 1 else any(c[1] == 1 for c in cands)
        assert len(cands) <= 20


@pytest.mark.parametrize("size", [(2, 3, 6), (3, 4, 7)], ids=lambda s: "o%d_v%d" % s[:2])
@pytest.mark.parametrize("with_scc", [False, True], ids=["ccsd", "sccsd"])
def test_overlap_and_state_through_the_c_abi(host_lib, size, with_scc):
    """O_ab of the natural projection (Sec. 2.4.1) through the C ABI equals the
    oracle's, is symmetric in a and b, and uses T without zeta X3; the state
    amplitudes read back are those of the last residual call."""
    B, lib = host_lib
    from oracle import scc as sc
    o, v, J = size
    eps, L = syn.system(o, v, J, 0.3, 61 + o)
    t = syn.random_vectors(o, v, 1, 62, scale=0.1)[0]
    Ra, Rb = syn.random_vectors(o, v, 2, 63, normalise=True)
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    ctx.residual(t, scc=(0.37, Ra, Rb) if with_scc else None)
    O = ctx.overlap(0.3, Ra, -0.2, Rb)
    ref = float(sc.overlap(torch.tensor(t), 0.3, torch.tensor(Ra), -0.2, torch.tensor(Rb), o, v))
    assert abs(O - ref) < 1e-13 * max(1.0, abs(ref))
    assert abs(ctx.overlap(-0.2, Rb, 0.3, Ra) - O) < 1e-13 * max(1.0, abs(O))
    assert np.array_equal(ctx.state_amplitudes(), t)
    ctx.close()


def test_every_documented_argument_error(host_lib):
    """The SCCSD_EINVAL (-1) and SCCSD_ESTATE (-4) cases the header documents,
    through the C ABI before any device work, each leaving a message in
    sccsd_last_error."""
    B, lib = host_lib
    nan = float("nan")
    lib.sccsd_strerror.argtypes = [ctypes.c_int]
    lib.sccsd_strerror.restype = ctypes.c_char_p
    assert lib.sccsd_strerror(-1) == b"invalid argument"
    texts = {lib.sccsd_strerror(code) for code in range(0, -8, -1)}
    assert len(texts) == 8 and all(texts)          # one distinct text per code
    lib.sccsd_destroy(None)                        # a NULL context is ignored
    assert lib.sccsd_last_error(None)
    one = np.zeros(4)
    P = one.ctypes.data
    assert lib.sccsd_gemm_tn(0, -1, 2, 2, 1.0, P, P, P, None) == -1
    assert lib.sccsd_gemm_tn(3, 2, 2, 2, 1.0, P, P, P, None) == -1
    assert lib.sccsd_gemm_tn(0, 0, 2, 2, 1.0, P, P, P, None) == 0     # empty C
    assert lib.sccsd_gemm_tn(0, 2, 2, 2, 1.0, P, P, P, None) == -1    # host pointers
    h = ctypes.c_void_p()
    eps = np.linspace(-1.0, 1.0, 5)
    L = np.zeros((3, 5, 5))
    assert lib.sccsd_init(None, 2, 3, 3, eps.ctypes.data, L.ctypes.data, 0, None) == -1
    assert lib.sccsd_init(ctypes.byref(h), 2, 3, 3, eps.ctypes.data, L.ctypes.data, 3, None) == -1
    assert lib.sccsd_init(ctypes.byref(h), 2, 0, 3, eps.ctypes.data, L.ctypes.data, 0, None) == -1
    o, v, J = 2, 3, 6
    eps, L = syn.system(o, v, J, 0.3, 71)
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    d = ctx.dim
    x = np.zeros(d)
    X = x.ctypes.data
    out = np.zeros(4 * d + 1)
    Y = out.ctypes.data
    n = o + v
    D1 = np.zeros((n, n))
    zi = ctypes.c_int()
    zd = ctypes.c_double()

    def expect(code, rc):
        assert rc == code, rc
        assert lib.sccsd_last_error(ctx.h)

    # before any state
    expect(-4, lib.sccsd_jacobian_left(ctx.h, 1, X, Y))
    expect(-4, lib.sccsd_densities(ctx.h, 1.0, X, 0.0, X, D1.ctypes.data, None))
    expect(-4, lib.sccsd_overlap(ctx.h, 0.0, X, 0.0, X, ctypes.addressof(zd)))
    expect(-4, lib.sccsd_state_amplitudes(ctx.h, Y))
    expect(-4, lib.sccsd_solve_states(ctx.h, 1, 0, 1e-8, 10, 0.0, Y, None, None))
    # residual arguments
    expect(-1, lib.sccsd_residual(ctx.h, None, 0.0, None, None, None, None))
    expect(-1, lib.sccsd_residual(ctx.h, X, 0.0, X, None, None, None))
    expect(-1, lib.sccsd_residual(ctx.h, X, nan, X, X, None, None))
    assert lib.sccsd_residual(ctx.h, X, 0.0, None, None, None, None) == 0
    # transforms, densities, overlap, state
    expect(-1, lib.sccsd_jacobian_right(ctx.h, 1, None, Y, None))
    expect(-1, lib.sccsd_densities(ctx.h, 1.0, None, 0.0, X, D1.ctypes.data, None))
    expect(-1, lib.sccsd_densities(ctx.h, nan, X, 0.0, X, D1.ctypes.data, None))
    expect(-1, lib.sccsd_overlap(ctx.h, 0.0, None, 0.0, X, ctypes.addressof(zd)))
    expect(-1, lib.sccsd_state_amplitudes(ctx.h, None))
    expect(-1, lib.sccsd_set_precision(ctx.h, 3))
    # solvers
    expect(-1, lib.sccsd_solve_ground(ctx.h, None, 0.0, None, None, 0.0, 10, 0.0, None, None, None))
    expect(-1, lib.sccsd_solve_ground(ctx.h, None, 0.0, None, None, 1e-8, 0, 0.0, None, None, None))
    expect(-1, lib.sccsd_solve_ground(ctx.h, None, 0.0, X, None, 1e-8, 10, 0.0, None, None, None))
    for nroots, side, tol, maxit, om in [(0, 0, 1e-8, 10, Y), (13, 0, 1e-8, 10, Y),
                                         (1, 2, 1e-8, 10, Y), (1, 0, 0.0, 10, Y),
                                         (1, 0, 1e-8, 0, Y), (1, 0, 1e-8, 10, None)]:
        expect(-1, lib.sccsd_solve_states(ctx.h, nroots, side, tol, maxit, 0.0, om, None, None))
    for args in [(0.0, 10, 1e-8, 1e-8), (1e-8, 0, 1e-8, 1e-8), (1e-8, 10, 0.0, 1e-8),
                 (1e-8, 10, 1e-8, -1.0)]:
        expect(-1, lib.sccsd_solve_scc(ctx.h, *args, None, None, None, None, None, None, None))
    # multipliers: bad targets and NULL inputs
    vecs = np.zeros(5 * d)
    scal = np.zeros(5)
    u = np.zeros(3 * d + 1)
    for kind, m, nn in [(0, 0, 2), (1, 0, 0), (1, 2, 0), (2, 0, 1)]:
        expect(-1, lib.sccsd_solve_multipliers(ctx.h, vecs.ctypes.data, scal.ctypes.data, kind, m,
                                               nn, 1e-8, 10, 0.0, None, None, None, None, None,
                                               ctypes.addressof(zi)))
        expect(-1, lib.sccsd_multiplier_residual(ctx.h, vecs.ctypes.data, scal.ctypes.data, kind,
                                                 m, nn, u.ctypes.data, Y))
    expect(-1, lib.sccsd_solve_multipliers(ctx.h, None, scal.ctypes.data, 0, 0, 0, 1e-8, 10, 0.0,
                                           None, None, None, None, None, None))
    expect(-1, lib.sccsd_multiplier_residual(ctx.h, vecs.ctypes.data, scal.ctypes.data, 0, 0, 0,
                                             None, Y))
    # derivative assembly: NULL inputs, or Gamma without its perturbation
    D1 = np.zeros((n, n))
    expect(-1, lib.sccsd_integral_derivative(ctx.h, None, None, D1.ctypes.data, None,
                                             ctypes.addressof(zd)))
    expect(-1, lib.sccsd_integral_derivative(ctx.h, D1.ctypes.data, D1.ctypes.data,
                                             D1.ctypes.data, None, ctypes.addressof(zd)))
    expect(-1, lib.sccsd_input_derivative(ctx.h, D1.ctypes.data, None, None, None,
                                          ctypes.addressof(zd)))
    ctx.close()


# ------------------------------------ solvers through the C ABI (host double)

def _golden(name):
    import json
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        return json.load(f)


@pytest.mark.parametrize("with_scc", [False, True], ids=["ccsd", "sccsd"])
def test_ground_solver_through_the_c_abi(host_lib, with_scc):
    """sccsd_solve_ground (Jacobi + DIIS with dressed denominators, the
    solver's own control flow) reaches the oracle's ground state (Sec. 2.1),
    with the SCC term at fixed zeta, R_a, R_b (Sec. 2.4.2)."""
    from oracle import solvers as sv
    B, lib = host_lib
    o, v, J = 3, 4, 9
    eps, L = syn.system(o, v, J, 0.2, 55)
    prob = cc.Problem(eps, L, o)
    Ra, Rb = syn.random_vectors(o, v, 2, 56, normalise=True)
    scc = (0.3, Ra, Rb) if with_scc else None
    scct = (0.3, torch.tensor(Ra), torch.tensor(Rb)) if with_scc else None
    x, E0, _ = sv.ground_state(prob, tol=1e-12, scc=scct)
    Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    e, t, it = ctx.solve_ground(tol=1e-11, maxit=200, scc=scc)
    assert abs(e - (E0 - Ehf)) < 1e-10
    assert np.abs(t - x).max() < 1e-9
    assert 0 < it < 200
    ctx.close()


@pytest.mark.parametrize("side", ["right", "left"])
def test_davidson_through_the_c_abi(host_lib, side):
    """sccsd_solve_states (Davidson with restarts and the device-side subspace
    eigenproblem, here the test double's) returns the lowest roots of the dense
    Jacobian (Sec. 2.1), with unit vectors that satisfy their eigen-equations."""
    from oracle import solvers as sv
    B, lib = host_lib
    o, v, J = 3, 4, 9
    eps, L = syn.system(o, v, J, 0.2, 55)
    prob = cc.Problem(eps, L, o)
    x, _, _ = sv.ground_state(prob, tol=1e-12)
    wd, _ = sv.eom_dense(prob, x, 3, side=side)
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    ctx.residual(x)
    w, V, it = ctx.solve_states(3, side=side, tol=1e-9)
    assert np.abs(w - wd).max() < 1e-9
    op = ctx.jacobian_right if side == "right" else ctx.jacobian_left
    AV = op(np.ascontiguousarray(V))
    for k in range(3):
        assert abs(np.linalg.norm(V[k]) - 1.0) < 1e-12
        assert np.linalg.norm(AV[k] - w[k] * V[k]) < 1e-8
    ctx.close()


def test_expired_device_wait_maps_to_ecuda_and_the_context_recovers(host_lib):
    """An expired bounded wait in a tensor-core kernel is recorded in the
    kernel's error flag and raised by the backend at the next synchronisation
    (the device kernels never trap). The C ABI reports it as SCCSD_ECUDA with
    the wait text in sccsd_last_error, and the context stays usable: the next
    call gives the oracle's result. The expiry is injected on the host (the
    test double raises the backend's error at a chosen synchronisation)."""
    B, lib = host_lib
    o, v, J = 2, 3, 6
    eps, L = syn.system(o, v, J, 0.3, 4)
    prob = cc.Problem(eps, L, o)
    x = syn.random_vectors(o, v, 1, 5, scale=0.1)[0]
    R = syn.random_vectors(o, v, 2, 6, normalise=True)
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    ctx.residual(x)
    os.environ["SCCSD_HOST_FAKE_WAIT_EXPIRY"] = "0"
    try:
        with pytest.raises(B.SccsdError) as ei:
            ctx.jacobian_right(R)
    finally:
        del os.environ["SCCSD_HOST_FAKE_WAIT_EXPIRY"]
    assert ei.value.code == -3
    assert "wait expired" in str(ei.value)
    sig = ctx.jacobian_right(R)
    for k in range(2):
        ref = rp.jacobian_right(prob, x, R[k]).numpy()
        assert np.abs(sig[k] - ref).max() < 1e-12
    ctx.close()


def test_left_normalisation_through_the_c_abi(host_lib):
    """sccsd_normalize_left scales each left eigenvector so that <L_k|R_k> = 1
    (Sec. 2.1; the plain dot product in the biorthonormal bra basis). Checked
    on the Davidson roots of both sides: after scaling, L_k . R_l is the
    identity (left and right vectors of distinct roots are biorthogonal), and
    the left vectors still satisfy their eigen-equation. Zero products and
    NULL pointers are rejected; nvec = 0 is a no-op."""
    from oracle import solvers as sv
    B, lib = host_lib
    o, v, J = 3, 4, 9
    eps, L = syn.system(o, v, J, 0.2, 55)
    prob = cc.Problem(eps, L, o)
    x, _, _ = sv.ground_state(prob, tol=1e-12)
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    ctx.residual(x)
    wr, VR, _ = ctx.solve_states(3, side="right", tol=1e-10)
    wl, VL, _ = ctx.solve_states(3, side="left", tol=1e-10)
    assert np.abs(wr - wl).max() < 1e-9
    raw = VL.copy()
    out = ctx.normalize_left(VR, VL)
    S = out @ VR.T
    assert np.abs(S - np.eye(3)).max() < 1e-7
    for k in range(3):
        # the same direction, only rescaled by 1 / (L_k . R_k)
        assert np.abs(out[k] - raw[k] / (raw[k] @ VR[k])).max() < 1e-13
    AL = ctx.jacobian_left(np.ascontiguousarray(out))
    for k in range(3):
        assert np.linalg.norm(AL[k] - wl[k] * out[k]) < 1e-7 * np.linalg.norm(out[k])
    # errors: a left vector orthogonal to its right vector, NULL, nvec < 0
    Z = np.zeros((1, ctx.dim))
    with pytest.raises(B.SccsdError) as ei:
        ctx.normalize_left(VR[:1].copy(), Z)
    assert ei.value.code == -1
    assert lib.sccsd_normalize_left(ctx.h, 1, None, None) == -1
    assert lib.sccsd_normalize_left(ctx.h, -1, None, None) == -1
    assert lib.sccsd_normalize_left(ctx.h, 0, None, None) == 0
    ctx.close()


def test_scc_loop_through_the_c_abi(host_lib):
    """sccsd_solve_scc (ground state and two roots re-converged at each zeta,
    secant on O_ab; Sec. 2.2, 2.4) on a system with an active constraint
    reaches the stored oracle solution, and the oracle's O_ab vanishes at the
    returned states."""
    from oracle import scc as sc
    B, lib = host_lib
    g = _golden("scc_active_o3_v8.json")
    p = g["inputs"]
    eps, L = syn.system(p["o"], p["v"], p["J"], p["sd"], p["seed"])
    ctx = B.Context(p["o"], p["v"], p["J"], eps, L, lib=lib)
    r = ctx.solve_scc(tol=1e-10)
    t = ctx.state_amplitudes()
    ctx.close()
    assert abs(r["zeta"] - g["values"]["zeta"]) < 1e-7
    assert np.abs(r["omega"] - np.array(g["values"]["omega"])).max() < 1e-8
    assert abs(r["e_corr"] - g["values"]["e_corr"]) < 1e-9
    O = float(sc.overlap(torch.tensor(t), r["r0"][0], torch.tensor(r["Ra"]), r["r0"][1],
                         torch.tensor(r["Rb"]), p["o"], p["v"]))
    assert abs(O) < 1e-9
    assert abs(r["zeta"]) > 0.3           # the constraint is active


def test_four_constrained_states_and_refined_ground_solve(host_lib):
    """Four states (six pairs) through the several-states model: the residual
    and A R against the oracle's sum over the six pairs; and the ground solve
    with these terms in the emulated split-BF16 precision with FP64 refinement
    zeroes the oracle's FP64 residual."""
    B, lib = host_lib
    o, v, J = 2, 4, 8
    eps, L = syn.system(o, v, J, 0.3, 97)
    prob = cc.Problem(eps, L, o)
    t = syn.random_vectors(o, v, 1, 98, scale=0.1)[0]
    R4 = syn.random_vectors(o, v, 4, 99, normalise=True)
    Rt = syn.random_vectors(o, v, 1, 100, normalise=True)
    pairs = [(k, l) for k in range(4) for l in range(k + 1, 4)]
    zeta = np.array([0.21, -0.13, 0.08, 0.17, -0.05, 0.11])
    scct = [(float(z), torch.tensor(R4[k]), torch.tensor(R4[l])) for z, (k, l) in zip(zeta, pairs)]
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    _, om = ctx.residual_states(t, zeta, R4)
    assert np.abs(om - rp.residual(prob, t, scc=scct)[1].numpy()).max() < 1e-12
    s = ctx.jacobian_right(Rt)
    assert np.abs(s[0] - rp.jacobian_right(prob, t, Rt[0], scc=scct).numpy()).max() < 1e-12
    ctx.close()
    ctx = B.Context(o, v, J, eps, L, precision="bf16x3", lib=lib)
    z = 0.5 * zeta
    _, tg, _ = ctx.solve_ground_states(z, R4, tol=1e-10, maxit=300, refine_tol=1e-5)
    sccg = [(0.5 * zz, x, y) for zz, x, y in scct]
    assert np.linalg.norm(rp.residual(prob, tg, scc=sccg)[1].numpy()) < 1e-9
    ctx.close()


@pytest.mark.parametrize("fixture", ["scc_active_o3_v8.json", "scc_state_projection_o3_v8.json"],
                         ids=["natural", "state"])
def test_broyden_loop_of_several_states_with_two_states_is_the_two_state_solution(host_lib,
                                                                                  fixture):
    """sccsd_solve_scc_states with n = 2 runs the several-states model (one
    X3 term per state) and Broyden's update, which for one unknown is the
    secant step of the two-state loop (the oracle's loops are pinned to agree,
    tests/test_oracle_pins.py): it reaches the stored oracle solutions of the
    active two-state system, natural and state projection, with O_01 = 0 of
    the oracle at the returned state."""
    from oracle import scc as sc
    B, lib = host_lib
    g = _golden(fixture)
    p = g["inputs"]
    eps, L = syn.system(p["o"], p["v"], p["J"], p["sd"], p["seed"])
    ctx = B.Context(p["o"], p["v"], p["J"], eps, L, lib=lib)
    ctx.set_projection(p["projection"])
    r = ctx.solve_scc_states(2, tol=1e-10)
    t = ctx.state_amplitudes()
    ctx.close()
    assert abs(r["zeta"][(0, 1)] - g["values"]["zeta"]) < 1e-7
    assert np.abs(r["omega"] - np.array(g["values"]["omega"])).max() < 1e-8
    assert abs(r["e_corr"] - g["values"]["e_corr"]) < 1e-9
    ovl = sc.overlap_states if p["projection"] == "state" else sc.overlap
    O = float(ovl(torch.tensor(t), r["r0"][0], torch.tensor(r["R"][0]), r["r0"][1],
                  torch.tensor(r["R"][1]), p["o"], p["v"]))
    assert abs(O) < 1e-9 and abs(r["O"][(0, 1)]) < 1e-9


@pytest.mark.parametrize("fixture", ["scc_three_states_o3_v6.json",
                                     "scc_three_states_state_projection_o3_v6.json"],
                         ids=["natural", "state"])
def test_three_constrained_states_reach_the_oracle_solution(host_lib, fixture):
    """sccsd_solve_scc_states with three states on the two-irrep system (the
    stored oracle solutions, Sec. 2.2 with K of three states, natural and
    state projection over all three): the active pair (0, 2) has the oracle's
    zeta, the pairs of different symmetry stay at zeta = 0 (Sec. 3.1.1), the
    energies agree, and every O_kl of the oracle vanishes at the returned
    state."""
    from oracle import scc as sc
    B, lib = host_lib
    g = _golden(fixture)
    p = g["inputs"]
    eps, L, _, _ = syn.symmetric_system(p["o"], p["v"], p["J"], p["sd"], p["seed"],
                                        p["irrep_occ"], p["irrep_vir"])
    ctx = B.Context(p["o"], p["v"], p["J"], eps, L, lib=lib)
    ctx.set_projection(p["projection"])
    r = ctx.solve_scc_states(3, tol=1e-10, ground_tol=1e-11, eom_tol=1e-9)
    t = ctx.state_amplitudes()
    ctx.close()
    pairs = [(0, 1), (0, 2), (1, 2)]
    for kl, z in zip(pairs, g["values"]["zeta"]):
        assert abs(r["zeta"][kl] - z) < 1e-7, kl
    assert abs(r["zeta"][(0, 2)]) > 0.3
    assert np.abs(r["omega"] - np.array(g["values"]["omega"])).max() < 1e-8
    assert abs(r["e_corr"] - g["values"]["e_corr"]) < 1e-9
    O = sc.overlaps(torch.tensor(t), [(r["r0"][k], torch.tensor(r["R"][k])) for k in range(3)],
                    p["o"], p["v"], p["projection"])
    for kl in pairs:
        assert abs(float(O[kl])) < 1e-9, kl


def test_davidson_on_small_systems_is_full_ci_for_two_electrons(host_lib):
    """The subspace shrinks to the problem (min(48, dim) vectors): for two
    electrons (o=1, v=5, dim 20) the Davidson roots through the C ABI are the
    stored full-CI excitation energies (CCSD is exact, Sec. 2.1); a request
    that leaves no room for 2 nroots + 2 vectors is refused."""
    B, lib = host_lib
    g = _golden("fci_two_electron_o1_v5.json")
    p = g["inputs"]
    eps, L = syn.system(p["o"], p["v"], p["J"], p["sd"], p["seed"])
    ctx = B.Context(p["o"], p["v"], p["J"], eps, L, lib=lib)
    e, _, _ = ctx.solve_ground(tol=1e-12, maxit=300)
    assert abs(e - g["values"]["e_corr"]) < 1e-10
    for side in ("right", "left"):
        w, _, _ = ctx.solve_states(3, side=side, tol=1e-10)
        assert np.abs(w - np.array(g["values"]["excitation_energies"][:3])).max() < 1e-9, side
    with pytest.raises(B.SccsdError) as ei:
        ctx.solve_states(10)              # 22 vectors > dim 20
    assert ei.value.code == -1
    ctx.close()


def test_whole_method_through_the_c_abi(host_lib):
    """The chain of the method on the CPU test double, on the system with an
    active constraint: the SCCSD state (sccsd_solve_scc and the left roots),
    then the multipliers of a gradient and of a coupling (Sec. 2.3). The
    oracle's stationarity equations vanish at the C-ABI solution, and the
    effective one-particle densities have trace 2o (the gradient of E with
    respect to a uniform shift of h counts the electrons) and 0 (a coupling)."""
    from oracle import multipliers as mu
    B, lib = host_lib
    g = _golden("scc_active_o3_v8.json")
    p = g["inputs"]
    o = p["o"]
    eps, L = syn.system(o, p["v"], p["J"], p["sd"], p["seed"])
    prob = cc.Problem(eps, L, o)
    ctx = B.Context(o, p["v"], p["J"], eps, L, lib=lib)
    state = ctx.scc_state(tol=1e-10, ground_tol=1e-11, eom_tol=1e-9, left_tol=1e-9)
    assert abs(state["zeta"] - g["values"]["zeta"]) < 1e-7
    st = {"t": torch.tensor(state["t"]), "Ra": torch.tensor(state["Ra"]),
          "Rb": torch.tensor(state["Rb"]), "La": torch.tensor(state["La"]),
          "Lb": torch.tensor(state["Lb"]), "zeta": state["zeta"], "r0a": state["r0a"],
          "r0b": state["r0b"], "omega": (state["omega_a"], state["omega_b"])}
    Ehf = float(cc.energy_residual(torch.zeros(prob.dim, dtype=torch.float64), prob)[0])
    st["E0"] = Ehf + state["e_corr"]
    dim = prob.dim
    for target, trace in [(("gradient", 0), 2.0 * o), (("coupling", 0, 1), 0.0)]:
        res = ctx.solve_multipliers(state, target, tol=1e-10, maxit=800)
        assert abs(np.trace(res["D1"]) - trace) < 1e-8, target
        d = [1.0 if (target[0] == "gradient" and k == target[1]) else 0.0 for k in range(2)]
        r0 = [state["r0a"], state["r0b"]]
        lam = [state["La"], state["Lb"]]
        Lbar = [res["K"][k] - (d[k] - res["lb0"][k] * r0[k]) * lam[k] for k in range(2)]
        u = np.concatenate([res["zbar"], Lbar[0], Lbar[1], [res["gbar"]]])
        fmap = mu.residual_map(prob, st, target)
        r = fmap(torch.tensor(u)).numpy()
        b = fmap(torch.zeros(3 * dim + 1, dtype=torch.float64))
        assert np.linalg.norm(r) < 1e-8 * max(1.0, float(torch.linalg.norm(b))), target
    ctx.close()


# --------------------------- mixed precision on the double (BF16 emulation)

def test_mixed_precision_emulation_error_levels(host_lib):
    """The double emulates the mixed modes (BF16 slices, FP32 accumulation):
    A R differs from the oracle at the level of the split (BF16x3 about 16
    bits, BF16 about 8), so the refinement tests below refine something."""
    from oracle import solvers as sv
    B, lib = host_lib
    o, v, J = 3, 4, 9
    eps, L = syn.system(o, v, J, 0.2, 55)
    prob = cc.Problem(eps, L, o)
    x, _, _ = sv.ground_state(prob, tol=1e-12)
    R = syn.random_vectors(o, v, 1, 9, normalise=True)
    ref = rp.jacobian_right(prob, x, R[0]).numpy()
    for prec, lo, hi in [("bf16x3", 1e-8, 1e-4), ("bf16", 1e-5, 3e-2)]:
        ctx = B.Context(o, v, J, eps, L, lib=lib, precision=prec)
        ctx.residual(x)
        err = np.abs(ctx.jacobian_right(R)[0] - ref).max() / np.abs(ref).max()
        ctx.close()
        assert lo < err < hi, (prec, err)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_mixed_solvers_refine_to_fp64(host_lib, prec):
    """Mixed iterations followed by FP64 refinement (the solvers' switch) give
    the FP64 ground state and EOM roots (Sec. 2.1)."""
    from oracle import solvers as sv
    B, lib = host_lib
    o, v, J = 3, 4, 9
    eps, L = syn.system(o, v, J, 0.2, 55)
    prob = cc.Problem(eps, L, o)
    x, E0, _ = sv.ground_state(prob, tol=1e-12)
    Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    ctx = B.Context(o, v, J, eps, L, lib=lib, precision=prec)
    e, t, _ = ctx.solve_ground(tol=1e-11, maxit=300, refine_tol=1e-4)
    assert abs(e - (E0 - Ehf)) < 1e-10
    for side in ("right", "left"):
        w, _, _ = ctx.solve_states(3, side=side, tol=1e-9, refine_tol=1e-4)
        wd, _ = sv.eom_dense(prob, x, 3, side=side)
        assert np.abs(w - wd).max() < 1e-9, side
    ctx.close()


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_mixed_scc_loop_refines_to_fp64(host_lib, prec):
    """In a mixed context the SCC loop takes r0 = eta.R / omega and O_ab in
    FP64, so zeta, the energies and the roots are the FP64 solution."""
    B, lib = host_lib
    g = _golden("scc_active_o3_v8.json")
    p = g["inputs"]
    eps, L = syn.system(p["o"], p["v"], p["J"], p["sd"], p["seed"])
    ctx = B.Context(p["o"], p["v"], p["J"], eps, L, lib=lib, precision=prec)
    r = ctx.solve_scc(tol=1e-10)
    ctx.close()
    assert abs(r["zeta"] - g["values"]["zeta"]) < 1e-7
    assert np.abs(r["omega"] - np.array(g["values"]["omega"])).max() < 1e-8
    assert abs(r["e_corr"] - g["values"]["e_corr"]) < 1e-9


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_mixed_multipliers_refine_to_fp64(host_lib, prec):
    """Mixed correction solves driven by FP64 residuals (Sec. 2.3.3 system)
    give the FP64 effective densities; where the mixed corrections stall (BF16
    here, with every contraction in BF16) the solver finishes in FP64."""
    B, lib = host_lib
    g = _golden("scc_active_o3_v8.json")
    p = g["inputs"]
    eps, L = syn.system(p["o"], p["v"], p["J"], p["sd"], p["seed"])
    ctx = B.Context(p["o"], p["v"], p["J"], eps, L, lib=lib)
    state = ctx.scc_state(tol=1e-10, ground_tol=1e-11, eom_tol=1e-9, left_tol=1e-9)
    ref = ctx.solve_multipliers(state, ("gradient", 0), tol=1e-10, maxit=800)
    ctx.close()
    ctx = B.Context(p["o"], p["v"], p["J"], eps, L, lib=lib, precision=prec)
    ctx.residual(state["t"], scc=(state["zeta"], state["Ra"], state["Rb"]))
    res = ctx.solve_multipliers(state, ("gradient", 0), tol=1e-10, maxit=800, refine_tol=1e-6)
    ctx.close()
    assert np.abs(res["D1"] - ref["D1"]).max() < 1e-8
    assert np.abs(res["Gamma"] - ref["Gamma"]).max() < 1e-8


def test_ground_solver_guess_and_preconditioner(host_lib):
    """The learned part only supplies a starting point and initial update
    denominators: with any positive preconditioner and a nearby guess the
    ground solver reaches the same state (the plain solver decides); a
    preconditioner with a non-positive entry is rejected."""
    from oracle import solvers as sv
    B, lib = host_lib
    o, v, J = 3, 4, 9
    eps, L = syn.system(o, v, J, 0.2, 55)
    prob = cc.Problem(eps, L, o)
    x, E0, _ = sv.ground_state(prob, tol=1e-12)
    Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    D = sv.denominators(prob)
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    rng = np.random.default_rng(3)
    ctx.set_preconditioner(np.ascontiguousarray(D * rng.uniform(0.7, 1.6, D.size)))
    t0 = x + 1e-3 * rng.normal(size=x.size)
    e, t, _ = ctx.solve_ground(t0=t0, tol=1e-11, maxit=300)
    assert abs(e - (E0 - Ehf)) < 1e-10 and np.abs(t - x).max() < 1e-9
    bad = D.copy()
    bad[7] = 0.0
    with pytest.raises(B.SccsdError) as ei:
        ctx.set_preconditioner(bad)
    assert ei.value.code == -1
    bad[7] = np.nan
    with pytest.raises(B.SccsdError):
        ctx.set_preconditioner(bad)
    ctx.set_preconditioner(None)
    e2, _, _ = ctx.solve_ground(tol=1e-11, maxit=300)
    assert abs(e2 - e) < 1e-10
    ctx.close()


def test_init_rejects_bad_integrals(host_lib):
    """sccsd_init: L^J must be finite and symmetric in pq, eps ascending within
    each block with a gap between them (SCCSD_EINVAL otherwise)."""
    B, lib = host_lib
    o, v, J = 2, 3, 4
    eps, L = syn.system(o, v, J, 0.3, 81)
    h = ctypes.c_void_p()

    def init(e, l):
        e = np.ascontiguousarray(e)
        l = np.ascontiguousarray(l)
        rc = lib.sccsd_init(ctypes.byref(h), o, v, J, e.ctypes.data, l.ctypes.data, 0, None)
        if rc == 0:
            lib.sccsd_destroy(h)
        return rc

    assert init(eps, L) == 0
    bad = L.copy()
    bad[1, 0, 3] += 1e-6                  # breaks L^J_pq = L^J_qp
    assert init(eps, bad) == -1
    bad = L.copy()
    bad[2, 4, 4] = np.inf
    assert init(eps, bad) == -1
    e2 = eps.copy()
    e2[o] = e2[o - 1]                     # no gap
    assert init(e2, L) == -1
    e3 = eps.copy()
    e3[o:] = e3[o:][::-1]                 # virtual block descending
    assert init(e3, L) == -1


@pytest.mark.parametrize("projection", ["natural", "state"])
def test_gradient_and_coupling_by_finite_differences(host_lib, projection):
    """Gradients and couplings along perturbations of eps and L by finite
    differences of re-converged states through the C ABI (tests/
    derivative_checks.py), for SCCSD(E) and SCCSD(K) (Sec. 2.4.1), on the
    system with an active constraint; for SCCSD(K) the oracle's stationarity
    equations also vanish at the C-ABI multipliers."""
    import derivative_checks as dc
    from oracle import multipliers as mu
    B, lib = host_lib
    g = _golden("scc_active_o3_v8.json")
    p = g["inputs"]
    o, v, J = p["o"], p["v"], p["J"]
    eps, L = syn.system(o, v, J, p["sd"], p["seed"])

    def oracle_equations(ctx, st):
        prob = cc.Problem(eps, L, o)
        ost = {"t": torch.tensor(st["t"]), "Ra": torch.tensor(st["Ra"]),
               "Rb": torch.tensor(st["Rb"]), "La": torch.tensor(st["La"]),
               "Lb": torch.tensor(st["Lb"]), "zeta": st["zeta"], "r0a": st["r0a"],
               "r0b": st["r0b"], "omega": (st["omega_a"], st["omega_b"]),
               "E0": dc.e_hf(eps, L, o) + st["e_corr"], "projection": projection}
        for target in [("gradient", 0), ("coupling", 0, 1)]:
            res = ctx.solve_multipliers(st, target, tol=1e-11, maxit=800, densities=False)
            d = [1.0 if (target[0] == "gradient" and k == target[1]) else 0.0 for k in range(2)]
            r0 = [st["r0a"], st["r0b"]]
            lam = [st["La"], st["Lb"]]
            Lbar = [res["K"][k] - (d[k] - res["lb0"][k] * r0[k]) * lam[k] for k in range(2)]
            u = np.concatenate([res["zbar"], Lbar[0], Lbar[1], [res["gbar"]]])
            fmap = mu.residual_map(prob, ost, target)
            r = fmap(torch.tensor(u)).numpy()
            b = fmap(torch.zeros(u.size, dtype=torch.float64))
            assert np.linalg.norm(r) < 1e-8 * max(1.0, float(torch.linalg.norm(b))), target

    dc.check(lambda e, l: B.Context(o, v, J, e, l, lib=lib), eps, L, o, v, J, projection,
             extra=oracle_equations if projection == "state" else None)
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    with pytest.raises(B.SccsdError):
        ctx.integral_derivative(np.eye(o + v), np.zeros((J, o + v, o + v)), np.eye(o + v), None)
    ctx.close()

# ------------------------------------- SCCSD(K): the state projection (Sec. 2.4.1)

@pytest.mark.parametrize("with_scc", [False, True], ids=["ccsd", "sccsd"])
def test_state_projection_overlap_through_the_c_abi(host_lib, with_scc):
    from oracle import scc as sc
    B, lib = host_lib
    o, v, J = 3, 4, 7
    eps, L = syn.system(o, v, J, 0.3, 64)
    t = syn.random_vectors(o, v, 1, 65, scale=0.1)[0]
    Ra, Rb = syn.random_vectors(o, v, 2, 66, normalise=True)
    ctx = B.Context(o, v, J, eps, L, lib=lib)
    ctx.residual(t, scc=(0.2, Ra, Rb) if with_scc else None)
    O = ctx.overlap_states(0.3, Ra, -0.2, Rb)
    ref = float(sc.overlap_states(torch.tensor(t), 0.3, torch.tensor(Ra), -0.2, torch.tensor(Rb),
                                  o, v))
    assert abs(O - ref) < 1e-13 * max(1.0, abs(ref))
    with pytest.raises(B.SccsdError):
        ctx.overlap_states(0.3, Ra, 0.6, 2.0 * Ra)      # linearly dependent states
    ctx.close()


def test_state_projection_scc_loop_through_the_c_abi(host_lib):
    """SCCSD(K): the SCC loop constraining O_ab of the state projection reaches
    the stored oracle solution."""
    from oracle import scc as sc
    B, lib = host_lib
    g = _golden("scc_state_projection_o3_v8.json")
    p = g["inputs"]
    eps, L = syn.system(p["o"], p["v"], p["J"], p["sd"], p["seed"])
    ctx = B.Context(p["o"], p["v"], p["J"], eps, L, lib=lib)
    with pytest.raises(B.SccsdError):
        ctx.set_projection(2)
    ctx.set_projection("state")
    r = ctx.solve_scc(tol=1e-10)
    t = ctx.state_amplitudes()
    assert abs(r["zeta"] - g["values"]["zeta"]) < 1e-7
    assert np.abs(r["omega"] - np.array(g["values"]["omega"])).max() < 1e-8
    assert abs(r["e_corr"] - g["values"]["e_corr"]) < 1e-9
    O = float(sc.overlap_states(torch.tensor(t), r["r0"][0], torch.tensor(r["Ra"]), r["r0"][1],
                                torch.tensor(r["Rb"]), p["o"], p["v"]))
    assert abs(O) < 1e-9
    # the natural-projection solution of the same system differs (small, as the paper notes)
    nat = _golden("scc_active_o3_v8.json")["values"]["zeta"]
    assert 1e-4 < abs(r["zeta"] - nat) < 1e-2
    ctx.close()


def test_random_shapes_match_the_oracle(host_lib):
    """Property check over random tiny shapes (o 1..3, v 1..5, J 1..6, any
    seeds, with or without the SCC terms): residual, A R, A^T L and the
    densities through the C ABI equal the oracle's, so the graph's index
    bookkeeping holds for degenerate and ragged layouts."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    B, lib = host_lib

    @hyp.settings(max_examples=25, deadline=None, derandomize=True)
    @hyp.given(o=st.integers(1, 3), v=st.integers(1, 5), J=st.integers(1, 6),
               seed=st.integers(0, 10_000), with_scc=st.booleans())
    def check(o, v, J, seed, with_scc):
        eps, L = syn.system(o, v, J, 0.3, seed)
        prob = cc.Problem(eps, L, o)
        t = syn.random_vectors(o, v, 1, seed + 1, scale=0.1)[0]
        R = syn.random_vectors(o, v, 2, seed + 2, normalise=True)
        Ra, Rb = syn.random_vectors(o, v, 2, seed + 3, normalise=True)
        scc = (0.3, Ra, Rb) if with_scc else None
        scct = (0.3, torch.tensor(Ra), torch.tensor(Rb)) if with_scc else None
        ctx = B.Context(o, v, J, eps, L, lib=lib)
        try:
            e, om = ctx.residual(t, scc=scc)
            E0, Om = rp.residual(prob, t, scc=scct)
            Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
            assert abs(e - (float(E0) - Ehf)) < 1e-12
            assert np.abs(om - Om.numpy()).max() < 1e-12
            s = ctx.jacobian_right(R)
            sl = ctx.jacobian_left(R)
            for k in range(2):
                ref = rp.jacobian_right(prob, t, R[k], scc=scct).numpy()
                assert np.abs(s[k] - ref).max() < 1e-12
                ref = rp.jacobian_left(prob, t, R[k], scc=scct).numpy()
                assert np.abs(sl[k] - ref).max() < 1e-12
            D1, G = ctx.densities(0.4, R[0], -0.7, R[1])
            D1r, Gr = rp.densities(prob, t, 0.4, R[0], -0.7, R[1], scc=scct)
            assert np.abs(D1 - D1r.numpy()).max() < 1e-12
            assert np.abs(G - Gr.numpy()).max() < 1e-12
        finally:
            ctx.close()

    check()


def test_binding_signatures_match_the_header():
    """Every ctypes signature the binding declares has as many arguments as the
    prototype in include/sccsd.h (a missing or miscounted argument would pass
    pointers as C ints or shift every later argument)."""
    from paper_2403_01007_gb300 import binding
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(sccsd_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", txt):
        args = m.group(2).strip()
        protos[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1

    class Fn:
        argtypes = None

    class FakeLib:
        def __getattr__(self, name):
            f = Fn()
            object.__setattr__(self, name, f)
            return f

    lib = binding._declare(FakeLib())
    declared = {k: v.argtypes for k, v in vars(lib).items() if isinstance(v, Fn)}
    checked = 0
    for name, argtypes in declared.items():
        if argtypes is None or name not in protos:
            continue
        assert len(argtypes) == protos[name], (name, len(argtypes), protos[name])
        checked += 1
    assert checked >= 40
