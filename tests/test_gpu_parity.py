"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle."""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle import response as rp
from paper_2403_01007_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2403_01007_gb300 import binding
    return binding


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


def maxrel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


# ----------------------------------------------------------- contraction primitive

def test_tc_gemm_exact_integers(B):
    """Small integers are exact in BF16 and their FP32 sums stay below 2^24,
    so the tensor-core GEMM must agree bit for bit (ragged M, N, K)."""
    rng = np.random.default_rng(5)
    M, N, K = 300, 517, 704
    A = rng.integers(-8, 9, size=(M, K)).astype(np.float64)
    Bm = rng.integers(-8, 9, size=(N, K)).astype(np.float64)
    C = torch.empty((M, N), dtype=torch.float64, device="cuda:0")
    B.gemm_tn(dev(A), dev(Bm), C, precision="bf16")
    assert np.array_equal(C.cpu().numpy(), A @ Bm.T)


@pytest.mark.parametrize("shape", [(100000, 21, 21), (5000, 6, 663), (40000, 2, 90),
                                   (25200, 300, 128), (300, 4200, 64), (126, 21, 84000),
                                   (1, 300, 5000)], ids=str)
def test_tc_gemm_exact_integer_shapes(B, shape):
    """Every form of the persistent tensor-core kernel on exact integer data:
    short K (the eight-warp form), N down to 2, an A operand that dominates
    (N-fastest work order), few output tiles with split-K, and M = 1 (which
    stays on the FP64 matrix-vector kernel)."""
    M, N, K = shape
    rng = np.random.default_rng(M + N + K)
    amp = 3 if K > 3000 else 8
    A = rng.integers(-amp, amp + 1, size=(M, K)).astype(np.float64)
    Bm = rng.integers(-amp, amp + 1, size=(N, K)).astype(np.float64)
    assert amp * amp * K < 2 ** 24      # every partial sum exact in FP32
    C = torch.empty((M, N), dtype=torch.float64, device="cuda:0")
    for rep in range(2):
        C.fill_(float("nan"))
        B.gemm_tn(dev(A), dev(Bm), C, precision="bf16")
        assert np.array_equal(C.cpu().numpy(), A @ Bm.T), (shape, rep)


def test_tc_gemm_split_accuracy(B):
    rng = np.random.default_rng(6)
    M, N, K = 1000, 777, 1300
    A = rng.normal(size=(M, K))
    Bm = rng.normal(size=(N, K))
    ref = A @ Bm.T
    C = torch.empty((M, N), dtype=torch.float64, device="cuda:0")
    B.gemm_tn(dev(A), dev(Bm), C, precision="bf16x3")
    err3 = np.abs(C.cpu().numpy() - ref).max() / np.abs(ref).max()
    B.gemm_tn(dev(A), dev(Bm), C, precision="bf16")
    err1 = np.abs(C.cpu().numpy() - ref).max() / np.abs(ref).max()
    B.gemm_tn(dev(A), dev(Bm), C, precision="fp64")
    err0 = np.abs(C.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err0 < 1e-14
    assert err1 < 2e-2
    # three slices leave FP32 accumulation (24-bit) as the limit: |err| <~ sqrt(K) u32 |C|
    assert err3 < 1e-5


def test_fp64_gemm_shapes(B):
    """Every FP64 route: dot products, matrix-vector, skinny tiles, split K."""
    rng = np.random.default_rng(7)
    for (M, N, K) in [(100, 30, 50000), (200, 21, 132600), (1, 1, 9000), (21, 42, 840000),
                      (40000, 1, 663), (1, 5000, 700), (5000, 70, 3000), (20, 3000, 5000),
                      (3000, 20, 5000), (33, 33, 100000)]:
        A = rng.normal(size=(M, K))
        Bm = rng.normal(size=(N, K))
        C = torch.empty((M, N), dtype=torch.float64, device="cuda:0")
        B.gemm_tn(dev(A), dev(Bm), C, alpha=0.5, precision="fp64")
        ref = 0.5 * A @ Bm.T
        assert np.abs(C.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max() * np.sqrt(K)


# ----------------------------------------------------------------- FP64 parity

def run_all(B, o, v, J, sd, seed, precision="fp64", scc=False, on_device=False):
    eps, L = syn.system(o, v, J, sd, seed)
    prob = cc.Problem(eps, L, o)
    t = syn.random_vectors(o, v, 1, seed + 1, scale=0.02)[0]
    R, Lv, Ra, Rb = syn.random_vectors(o, v, 4, seed + 2, normalise=True)
    conv = dev if on_device else (lambda x: np.ascontiguousarray(x))
    ctx = B.Context(o, v, J, conv(eps), conv(L), precision=precision)
    sccarg = (0.31, conv(Ra), conv(Rb)) if scc else None
    scct = (0.31, torch.tensor(Ra), torch.tensor(Rb)) if scc else None
    out = {}
    om = torch.empty(prob.dim, dtype=torch.float64, device="cuda:0") if on_device else None
    e, om = ctx.residual(conv(t), omega=om, scc=sccarg)
    om = om.cpu().numpy() if on_device else om
    E0, Om = rp.residual(prob, t, scc=scct)
    Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    out["E"] = (e, float(E0) - Ehf)
    out["omega"] = (om, Om.numpy())
    sig, eta = ctx.jacobian_right(np.ascontiguousarray(R), with_eta=True)
    out["AR"] = (sig, rp.jacobian_right(prob, t, R, scc=scct).numpy())
    out["etaR"] = (eta[0], float(rp.eta(prob, t, scc=scct) @ torch.tensor(R)))
    out["ATL"] = (ctx.jacobian_left(np.ascontiguousarray(Lv)),
                  rp.jacobian_left(prob, t, Lv, scc=scct).numpy())
    D1, G = ctx.densities(0.6, np.ascontiguousarray(Lv), -0.3, np.ascontiguousarray(R))
    D1r, Gr = rp.densities(prob, t, 0.6, Lv, -0.3, R, scc=scct)
    out["D1"] = (D1, D1r.numpy())
    out["Gamma"] = (G, Gr.numpy())
    ctx.close()
    return out


@pytest.mark.parametrize("scc", [False, True], ids=["ccsd", "sccsd"])
@pytest.mark.parametrize("size", [(1, 1, 3), (2, 3, 6), (3, 5, 9)], ids=lambda s: "o%d_v%d" % s[:2])
def test_fp64_parity_tiny(B, size, scc):
    o, v, J = size
    out = run_all(B, o, v, J, 0.3, 1234 + o * 10 + v, scc=scc)
    for k, (a, b) in out.items():
        assert maxrel(a, b) < 1e-12, k


def test_fp64_parity_small_device_pointers(B):
    w = syn.SMALL
    out = run_all(B, w.o, w.v, w.J, w.sd, syn.seed_of(w.config), scc=True, on_device=True)
    for k, (a, b) in out.items():
        assert maxrel(a, b) < 1e-11, k


def test_fp64_parity_ragged(B):
    """Sizes that are not multiples of any tile (v = 37, o = 7)."""
    out = run_all(B, 7, 37, 41, 0.05, 777)
    for k, (a, b) in out.items():
        assert maxrel(a, b) < 1e-11, k


# --------------------------------------------------------------- error paths

def test_error_codes(B):
    import ctypes
    lib = B.load()
    h = ctypes.c_void_p()
    eps = np.linspace(-1, 1, 4)
    L = np.zeros((2, 4, 4))
    assert lib.sccsd_init(ctypes.byref(h), 0, 4, 2, eps.ctypes.data, L.ctypes.data, 0, None) == -1
    assert lib.sccsd_init(ctypes.byref(h), 2, 2, 2, eps.ctypes.data, L.ctypes.data, 7, None) == -1
    bad = np.array([-1.0, -2.0, 0.5, 1.0])   # occupied eps not ascending
    assert lib.sccsd_init(ctypes.byref(h), 2, 2, 2, bad.ctypes.data, L.ctypes.data, 0, None) == -1
    ctx = B.Context(2, 2, 2, eps, L)
    R = np.zeros(B.dim(2, 2))
    with pytest.raises(B.SccsdError) as ei:
        ctx.jacobian_right(R)
    assert ei.value.code == -4
    ctx.close()


@pytest.mark.parametrize("nvec", [1, 3, 8, 11])
def test_batched_transforms(B, nvec):
    """Batches of trial vectors (chunked by 8 inside the library) give the
    same A R, eta.R and A^T L as the oracle vector by vector."""
    o, v, J = 3, 6, 10
    eps, L = syn.system(o, v, J, 0.2, 4242)
    prob = cc.Problem(eps, L, o)
    t = syn.random_vectors(o, v, 1, 4243, scale=0.05)[0]
    R = syn.random_vectors(o, v, nvec, 4244 + nvec, normalise=True)
    ctx = B.Context(o, v, J, eps, L)
    ctx.residual(t)
    s, eta = ctx.jacobian_right(dev(R), with_eta=True)
    s = s.cpu().numpy()
    sl = ctx.jacobian_left(dev(R)).cpu().numpy()
    for k in range(nvec):
        assert maxrel(s[k], rp.jacobian_right(prob, t, R[k]).numpy()) < 1e-12
        assert abs(eta[k] - float(rp.eta(prob, t) @ torch.tensor(R[k]))) < 1e-12
        assert maxrel(sl[k], rp.jacobian_left(prob, t, R[k]).numpy()) < 1e-12
    ctx.close()


@pytest.mark.parametrize("precision,tol", [("bf16x3", 2e-4), ("bf16", 3e-2)])
def test_mixed_precision_medium(B, precision, tol):
    """o=10, v=90, J=300: the contractions run on tcgen05 tensor cores. Errors
    against the FP64 oracle stay at the level the operand split allows
    (BF16x3: about 16 significant bits per product, FP32 accumulation;
    BF16: 8 bits)."""
    w = syn.MEDIUM
    eps, L = syn.workload_system(w)
    prob = cc.Problem(eps, L, w.o)
    t = syn.random_vectors(w.o, w.v, 1, 91, scale=1e-3)[0]
    R = syn.random_vectors(w.o, w.v, 2, 92, normalise=True)
    ctx = B.Context(w.o, w.v, w.J, eps, L, precision=precision)
    e, om = ctx.residual(t)
    E0, Om = rp.residual(prob, t)
    Ehf = float(rp.residual(prob, np.zeros(prob.dim))[0])
    assert maxrel(om, Om.numpy()) < tol
    assert abs(e - (float(E0) - Ehf)) < tol * max(1.0, abs(float(E0) - Ehf))
    s = ctx.jacobian_right(dev(R)).cpu().numpy()
    sl = ctx.jacobian_left(dev(R)).cpu().numpy()
    for k in range(2):
        assert maxrel(s[k], rp.jacobian_right(prob, t, R[k]).numpy()) < tol
        assert maxrel(sl[k], rp.jacobian_left(prob, t, R[k]).numpy()) < tol
    ctx.close()


def test_full_size_bench_configuration(B):
    """o=21, v=200, J=663 with the benchmark's own inputs and batch of six
    trial vectors. The oracle needs minutes per transform at this size, so the
    checks are ones that hold at any size:
      * A R in BF16 and BF16x3 against the FP64 GPU path (pinned to the
        oracle element by element at the small and ragged sizes above);
      * <L, A R> = <A^T L, R> for the FP64 right and left transforms, which
        the exact Jacobian satisfies up to rounding."""
    w = syn.LARGE
    eps, L = syn.workload_system(w)
    t = syn.random_vectors(w.o, w.v, 1, syn.seed_of(w.config, 50), scale=1e-3)[0]
    R = syn.random_vectors(w.o, w.v, 6, syn.seed_of(w.config, 60), normalise=True)
    Lv = syn.random_vectors(w.o, w.v, 1, syn.seed_of(w.config, 70), normalise=True)
    Rd = dev(R)

    out = {}
    for prec in ("bf16", "bf16x3"):
        ctx = B.Context(w.o, w.v, w.J, dev(eps), dev(L), precision=prec)
        ctx.residual(t)
        out[prec] = ctx.jacobian_right(Rd).cpu().numpy()
        ctx.close()
        del ctx
        torch.cuda.empty_cache()

    ctx = B.Context(w.o, w.v, w.J, dev(eps), dev(L), precision="fp64")
    ctx.residual(t)
    s64 = ctx.jacobian_right(dev(R[:2])).cpu().numpy()
    l64 = ctx.jacobian_left(dev(Lv)).cpu().numpy()[0]
    ctx.close()

    for k in range(2):
        assert maxrel(out["bf16"][k], s64[k]) < 2e-2
        assert maxrel(out["bf16x3"][k], s64[k]) < 2e-4
        a = float(np.dot(Lv[0], s64[k]))
        b = float(np.dot(l64, R[k]))
        scale = np.linalg.norm(s64[k]) + np.linalg.norm(l64)
        assert abs(a - b) < 1e-11 * scale
    # every row of the batch is a finite, non-trivial transform
    assert np.all(np.isfinite(out["bf16"])) and np.all(np.linalg.norm(out["bf16"], axis=1) > 0)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_transform_edge_cases(B, precision):
    """Empty batches are no-ops; zero vectors give exact zeros in both modes
    (the BF16 split of zero is zero, and A R is linear in R, Sec. 2.1); in
    FP64 the transforms are linear to rounding. Ragged o=7, v=37."""
    o, v, J = 7, 37, 41
    eps, L = syn.system(o, v, J, 0.05, 778)
    ctx = B.Context(o, v, J, eps, L, precision=precision)
    ctx.residual(syn.random_vectors(o, v, 1, 779, scale=0.02)[0])
    lib = ctx.lib
    assert lib.sccsd_jacobian_right(ctx.h, 0, None, None, None) == 0
    assert lib.sccsd_jacobian_left(ctx.h, 0, None, None) == 0
    Z = torch.zeros(3, ctx.dim, dtype=torch.float64, device="cuda:0")
    s, eta = ctx.jacobian_right(Z, with_eta=True)
    assert not s.any() and not np.any(eta)
    assert not ctx.jacobian_left(Z).any()
    if precision == "fp64":
        R1, R2 = syn.random_vectors(o, v, 2, 780, normalise=True)
        a, b = 0.7, -1.9
        X = dev(np.stack([R1, R2, a * R1 + b * R2]))
        s = ctx.jacobian_right(X).cpu().numpy()
        sl = ctx.jacobian_left(X).cpu().numpy()
        for y in (s, sl):
            assert np.abs(y[2] - (a * y[0] + b * y[1])).max() < 1e-12 * np.abs(y).max()
    ctx.close()
