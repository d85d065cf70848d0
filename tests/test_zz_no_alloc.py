"""The allocation-free contraction entry point against the regular one.

sccsd_gemm_tn_noalloc exists for callers that cannot let the library call
cudaMalloc (memory fully owned by their own pool allocator, or no tolerance
for the device synchronisation an allocation implies). It must give the same
result as sccsd_gemm_tn on FP64, also on a second call that reuses the
shared scratch array left behind by the first, including the shapes where
the array's capacity (not the multiprocessor count) limits the K split, and
the same edge cases (M or N = 0 writes nothing, K = 0 gives zeros).
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _compare(B, M, N, K, alpha, rng, stream=None):
    A = torch.tensor(rng.normal(size=(M, K)), device="cuda:0")
    Bm = torch.tensor(rng.normal(size=(N, K)), device="cuda:0")
    C1 = torch.empty((M, N), dtype=torch.float64, device="cuda:0")
    C2 = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda:0")
    B.gemm_tn(A, Bm, C1, alpha=alpha, precision="fp64")
    torch.cuda.synchronize()
    B.gemm_tn_noalloc(A, Bm, C2, alpha=alpha, stream=stream)
    return C1, C2, A, Bm


def test_noalloc_matches_regular_entry_point_twice():
    from paper_2403_01007_gb300 import binding as B
    lib = B.load()
    cap = lib.sccsd_gemm_tn_noalloc_capacity()
    assert cap == 1 << 20
    rng = np.random.default_rng(11)
    # two calls in a row with different shapes and data; the last two have
    # M * N close to the capacity, so that cap / (M N) (1 and 3) is the binding
    # limit on the number of K chunks rather than the multiprocessor count
    for (M, N, K, alpha) in [(100, 30, 50000, 0.5), (257, 129, 9000, -1.25),
                             (1024, 1000, 4096, 0.75), (500, 600, 20000, 2.0)]:
        C1, C2, _, _ = _compare(B, M, N, K, alpha, rng)
        torch.cuda.synchronize()
        ref = C1.cpu().numpy()
        got = C2.cpu().numpy()
        # same FP64 arithmetic, only the split of K differs: rounding-level agreement
        tol = 1e-12 * np.sqrt(K) * np.abs(ref).max()
        assert np.abs(got - ref).max() <= tol, (M, N, K)


def test_noalloc_runs_in_stream_order():
    """The call only enqueues its work: two calls on one side stream, read
    after that stream is synchronised, both equal the regular entry point."""
    from paper_2403_01007_gb300 import binding as B
    rng = np.random.default_rng(12)
    s = torch.cuda.Stream()
    M, N, K = 300, 200, 30000
    A = torch.tensor(rng.normal(size=(M, K)), device="cuda:0")
    Bm = torch.tensor(rng.normal(size=(N, K)), device="cuda:0")
    ref = torch.empty((M, N), dtype=torch.float64, device="cuda:0")
    B.gemm_tn(A, Bm, ref, precision="fp64")
    torch.cuda.synchronize()
    Ca = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda:0")
    Cb = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda:0")
    torch.cuda.synchronize()
    B.gemm_tn_noalloc(A, Bm, Ca, alpha=1.0, stream=s)
    B.gemm_tn_noalloc(A, Bm, Cb, alpha=-2.0, stream=s)
    s.synchronize()
    r = ref.cpu().numpy()
    tol = 1e-12 * np.sqrt(K) * np.abs(r).max()
    assert np.abs(Ca.cpu().numpy() - r).max() <= tol
    assert np.abs(Cb.cpu().numpy() + 2.0 * r).max() <= 2 * tol


def test_noalloc_edge_cases_match_regular_entry_point():
    """M or N = 0 writes nothing and returns OK; K = 0 sets C to zero."""
    from paper_2403_01007_gb300 import binding as B
    lib = B.load()
    A = torch.ones((4, 8), dtype=torch.float64, device="cuda:0")
    C = torch.full((4, 4), 7.0, dtype=torch.float64, device="cuda:0")
    p = ctypes.c_void_p
    for (M, N) in [(0, 4), (4, 0)]:
        assert lib.sccsd_gemm_tn_noalloc(M, N, 8, 1.0, p(A.data_ptr()), p(A.data_ptr()),
                                         p(C.data_ptr()), None) == 0
        assert lib.sccsd_gemm_tn(0, M, N, 8, 1.0, p(A.data_ptr()), p(A.data_ptr()),
                                 p(C.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert torch.all(C == 7.0)
    assert lib.sccsd_gemm_tn_noalloc(4, 4, 0, 1.0, p(A.data_ptr()), p(A.data_ptr()),
                                     p(C.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert torch.all(C == 0.0)
    C.fill_(7.0)
    assert lib.sccsd_gemm_tn(0, 4, 4, 0, 1.0, p(A.data_ptr()), p(A.data_ptr()),
                             p(C.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert torch.all(C == 0.0)


def test_noalloc_rejects_oversized_output():
    from paper_2403_01007_gb300 import binding as B
    lib = B.load()
    cap = lib.sccsd_gemm_tn_noalloc_capacity()
    M = N = int(np.sqrt(cap)) + 1          # M * N just above the capacity
    A = torch.zeros((M, 16), dtype=torch.float64, device="cuda:0")
    C = torch.zeros((M, N), dtype=torch.float64, device="cuda:0")
    with pytest.raises(B.SccsdError) as ei:
        B.gemm_tn_noalloc(A, A, C)
    assert ei.value.code == -1
