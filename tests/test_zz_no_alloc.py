"""The allocation-free contraction entry point against the regular one.

sccsd_gemm_tn_noalloc exists for callers that cannot let the library call
cudaMalloc (memory fully owned by their own pool allocator, or no tolerance
for the device synchronisation an allocation implies). It must give the same
result as sccsd_gemm_tn on FP64, also on a second call that reuses the
shared scratch array left behind by the first.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_point_twice():
    from paper_2403_01007_gb300 import binding as B
    lib = B.load()
    cap = lib.sccsd_gemm_tn_noalloc_capacity()
    assert cap == 1 << 20
    rng = np.random.default_rng(11)
    # two calls in a row with different shapes and data
    for (M, N, K, alpha) in [(100, 30, 50000, 0.5), (257, 129, 9000, -1.25)]:
        A = torch.tensor(rng.normal(size=(M, K)), device="cuda:0")
        Bm = torch.tensor(rng.normal(size=(N, K)), device="cuda:0")
        C1 = torch.empty((M, N), dtype=torch.float64, device="cuda:0")
        C2 = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda:0")
        B.gemm_tn(A, Bm, C1, alpha=alpha, precision="fp64")
        B.gemm_tn_noalloc(A, Bm, C2, alpha=alpha)
        ref = C1.cpu().numpy()
        got = C2.cpu().numpy()
        # same FP64 arithmetic, only the split of K differs: rounding-level agreement
        tol = 1e-12 * np.sqrt(K) * np.abs(ref).max()
        assert np.abs(got - ref).max() <= tol


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
