"""Launch-shape tuning of the tensor-core contractions: tuned shapes give the
same Jacobian transforms as the fixed rule (up to the FP32 order of split K
ranges), the tuning runs leave the caller's outputs alone, and an exported
table reproduces the tuned results bit for bit in a fresh context."""
import numpy as np
import pytest
import torch

from paper_2403_01007_gb300 import binding as B
from paper_2403_01007_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_tuned_launch_shapes_give_the_same_transforms(prec):
    w = syn.MEDIUM
    eps, L = syn.workload_system(w)
    t = syn.random_vectors(w.o, w.v, 1, 191, scale=1e-3)[0]
    R = torch.tensor(syn.random_vectors(w.o, w.v, 3, 192, normalise=True), device="cuda")

    def run(tune):
        ctx = B.Context(w.o, w.v, w.J, eps, L, precision=prec)
        if tune:
            ctx.set_autotune(True)
        e, om = ctx.residual(t)
        s = ctx.jacobian_right(R).clone()
        l = ctx.jacobian_left(R).clone()
        return ctx, e, om, s, l

    B.autotune_clear()
    try:
        c0, e0, om0, s0, l0 = run(False)
        c0.close()
        assert B.autotune_entries() == 0          # tuning off records nothing

        c1, e1, om1, s1, l1 = run(True)
        n = B.autotune_entries()
        assert n > 0
        s1b = c1.jacobian_right(R)
        assert B.autotune_entries() == n          # known shapes are not tuned again
        assert torch.equal(s1b, s1)
        # tuned and default shapes differ only where the split of K differs:
        # one FP32 tensor-core accumulation over all K = v^2 = 8100 products
        # against shorter FP32 ranges summed in FP64. Each order is within
        # about K * 2^-24 = 5e-4 of the exact sum of the same BF16 products.
        tol = 1e-3
        assert _rel(s1, s0) < tol and _rel(l1, l0) < tol
        assert np.abs(om1 - om0).max() < tol * np.abs(om0).max()
        assert abs(e1 - e0) < tol * abs(e0)
        text = B.autotune_export()
        c1.set_autotune(False)                    # frees the tuning scratch
        assert torch.equal(c1.jacobian_right(R), s1)
        c1.close()
        assert len(text.strip().splitlines()) == n

        B.autotune_clear()
        B.autotune_import(text)
        c2, e2, om2, s2, l2 = run(False)
        c2.close()
        assert B.autotune_entries() == n
        assert torch.equal(s2, s1) and torch.equal(l2, l1)
        assert np.array_equal(om2, om1) and e2 == e1
    finally:
        B.autotune_clear()


def test_captured_graphs_use_the_tuned_shapes():
    """Uneven instances tuned by one uncaptured call each, then captured and
    joined into one launch: the graph reads the table (no tuning, no buffer
    growth while capturing) and equals the per-instance calls bit for bit."""
    B.autotune_clear()
    items = []
    try:
        for k, (o, v) in enumerate([(3, 20), (4, 27), (5, 33)]):
            J = 3 * (o + v)
            eps, L = syn.system(o, v, J, 0.05, 4100 + k)
            st = torch.cuda.Stream()
            ctx = B.Context(o, v, J, eps, L, precision="bf16", stream=st.cuda_stream)
            ctx.set_autotune(True)
            ctx.residual(syn.random_vectors(o, v, 1, 4200 + k, scale=0.02)[0])
            R = torch.tensor(syn.random_vectors(o, v, 3, 4300 + k, normalise=True), device="cuda")
            W = torch.empty_like(R)
            ref = ctx.jacobian_right(R).clone()          # tunes this instance's shapes
            ctx.set_autotune(False)
            items.append((ctx, R, W, ref))
        n = B.autotune_entries()
        assert n > 0
        batch = B.GraphBatch([ctx.capture_transform(R, W) for ctx, R, W, _ in items])
        try:
            s = torch.cuda.Stream()
            batch.launch(s.cuda_stream)
            torch.cuda.synchronize()
        finally:
            batch.close()
        assert B.autotune_entries() == n
        for ctx, R, W, ref in items:
            assert torch.equal(W, ref)
    finally:
        for ctx, *_ in items:
            ctx.close()
        B.autotune_clear()
