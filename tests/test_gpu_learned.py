"""Learned guess/preconditioner: GPU kernels against the FP64 reference, and
what the trained network gains over the plain method."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2403_01007_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def bf16(x):
    return torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float32).numpy()


def test_mlp_gradient_matches_reference():
    """The BF16 forward/backward kernels give the gradient of the FP64
    reference evaluated at the BF16-rounded weights and inputs, to the accuracy
    of BF16 activations (a few 1e-3 relative)."""
    from paper_2403_01007_gb300 import binding as B
    net = B.Mlp(n_in=10, hidden=64, layers=2, n_out=2, seed=3)
    rng = np.random.default_rng(4)
    N = 2048
    X = rng.normal(size=(N, 10)).astype(np.float32)
    T = rng.normal(size=(N, 2)).astype(np.float32)
    p = net.get_params()
    sizes = [(10, 64), (64, 64), (64, 2)]
    assert p.size == sum(a * b + b for a, b in sizes)
    # the kernels hold weights in BF16 (biases in FP32)
    pw = p.copy()
    off = 0
    for (din, dout) in sizes:
        pw[off:off + din * dout] = bf16(p[off:off + din * dout])
        off += din * dout + dout
    g, loss = net.gradient(torch.tensor(X, device="cuda:0"), torch.tensor(T, device="cuda:0"))
    lref, gref = omlp.loss_and_grad(pw, sizes, bf16(X), T)
    assert abs(loss - lref) < 2e-2 * abs(lref)
    rel = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    assert rel < 2e-2, rel
    # forward output against the reference
    Y = torch.empty((N, 2), device="cuda:0")
    net.forward(torch.tensor(X, device="cuda:0"), Y)
    layers = omlp.unflatten(pw.astype(np.float64), sizes)
    a = bf16(X).astype(np.float64)
    for k, (W, b) in enumerate(layers):
        a = a @ W + b
        if k < len(layers) - 1:
            a = bf16(np.maximum(a, 0.0)).astype(np.float64)
    assert np.abs(Y.cpu().numpy() - a).max() < 2e-2 * np.abs(a).max()
    net.close()


def _bf16_params(p, sizes):
    pw = p.copy()
    off = 0
    for (din, dout) in sizes:
        pw[off:off + din * dout] = bf16(p[off:off + din * dout])
        off += din * dout + dout
    return pw


def _reference_forward(pw, sizes, X):
    """FP64 forward with the kernels' BF16 rounding of inputs and activations."""
    a = bf16(X).astype(np.float64)
    layers = omlp.unflatten(pw.astype(np.float64), sizes)
    for k, (W, b) in enumerate(layers):
        a = a @ W + b
        if k < len(layers) - 1:
            a = bf16(np.maximum(a, 0.0)).astype(np.float64)
    return a


@pytest.mark.parametrize("N", [37, 3001])
def test_tensor_core_layers_at_the_production_width(N):
    """The 10 -> 3 x 256 -> 2 network on the tcgen05 layer kernels: a batch
    inside one tile (N = 37, below one 64-row contraction block) and one of
    many tiles with a ragged tail (N = 3001); gradient and output against the
    FP64 reference at the BF16-rounded weights and inputs."""
    from paper_2403_01007_gb300 import binding as B
    net = B.Mlp(n_in=10, hidden=256, layers=3, n_out=2, seed=5)
    rng = np.random.default_rng(N)
    X = rng.normal(size=(N, 10)).astype(np.float32)
    T = rng.normal(size=(N, 2)).astype(np.float32)
    sizes = [(10, 256), (256, 256), (256, 256), (256, 2)]
    pw = _bf16_params(net.get_params(), sizes)
    g, loss = net.gradient(torch.tensor(X, device="cuda:0"), torch.tensor(T, device="cuda:0"))
    lref, gref = omlp.loss_and_grad(pw, sizes, bf16(X), T)
    assert abs(loss - lref) < 2e-2 * abs(lref)
    assert np.linalg.norm(g - gref) < 2e-2 * np.linalg.norm(gref)
    # each layer's weight and bias gradient on its own
    off = 0
    for (din, dout) in sizes:
        for n in (din * dout, dout):
            blk, ref = g[off:off + n], gref[off:off + n]
            assert np.linalg.norm(blk - ref) < 3e-2 * np.linalg.norm(ref) + 1e-7, (din, dout, n)
            off += n
    Y = torch.empty((N, 2), device="cuda:0")
    net.forward(torch.tensor(X, device="cuda:0"), Y)
    a = _reference_forward(pw, sizes, X)
    assert np.abs(Y.cpu().numpy() - a).max() < 2e-2 * np.abs(a).max()
    net.close()


def test_tensor_core_forward_at_the_full_row_count():
    """Forward over o^2 v^2 = 230 400 rows (every doubles amplitude of an o=8,
    v=60 system, 1800 row tiles on the persistent kernel), sampled rows
    against the FP64 reference; and training steps after it, so that buffers
    sized for inference grow for training."""
    from paper_2403_01007_gb300 import binding as B
    net = B.Mlp(n_in=10, hidden=256, layers=3, n_out=2, seed=6)
    N = 8 * 8 * 60 * 60
    rng = np.random.default_rng(12)
    X = rng.normal(size=(N, 10)).astype(np.float32)
    sizes = [(10, 256), (256, 256), (256, 256), (256, 2)]
    pw = _bf16_params(net.get_params(), sizes)
    Y = torch.empty((N, 2), device="cuda:0")
    net.forward(torch.tensor(X, device="cuda:0"), Y)
    rows = rng.choice(N, size=3000, replace=False)
    rows = np.concatenate([rows, [0, 127, 128, N - 1]])
    a = _reference_forward(pw, sizes, X[rows])
    assert np.abs(Y.cpu().numpy()[rows] - a).max() < 2e-2 * np.abs(a).max()
    Xd = torch.tensor(X[:8192], device="cuda:0")
    Td = torch.tensor(rng.normal(size=(8192, 2)).astype(np.float32), device="cuda:0")
    l0 = net.train_step(Xd, Td, 1e-3)
    for _ in range(20):
        l1 = net.train_step(Xd, Td, 1e-3)
    assert np.isfinite(l1) and l1 < l0
    net.close()


def test_training_decreases_loss_and_learned_solver_is_exact():
    """Train on solver-generated data of small systems, then solve fresh ones:
    the learned start converges to the plain solver's energy (1e-8 Eh), and the
    gain in iterations is reported."""
    from paper_2403_01007_gb300 import binding as B
    from paper_2403_01007_gb300 import learned as lrn
    train_sys = [lrn.system(4, 24, k) for k in range(6)]
    X, Y = lrn.generate(train_sys, samples_per_instance=8000)
    net = B.Mlp(seed=7)
    hist = lrn.train(net, X, Y, epochs=12, batch=2048, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    rows = lrn.evaluate(net, [lrn.system(5, 28, 100 + k) for k in range(3)])
    for r in rows:
        assert abs(r["de"]) < 1e-8
    gain = np.mean([r["plain_iters"] - r["learned_iters"] for r in rows])
    print("learned-guess rows:", rows, "mean iteration gain:", gain)
    net.close()
