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
