"""Batched uneven instances: per-instance Jacobian transforms captured into
CUDA graphs and joined into one launch must give the transforms of the
ordinary per-instance calls and of the FP64 oracle for every instance, and
must read their input vectors at launch time (Sec. 2.1 EOM transforms; the
batching itself is not in the paper)."""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle import response as rp
from paper_2403_01007_gb300 import binding as B
from paper_2403_01007_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _instances(n, seed, prec):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        o = int(rng.integers(2, 6))
        v = int(rng.integers(6, 17))
        J = 3 * (o + v)
        nst = int(rng.integers(2, 6))
        eps, L = syn.system(o, v, J, 0.05, seed * 1000 + k)
        st = torch.cuda.Stream()
        ctx = B.Context(o, v, J, eps, L, precision=prec, stream=st.cuda_stream)
        t = syn.random_vectors(o, v, 1, seed * 1000 + 500 + k, scale=0.05)[0]
        ctx.residual(t)
        R = torch.tensor(syn.random_vectors(o, v, nst, seed * 1000 + 700 + k, normalise=True),
                         device="cuda")
        out.append(dict(ctx=ctx, stream=st, R=R, W=torch.empty_like(R), o=o, v=v, k=k,
                        eps=eps, L=L, t=t))
    return out


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
@pytest.mark.parametrize("side", ["right", "left"])
def test_joined_graph_equals_per_instance_calls(prec, side):
    torch.cuda.synchronize()
    inst = _instances(9, 11 if side == "right" else 12, prec)
    graphs = [x["ctx"].capture_transform(x["R"], x["W"], side=side) for x in inst]
    batch = B.GraphBatch(graphs)
    tol = 1e-12 if prec == "fp64" else 1e-6
    try:
        for rnd in range(2):
            if rnd == 1:      # new inputs in place: the graph reads them at launch
                for x in inst:
                    x["R"].copy_(torch.tensor(syn.random_vectors(
                        x["o"], x["v"], x["R"].shape[0], 900 + x["k"], normalise=True)))
            for x in inst:
                x["W"].fill_(float("nan"))
            torch.cuda.synchronize()
            s = torch.cuda.Stream()
            batch.launch(s.cuda_stream)
            torch.cuda.synchronize()
            for x in inst:
                ctx = x["ctx"]
                ref = ctx.jacobian_right(x["R"]) if side == "right" else ctx.jacobian_left(x["R"])
                torch.cuda.synchronize()
                assert torch.isfinite(x["W"]).all()
                assert _rel(x["W"], ref) < tol, (x["o"], x["v"], _rel(x["W"], ref))
                # and each instance's launched transforms against the FP64 oracle
                # (within the split's error in BF16)
                prob = cc.Problem(x["eps"], x["L"], x["o"])
                fn = rp.jacobian_right if side == "right" else rp.jacobian_left
                Wh = x["W"].cpu().numpy()
                Rh = x["R"].cpu().numpy()
                otol = 1e-11 if prec == "fp64" else 3e-2
                for kv in range(Rh.shape[0]):
                    o_ref = fn(prob, x["t"], Rh[kv]).numpy()
                    err = np.abs(Wh[kv] - o_ref).max() / max(1e-300, np.abs(o_ref).max())
                    assert err < otol, (x["o"], x["v"], kv, err)
    finally:
        batch.close()
        for x in inst:
            x["ctx"].close()


def test_capture_argument_errors():
    o, v, J = 3, 7, 12
    eps, L = syn.system(o, v, J, 0.05, 5)
    ctx = B.Context(o, v, J, eps, L)          # default stream: capture refused
    ctx.residual(np.zeros(ctx.dim))
    R = torch.zeros(2, ctx.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(B.SccsdError):
        ctx.capture_transform(R, torch.empty_like(R))
    st = torch.cuda.Stream()
    ctx2 = B.Context(o, v, J, eps, L, stream=st.cuda_stream)
    ctx2.residual(np.zeros(ctx2.dim))
    Rh = np.zeros((2, ctx2.dim))
    with pytest.raises(B.SccsdError):       # host vectors: capture refused
        ctx2.capture_transform(Rh, np.empty_like(Rh))
    ctx.close()
    ctx2.close()
