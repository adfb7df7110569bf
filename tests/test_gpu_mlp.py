"""Cost-model kernels against the FP64 oracle (oracle/mlp.py): forward,
loss and analytic gradient, Adam step; and training reduces the loss."""

import numpy as np
import pytest
import torch

import synth
from gpu_util import built, dev  # noqa: F401
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def flat(P):
    return np.concatenate([P[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def unflat(v, d, H=64):
    out, k = {}, 0
    for name, shp in [("W1", (H, d)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (1, H)), ("b3", (1,))]:
        c = int(np.prod(shp))
        out[name] = np.asarray(v[k:k + c], dtype=np.float64).reshape(shp)
        k += c
    return out


def setup(d, B, seed=0):
    H = 64
    P = omlp.init_params(d, H, synth.uniform((omlp.n_params(d, H),), seed, synth.TID["mlp"]).numpy().astype(np.float64))
    for kk in ("b1", "b2", "b3"):
        P[kk] = synth.uniform(P[kk].shape, seed + 1, synth.TID["mlp"]).numpy().astype(np.float64) * 0.1
    # round parameters to FP32 so both sides start from the same values
    P = {k: v.astype(np.float32).astype(np.float64) for k, v in P.items()}
    X = synth.uniform((B, d), seed + 2, synth.TID["mlp"]).numpy()
    y = synth.uniform((B,), seed + 3, synth.TID["mlp"]).numpy()
    return P, X, y


@pytest.mark.parametrize("d,B", [(16, 1), (16, 37), (7, 100), (32, 1000), (16, 5000)])
def test_forward_and_gradient(built, d, B):
    kf = built
    P, X, y = setup(d, B)
    p = torch.tensor(flat(P), dtype=torch.float32, device=dev())
    Xd = torch.tensor(X, dtype=torch.float32, device=dev())
    yd = torch.tensor(y, dtype=torch.float32, device=dev())
    out = torch.empty(B, device=dev())
    kf.kf_mlp_forward(p, Xd, out)
    f, _ = omlp.forward(P, X.astype(np.float64))
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.double().cpu().numpy(), f, rtol=1e-5, atol=1e-5 * np.abs(f).max())
    g = torch.empty_like(p)
    loss = torch.empty(1, device=dev())
    ws = torch.zeros(kf.kf_mlp_workspace_size(d, B), dtype=torch.uint8, device=dev())
    kf.kf_mlp_loss_grad(p, Xd, yd, g, loss, ws)
    L, G = omlp.grad(P, X.astype(np.float64), y.astype(np.float64))
    torch.cuda.synchronize()
    assert abs(float(loss) - L) <= 1e-4 * max(1.0, abs(L))
    gg = g.double().cpu().numpy()
    ref = flat(G)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(gg, ref, rtol=1e-4, atol=1e-4 * scale)


def test_adam_step(built):
    kf = built
    d, B = 16, 64
    P, X, y = setup(d, B, seed=4)
    _, G = omlp.grad(P, X, y)
    Gf = {k: v.astype(np.float32).astype(np.float64) for k, v in G.items()}
    p = torch.tensor(flat(P), dtype=torch.float32, device=dev())
    g = torch.tensor(flat(Gf), dtype=torch.float32, device=dev())
    m = torch.zeros_like(p); v = torch.zeros_like(p)
    M = {k: np.zeros_like(x) for k, x in P.items()}; V = {k: np.zeros_like(x) for k, x in P.items()}
    Pr = {k: x.copy() for k, x in P.items()}
    for t in (1, 2, 3):
        kf.kf_mlp_adam(p, g, m, v, t, lr=0.01)
        omlp.adam_step(Pr, Gf, M, V, t, lr=0.01)
    torch.cuda.synchronize()
    np.testing.assert_allclose(p.double().cpu().numpy(), flat(Pr), rtol=1e-5, atol=1e-6)


def test_training_reduces_loss(built):
    """Fit y = sum of squares of the first inputs (a smooth target)."""
    kf = built
    d, B = 16, 2048
    P, X, _ = setup(d, B, seed=7)
    y = (X[:, :3] ** 2).sum(axis=1)
    p = torch.tensor(flat(P), dtype=torch.float32, device=dev())
    Xd = torch.tensor(X, dtype=torch.float32, device=dev())
    yd = torch.tensor(y, dtype=torch.float32, device=dev())
    g = torch.empty_like(p); m = torch.zeros_like(p); v = torch.zeros_like(p)
    loss = torch.empty(1, device=dev())
    ws = torch.zeros(kf.kf_mlp_workspace_size(d, B), dtype=torch.uint8, device=dev())
    kf.kf_mlp_loss_grad(p, Xd, yd, g, loss, ws)
    l0 = float(loss)
    for t in range(1, 301):
        kf.kf_mlp_loss_grad(p, Xd, yd, g, loss, ws)
        kf.kf_mlp_adam(p, g, m, v, t, lr=3e-3)
    kf.kf_mlp_loss_grad(p, Xd, yd, g, loss, ws)
    assert float(loss) < 0.2 * l0
