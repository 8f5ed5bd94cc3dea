"""GPU parity of the learned-proposal network (BF16 tensor-core kernels with
FP32 accumulation) against the FP64 CPU oracle.

Forward: against the oracle evaluated on the same BF16-rounded inputs,
weights and hidden activations (checks the tensor-core fragment layouts to
FP32 accumulation order, 1e-4), and against the unrounded FP64 oracle
(BF16 rounding only, 2e-2 relative L2).  Gradients: cosine distance < 2e-2
and relative L2 < 5e-2 per parameter tensor.  Adam: one step against the
oracle's update from the GPU's own gradients."""
import numpy as np
import pytest

import oracle.mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5826_gb300 import build, kn
    build.build()
    return torch, kn


def bf16(x):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _setup(kn, torch, B, seed):
    rng = np.random.default_rng(seed)
    p = M.init_params(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.1, p[k].shape)
    mu = rng.normal(0, 1, 64).astype(np.float32)
    sigma = rng.uniform(0.5, 2, 64).astype(np.float32)
    feat = (rng.normal(0, 1.5, (B, 64)) + mu).astype(np.float32)
    y = rng.normal(0, 1, B).astype(np.float32)
    net = kn.MLP()
    flat = kn.mlp_pack(p)
    net.set_params(flat, mu, sigma)
    pf = kn.mlp_unpack(flat)  # the FP32 values the GPU holds
    X = (feat.astype(np.float64) - mu) * (1.0 / sigma.astype(np.float32)).astype(np.float64)
    return net, pf, feat, y, X


@pytest.mark.parametrize("B", [1, 37, 512, 4099])
def test_forward(env, B):
    torch, kn = env
    net, p, feat, y, X = _setup(kn, torch, B, 3)
    tf = torch.from_numpy(feat).cuda()
    out = torch.empty(B, dtype=torch.float32, device="cuda")
    net.forward(tf, out)
    got = out.cpu().numpy().astype(np.float64)
    # oracle on BF16-rounded operands (what the tensor cores see)
    pr = dict(p)
    pr["W1"], pr["W2"] = bf16(p["W1"]), bf16(p["W2"])
    h1 = bf16(np.maximum(bf16(X) @ pr["W1"] + p["b1"], 0))
    h2 = bf16(np.maximum(h1 @ pr["W2"] + p["b2"], 0))
    ref = (h2 @ p["W3"])[:, 0] + p["b3"][0]
    # equal up to FP32 summation order; an order difference can flip the BF16
    # rounding of a hidden activation (one BF16 ulp, 2^-8), so bound that too
    scale = max(1.0, np.max(np.abs(ref)))
    err = np.abs(got - ref)
    assert np.mean(err <= 1e-5 * scale) >= 0.98
    assert np.max(err) <= 2e-3 * scale
    # plain FP64 oracle
    ref64, _ = M.forward(p, X)
    assert np.linalg.norm(got - ref64) <= 2e-2 * np.linalg.norm(ref64)
    net.close()


def test_gradients_and_adam(env):
    torch, kn = env
    B = 777
    net, p, feat, y, X = _setup(kn, torch, B, 5)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.backward(torch.from_numpy(feat).cuda(), torch.from_numpy(y).cuda(), loss)
    torch.cuda.synchronize()
    p0, g = net.get_params()
    gd = kn.mlp_unpack(g)
    ref = M.backward(p, X, y.astype(np.float64))
    assert loss.item() == pytest.approx(M.loss(p, X, y.astype(np.float64)), rel=2e-2)
    for k in ref:
        a, b = gd[k].reshape(-1), ref[k].reshape(-1)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300)
        assert 1 - cos < 2e-2, (k, cos)
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b), k
    # one Adam step from the GPU's own gradients against the oracle's update rule
    net.adam(lr=1e-2)
    p1, _ = net.get_params()
    pd = kn.mlp_unpack(p0.astype(np.float64))
    m = {k: np.zeros_like(v) for k, v in pd.items()}
    v = {k: np.zeros_like(v) for k, v in pd.items()}
    M.adam_step(pd, gd, m, v, step=1, lr=1e-2)
    assert np.allclose(kn.mlp_pack(pd), p1, rtol=1e-5, atol=1e-6)
    net.close()


def test_training_reduces_loss(env):
    """A smooth synthetic target is learned by the GPU training loop."""
    torch, kn = env
    rng = np.random.default_rng(9)
    B = 2048
    feat = rng.normal(0, 1, (8 * B, 64)).astype(np.float32)
    w = rng.normal(0, 0.3, 64)
    y = np.tanh(feat.astype(np.float64) @ w).astype(np.float32)
    net = kn.MLP()
    p = M.init_params(0)
    net.set_params(kn.mlp_pack(p), np.zeros(64, np.float32), np.ones(64, np.float32))
    tf = torch.from_numpy(feat).cuda()
    ty = torch.from_numpy(y).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    losses = []
    for epoch in range(12):
        for i in range(8):
            net.backward(tf[i * B:(i + 1) * B], ty[i * B:(i + 1) * B], loss)
            net.adam(lr=2e-3)
        losses.append(loss.item())
    assert losses[-1] < 0.25 * losses[0], losses
    net.close()
