"""The surrogate network on the tensor cores against its FP64 reference (oracle/mlp.py).

Both sides see the same BF16-rounded inputs and weights. The GPU also rounds the
hidden activations H1 and the back-propagated dZ2, dZ1 to BF16 before the tensor-core
products (8 significand bits: relative error <= 2^-9 each) and accumulates in FP32, so
the forward output is compared in relative L2 norm with a tolerance of 2e-2 (a few
2^-9 roundings compounded over three layers). The gradients also inherit ReLU masks
that flip where a pre-activation lies within that rounding of zero; each flip moves a
whole term of the bias sums, so every gradient block is held to 5e-2 in relative L2
norm and must point the same way (cosine >= 0.999). One Adam step is checked to FP32 rounding (1e-5
relative) against the reference update applied to the GPU's own gradients.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import mlp as ref  # noqa: E402
from paper_0908_0681_gb300 import engine, kt  # noqa: E402


def bf16(a):
    return torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).float().double().numpy()


def setup(n_in=80, B=256, seed=3):
    rng = np.random.default_rng(seed)
    p = ref.init(n_in, seed)
    p["b1"] = rng.normal(0, 0.1, 256)
    p["b2"] = rng.normal(0, 0.1, 256)
    p["b3"] = np.array([0.2])
    # the GPU keeps FP32 masters and multiplies their BF16 copies; the reference uses the same values
    q = {k: (bf16(v) if k in ("W1", "W2") else np.asarray(v, np.float32).astype(np.float64)) for k, v in p.items()}
    X = bf16(rng.normal(0, 1, (B, n_in)))
    t = rng.normal(0, 1, B)
    net = engine.Surrogate(n_in, max_batch=B, params=ref.pack(p))
    return net, q, X, t


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_forward_matches_reference():
    net, q, X, t = setup()
    y = net.predict(torch.as_tensor(X, device="cuda").to(torch.bfloat16)).double().cpu().numpy()
    y_ref, _ = ref.forward(q, X)
    assert rel(y, y_ref) < 2e-2
    assert kt.kt_mlp_error(net.h) == 0


def test_gradients_match_reference():
    net, q, X, t = setup()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    kt.kt_mlp_backward(net.h, torch.as_tensor(X, device="cuda").to(torch.bfloat16),
                       torch.as_tensor(t, dtype=torch.float32, device="cuda"), loss)
    g = ref.unpack(kt.kt_mlp_get_grads(net.h).astype(np.float64), 80)
    L_ref, g_ref = ref.loss_and_grads(q, X, t)
    assert abs(float(loss.item()) / L_ref - 1) < 2e-2
    for k in ref.PARAMS:
        a, b = g[k].ravel(), g_ref[k].ravel()
        assert rel(a, b) < 5e-2, (k, rel(a, b))
        assert a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30) > 0.999, k


def test_adam_step_matches_reference():
    net, q, X, t = setup()
    p0 = ref.unpack(net.params().astype(np.float64), 80)
    kt.kt_mlp_backward(net.h, torch.as_tensor(X, device="cuda").to(torch.bfloat16),
                       torch.as_tensor(t, dtype=torch.float32, device="cuda"))
    g = ref.unpack(kt.kt_mlp_get_grads(net.h).astype(np.float64), 80)
    kt.kt_mlp_adam(net.h, 1e-3)
    p1 = ref.unpack(net.params().astype(np.float64), 80)
    zeros = {k: np.zeros_like(v) for k, v in p0.items()}
    e, _, _ = ref.adam_step(p0, g, zeros, zeros, 1, 1e-3)
    for k in ref.PARAMS:
        assert np.abs(p1[k] - e[k]).max() <= 1e-5 * max(1.0, np.abs(e[k]).max()), k


def test_training_reduces_the_loss():
    """A smooth target of the inputs is learned: the epoch loss falls by an order of magnitude."""
    rng = np.random.default_rng(5)
    n_in, N = 80, 16384
    Xh = rng.normal(0, 1, (N, n_in))
    tgt = np.tanh(Xh[:, :8].sum(axis=1) / 3) - 0.5 * Xh[:, 8] ** 2 / 4
    X = torch.as_tensor(Xh, device="cuda").to(torch.bfloat16)
    t = torch.as_tensor(tgt, dtype=torch.float32, device="cuda")
    net = engine.Surrogate(n_in, max_batch=1024, seed=2)
    hist = net.train(X, t, epochs=25, batch=1024, lr=2e-3)
    assert hist[-1] < 0.1 * hist[0], hist
