"""The surrogate network on the tensor cores against its FP64 reference (oracle/mlp.py),
element by element.

Both sides see the same BF16 inputs and weights. The kernels round the hidden
activations H1 and the back-propagated dZ2, dZ1 to BF16 (the operands of the tensor-core
products) and accumulate in FP32. Two checks, both on every element:

1. Stage by stage. kt_mlp_get_tape returns the values each stage of the GPU consumed and
   produced. Every product and sum is recomputed in FP64 from the GPU's own inputs of that
   stage and must agree within the FP32 accumulation bound
   |fl(sum_k a_k b_k) - sum_k a_k b_k| <= 2 (K + 1) u sum_k |a_k b_k|, u = 2^-24
   (the factor 2 allows truncating accumulation in the tensor core; K is the length of
   the sum, the split-K slabs included). Every rounding step (bias + ReLU into BF16, the
   masked products into BF16) is recomputed with FP32 operations and round-to-nearest-even
   and must agree bit for bit, masks included (the mask is taken in FP32 on both sides).
2. End to end against loss_and_grads_bf16, the oracle's own chain with the same rounding
   points and no GPU input. Its values differ from the GPU's by FP32 accumulation, by one
   BF16 ulp (2^-7 relative) wherever the two sides' unrounded values straddle a rounding
   boundary, and by whole terms wherever a pre-activation lies within the accumulated
   difference of zero (a ReLU mask that may flip). The test propagates these bounds
   through the layers and holds every forward output and every gradient to its own bound.
One Adam step is checked to FP32 rounding (1e-5 relative) against the reference update
applied to the GPU's own gradients.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import mlp as ref  # noqa: E402
from paper_0908_0681_gb300 import engine, kt  # noqa: E402

U32 = 2.0 ** -24
ULP16 = 2.0 ** -7      # one BF16 ulp, relative (8 significand bits)
N_IN, BATCH = 80, 256


def f32(a):
    return np.asarray(a, dtype=np.float32)


def setup(n_in=N_IN, B=BATCH, seed=3):
    rng = np.random.default_rng(seed)
    p = ref.init(n_in, seed)
    p["b1"] = rng.normal(0, 0.1, 256)
    p["b2"] = rng.normal(0, 0.1, 256)
    p["b3"] = np.array([0.2])
    # the GPU keeps FP32 masters and multiplies their BF16 copies; the reference uses the same values
    q = {k: (ref.bf16(v) if k in ("W1", "W2") else f32(v).astype(np.float64)) for k, v in p.items()}
    X = ref.bf16(rng.normal(0, 1, (B, n_in)))
    t = f32(rng.normal(0, 1, B)).astype(np.float64)
    net = engine.Surrogate(n_in, max_batch=B, params=ref.pack(p))
    return net, q, X, t


def run_backward(net, X, t):
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    kt.kt_mlp_backward(net.h, torch.as_tensor(X, device="cuda").to(torch.bfloat16),
                       torch.as_tensor(t, dtype=torch.float32, device="cuda"), loss)
    g = ref.unpack(kt.kt_mlp_get_grads(net.h).astype(np.float64), X.shape[1])
    tape = kt.kt_mlp_get_tape(net.h, X.shape[0])
    assert kt.kt_mlp_error(net.h) == 0
    return float(loss.item()), g, tape


def acc_bound(absprod, K):
    """FP32 accumulation bound for sums of K products whose absolute values sum to absprod."""
    return 2.0 * (K + 1) * U32 * np.asarray(absprod, dtype=np.float64) + 1e-35


def check(name, got, want, bound):
    got, want, bound = (np.asarray(a, np.float64) for a in (got, want, bound))
    err = np.abs(got - want)
    bad = np.argwhere(~(err <= bound))
    assert bad.size == 0, (name, len(bad), bad[:5].tolist(), float((err / np.maximum(bound, 1e-300)).max()))
    return float((err / np.maximum(bound, 1e-300)).max())


def test_forward_stages_match_reference():
    """z1 = X W1^T, H1 = bf16(relu(z1 + b1)), z2 = H1 W2^T, y = w3 . relu(z2 + b2) + b3,
    each stage from the GPU's own inputs (the sampler's forward is the same code path)."""
    net, q, X, t = setup()
    _, _, tp = run_backward(net, X, t)
    W1, W2, b1, b2, w3, b3 = q["W1"], q["W2"], q["b1"], q["b2"], q["w3"], q["b3"]
    check("z1", tp["z1"], X @ W1.T, acc_bound(np.abs(X) @ np.abs(W1).T, N_IN))
    h1 = ref.from_bf16_bits(tp["h1"])
    want_h1 = ref.bf16(np.maximum(f32(tp["z1"]) + f32(b1), np.float32(0)))
    assert np.array_equal(h1, want_h1), int((h1 != want_h1).sum())
    check("z2", tp["z2"], h1 @ W2.T, acc_bound(np.abs(h1) @ np.abs(W2).T, 256))
    h2 = np.maximum(f32(tp["z2"]) + f32(b2), np.float32(0)).astype(np.float64)
    y = net.predict(torch.as_tensor(X, device="cuda").to(torch.bfloat16)).double().cpu().numpy()
    check("y", y, h2 @ w3 + b3[0], acc_bound(np.abs(h2) @ np.abs(w3) + abs(b3[0]), 257))
    # the backward pass's dy is 2 (y - t) / B of the same forward output
    want_dy = (np.float32(2) * (f32(y) - f32(t))) / np.float32(X.shape[0])
    check("dy", tp["dy"], want_dy, 2 * U32 * np.abs(want_dy) + 1e-38)


def test_backward_stages_match_reference():
    """dZ2 = bf16(dy w3 masked), the output-layer sums, dW2 = dZ2^T H1, dH1 = dZ2 W2,
    dZ1 = bf16(dH1 masked), gb1 and dW1 = dZ1^T X, each from the GPU's own inputs."""
    net, q, X, t = setup()
    _, g, tp = run_backward(net, X, t)
    B = X.shape[0]
    W2, b1, b2, w3 = q["W2"], q["b1"], q["b2"], q["w3"]
    h1 = ref.from_bf16_bits(tp["h1"])
    dy = tp["dy"].astype(np.float64)
    mask2 = (f32(tp["z2"]) + f32(b2)) > 0
    mask1 = (f32(tp["z1"]) + f32(b1)) > 0
    e2 = np.where(mask2, f32(tp["dy"])[:, None] * f32(w3)[None, :], np.float32(0))
    dz2 = ref.from_bf16_bits(tp["dz2"])
    assert np.array_equal(dz2, ref.bf16(e2)), int((dz2 != ref.bf16(e2)).sum())
    h2 = np.maximum(f32(tp["z2"]) + f32(b2), np.float32(0)).astype(np.float64)
    e2 = e2.astype(np.float64)
    check("gw3", g["w3"], h2.T @ dy, acc_bound(np.abs(h2).T @ np.abs(dy), B + 8))
    check("gb2", g["b2"], e2.sum(axis=0), acc_bound(np.abs(e2).sum(axis=0), B + 8))
    check("gb3", g["b3"], [dy.sum()], acc_bound([np.abs(dy).sum()], B + 8))
    check("dW2", g["W2"], dz2.T @ h1, acc_bound(np.abs(dz2).T @ np.abs(h1), B + 16))
    check("dh1", tp["dh1"], dz2 @ W2, acc_bound(np.abs(dz2) @ np.abs(W2), 256))
    e1 = np.where(mask1, f32(tp["dh1"]), np.float32(0))
    dz1 = ref.from_bf16_bits(tp["dz1"]).T
    assert np.array_equal(dz1, ref.bf16(e1)), int((dz1 != ref.bf16(e1)).sum())
    e1 = e1.astype(np.float64)
    check("gb1", g["b1"], e1.sum(axis=0), acc_bound(np.abs(e1).sum(axis=0), B + 8))
    check("dW1", g["W1"], dz1.T @ X, acc_bound(np.abs(dz1).T @ np.abs(X), B + 16))
    # the masks really cut: both layers have active and inactive units
    assert 0.1 < mask1.mean() < 0.9 and 0.1 < mask2.mean() < 0.9


def test_end_to_end_matches_bf16_oracle():
    """Every forward output and gradient element against the oracle's own BF16 chain (no
    GPU input), within bounds propagated through the layers from FP32 accumulation, one
    BF16 ulp at every rounding point and the ReLU masks that may flip."""
    net, q, X, t = setup()
    L_gpu, g, tp = run_backward(net, X, t)
    L, go, o = ref.loss_and_grads_bf16(q, X, t)
    B = X.shape[0]
    W1, W2, w3 = q["W1"], q["W2"], q["w3"]
    aX, aW1, aW2, aw3 = np.abs(X), np.abs(W1), np.abs(W2), np.abs(w3)
    # forward: absolute bounds on |gpu - oracle| per element
    e_a1 = acc_bound(aX @ aW1.T, N_IN) + U32 * (np.abs(o["a1"]) + np.abs(q["b1"]))
    e_h1 = e_a1 + ULP16 * (np.abs(o["h1"]) + e_a1)
    e_a2 = e_h1 @ aW2.T + acc_bound((np.abs(o["h1"]) + e_h1) @ aW2.T, 256) + U32 * (np.abs(o["a2"]) + np.abs(q["b2"]))
    e_h2 = e_a2
    e_y = e_h2 @ aw3 + acc_bound((np.abs(o["h2"]) + e_h2) @ aw3 + abs(q["b3"][0]), 257)
    y = net.predict(torch.as_tensor(X, device="cuda").to(torch.bfloat16)).double().cpu().numpy()
    check("y", y, o["y"], e_y)
    e_dy = 2.0 / B * e_y + 4 * U32 * np.abs(o["dy"])
    check("dy", tp["dy"], o["dy"], e_dy)
    # backward: an entry whose pre-activation is within its bound of zero may carry either mask
    amb2 = np.abs(o["a2"]) <= e_a2
    amb1 = np.abs(o["a1"]) <= e_a1
    de2 = np.outer(e_dy, aw3) + U32 * np.abs(np.outer(o["dy"], w3))
    e_e2 = np.where(amb2, np.abs(np.outer(o["dy"], w3)) + de2, de2)
    e_dz2 = e_e2 + ULP16 * (np.abs(o["dz2"]) + e_e2)
    A_e2 = np.abs(np.outer(o["dy"], w3)) + de2           # |e2| at most
    check("gb2", g["b2"], go["b2"], e_e2.sum(axis=0) + acc_bound(A_e2.sum(axis=0), B + 8))
    check("gb3", g["b3"], go["b3"], e_dy.sum() + acc_bound(np.abs(o["dy"]).sum() + e_dy.sum(), B + 8))
    check("gw3", g["w3"], go["w3"], e_dy @ (np.abs(o["h2"]) + e_h2) + np.abs(o["dy"]) @ e_h2
          + acc_bound((np.abs(o["dy"]) + e_dy) @ (np.abs(o["h2"]) + e_h2), B + 8))
    A_dz2, A_h1 = np.abs(o["dz2"]) + e_dz2, np.abs(o["h1"]) + e_h1
    check("dW2", g["W2"], go["W2"], e_dz2.T @ A_h1 + np.abs(o["dz2"]).T @ e_h1 + acc_bound(A_dz2.T @ A_h1, B + 16))
    e_dh1 = e_dz2 @ aW2 + acc_bound(A_dz2 @ aW2, 256)
    check("dh1", tp["dh1"], o["dh1"], e_dh1)
    A_dh1 = np.abs(o["dh1"]) + e_dh1
    e_e1 = np.where(amb1, A_dh1, e_dh1)
    e_dz1 = e_e1 + ULP16 * (np.abs(o["dz1"]) + e_e1)
    check("gb1", g["b1"], go["b1"], e_e1.sum(axis=0) + acc_bound(A_dh1.sum(axis=0), B + 8))
    check("dW1", g["W1"], go["W1"], e_dz1.T @ aX + acc_bound((np.abs(o["dz1"]) + e_dz1).T @ aX, B + 16))
    assert abs(L_gpu / L - 1) < 1e-2
    # the bounds stay informative: most gradient elements are held well inside 10% of their size
    for k in ("W1", "W2"):
        tight = np.abs(g[k] - go[k]) <= 0.1 * np.abs(go[k])
        assert tight.mean() > 0.8, (k, tight.mean())


def test_adam_step_matches_reference():
    net, q, X, t = setup()
    p0 = ref.unpack(net.params().astype(np.float64), N_IN)
    kt.kt_mlp_backward(net.h, torch.as_tensor(X, device="cuda").to(torch.bfloat16),
                       torch.as_tensor(t, dtype=torch.float32, device="cuda"))
    g = ref.unpack(kt.kt_mlp_get_grads(net.h).astype(np.float64), N_IN)
    kt.kt_mlp_adam(net.h, 1e-3)
    p1 = ref.unpack(net.params().astype(np.float64), N_IN)
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
