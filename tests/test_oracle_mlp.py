"""Pins of the surrogate's FP64 reference (oracle/mlp.py) against facts outside it:
central finite differences of the loss (the analytic backward pass must match them),
properties of Adam (the first bias-corrected step has length lr in every coordinate;
the update is invariant under positive rescaling of the gradient; a constant gradient
moves every step by lr), a hand-evaluated network, and a hand-built feature vector.
"""
import math

import numpy as np

from oracle import mlp


def _small(seed, n_in=16, hidden=8, B=6):
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0, 0.7, (hidden, n_in)), "b1": rng.normal(0, 0.3, hidden),
         "W2": rng.normal(0, 0.5, (hidden, hidden)), "b2": rng.normal(0, 0.3, hidden),
         "w3": rng.normal(0, 0.6, hidden), "b3": rng.normal(0, 0.3, 1)}
    X = rng.normal(0, 1, (B, n_in))
    t = rng.normal(0, 1, B)
    return p, X, t


def test_backward_matches_finite_differences():
    checked = 0
    for seed in range(6):
        p, X, t = _small(seed)
        _, (a1, _, a2, _) = mlp.forward(p, X)
        h = 1e-6
        if min(np.abs(a1).min(), np.abs(a2).min()) < 1e-4:
            continue  # a pre-activation too close to the ReLU kink for a finite difference
        L, g = mlp.loss_and_grads(p, X, t)
        for k in mlp.PARAMS:
            num = np.zeros_like(p[k])
            it = np.nditer(p[k], flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                q = {kk: vv.copy() for kk, vv in p.items()}
                q[k][idx] += h
                Lp, _ = mlp.loss_and_grads(q, X, t)
                q[k][idx] -= 2 * h
                Lm, _ = mlp.loss_and_grads(q, X, t)
                num[idx] = (Lp - Lm) / (2 * h)
            assert np.allclose(g[k], num, rtol=1e-6, atol=1e-8), k
        checked += 1
    assert checked >= 2


def test_hand_evaluated_network():
    # one hidden unit per layer, hidden = 1: y = w3 relu(W2 relu(W1 x + b1) + b2) + b3
    p = {"W1": np.array([[2.0, -1.0]]), "b1": np.array([0.5]), "W2": np.array([[3.0]]), "b2": np.array([-1.0]),
         "w3": np.array([0.25]), "b3": np.array([4.0])}
    X = np.array([[1.0, 1.0], [0.0, 2.0]])
    y, _ = mlp.forward(p, X)
    # row 0: a1 = 2 - 1 + 0.5 = 1.5; a2 = 4.5 - 1 = 3.5; y = 0.875 + 4
    # row 1: a1 = -2 + 0.5 < 0 -> 0; a2 = -1 -> 0; y = 4
    assert np.allclose(y, [4.875, 4.0])
    zero = {k: np.zeros_like(v) for k, v in p.items()}
    zero["b3"] = np.array([-1.5])
    assert np.allclose(mlp.forward(zero, X)[0], -1.5)


def test_adam_properties():
    rng = np.random.default_rng(1)
    p, X, t = _small(7)
    _, g = mlp.loss_and_grads(p, X, t)
    zeros = {k: np.zeros_like(v) for k, v in p.items()}
    lr = 1e-3
    p1, m1, v1 = mlp.adam_step(p, g, zeros, zeros, 1, lr)
    for k in mlp.PARAMS:
        step = p[k] - p1[k]
        nz = np.abs(g[k]) > 1e-3   # eps = 1e-8 changes the step by < 1e-5 relative there
        assert np.allclose(np.abs(step[nz]), lr, rtol=1e-4)          # bias-corrected first step
        assert np.all(np.sign(step[nz]) == np.sign(g[k][nz]))
    # invariance under gradient rescaling
    g5 = {k: 5.0 * v for k, v in g.items()}
    p1b, _, _ = mlp.adam_step(p, g5, zeros, zeros, 1, lr)
    for k in mlp.PARAMS:
        assert np.allclose(p1b[k], p1[k], atol=1e-9)
    # a constant gradient keeps moving every coordinate by lr per step
    q, m, v = p, zeros, zeros
    for s in range(1, 6):
        q, m, v = mlp.adam_step(q, g, m, v, s, lr)
    for k in mlp.PARAMS:
        nz = np.abs(g[k]) > 1e-3   # eps = 1e-8 changes the step by < 1e-5 relative there
        assert np.allclose(np.abs(p[k] - q[k])[nz], 5 * lr, rtol=1e-4)
    _ = rng


def test_feature_vector_by_hand():
    beta, nf = 10.0, 2
    # flavor 0: segment [1, 3] (length 2 -> bin 6) and segment [9, 0.5] wrapping (length 1.5 -> bin 4)
    # flavor 1: c at 4, c^+ at 6: one segment from 6 to 4 wrapping (length 8 -> bin 25)
    ops = [(0.5, 0, 0), (1.0, 0, 1), (3.0, 0, 0), (4.0, 1, 0), (6.0, 1, 1), (9.0, 0, 1)]
    # insertion of an anti-segment of flavor 1 (c at 5, c^+ at 5.5): the base is the configuration itself
    x = mlp.features(ops, nf, beta, kind=0, flavor=1, t_first=5.0, t_second=5.5, seg=False)
    assert len(x) == mlp.n_inputs(nf) == 80
    # occupied fractions of [5, 5.5): flavor 0 is empty there, flavor 1 occupied (its segment 6 -> 4 wraps)
    assert x[34 * nf + 3] == 0.0 and x[34 * nf + 4] == 0.0
    assert x[0] == 2 / 8 and x[1] == 1 / 8
    hist = x[nf:nf + 32 * nf].reshape(nf, 32)
    assert hist[0, 6] == 0.25 and hist[0, 4] == 0.25 and hist[1, 25] == 0.25 and hist.sum() == 0.75
    base = 33 * nf
    assert x[base] == 0.0 and x[base + 1 + 1] == 1.0 and x[base + 1] == 0.0
    assert abs(x[base + 1 + nf] - 0.05) < 1e-15 and x[base + 2 + nf] == -1.0
    assert not x[base + 3 + nf:34 * nf + 3].any() and not x[35 * nf + 3:].any()
    # removal of flavor 1's pair (the c^+ at 6 and the c at 4 after it): the base has no flavor-1 operator
    y = mlp.features(ops, nf, beta, kind=1, flavor=1, t_first=6.0, t_second=4.0, seg=True)
    hy = y[nf:nf + 32 * nf].reshape(nf, 32)
    assert y[1] == 0.0 and hy[1].sum() == 0.0 and hy[0, 6] == 0.25 and hy[0, 4] == 0.25
    assert abs(y[base + 1 + nf] - 0.8) < 1e-15 and y[base + 2 + nf] == 1.0
    # occupied fractions of the removed pair's interval [6, 4) (length 8, wrapping), base without
    # flavor 1: flavor 0 holds [9, 0.5) and [1, 3) inside it -> (1.5 + 2) / 8
    assert abs(y[34 * nf + 3] - 3.5 / 8) < 1e-15 and y[34 * nf + 4] == 0.0
    # a move and its reverse share their features: inserting that pair into the base
    z = mlp.features([op for op in ops if op[1] != 1], nf, beta, kind=0, flavor=1, t_first=6.0, t_second=4.0,
                     seg=True)
    assert np.array_equal(y, z)
    assert math.isclose(mlp.features([], nf, beta, 0, 0, 2.0, 7.0, False)[base + 1 + nf], 0.5)
    # cyclic overlaps by hand
    assert mlp._overlap(9.0, 3.0, 1.0, 1.0, beta) == 1.0     # [9, 12) wraps to cover [1, 2)
    assert mlp._overlap(2.0, 1.0, 5.0, 1.0, beta) == 0.0
    assert mlp._overlap(0.0, 10.0, 4.0, 10.0, beta) == 10.0


def test_bf16_rounding_against_hand_values():
    """bfloat16 keeps 8 significand bits (7 stored): 1 + 2^-8 is a tie between 1 and 1 + 2^-7 and goes
    to the even one (1); 1 + 3 * 2^-8 ties up to 1 + 2^-6; values just above a tie round up;
    signs and powers of two pass unchanged."""
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -(1 + 2 ** -8 + 2 ** -20), 2.0 ** -130,
                     3.0, 0.0, -2.0 ** 40])
    want = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -(1 + 2 ** -7), 2.0 ** -130, 3.0, 0.0, -2.0 ** 40])
    assert np.array_equal(mlp.bf16(vals), want)
    bits = np.array([0x3F80, 0xBF80, 0x4040, 0x0000], np.uint16)
    assert np.array_equal(mlp.from_bf16_bits(bits), [1.0, -1.0, 3.0, 0.0])
    # every output is representable: rounding twice changes nothing
    x = np.random.default_rng(1).normal(0, 5, 2000)
    assert np.array_equal(mlp.bf16(mlp.bf16(x)), mlp.bf16(x))
    assert np.abs(mlp.bf16(x) / x - 1).max() <= 2.0 ** -8   # unit roundoff of 8 significand bits


def test_bf16_chain_reduces_to_the_exact_one(monkeypatch):
    """loss_and_grads_bf16 is the chain rule of loss_and_grads with rounding points added:
    with the rounding replaced by the identity it must give the same loss and gradients."""
    p, X, t = _small(4)
    monkeypatch.setattr(mlp, "bf16", lambda a: np.asarray(a, dtype=np.float64))
    L1, g1, _ = mlp.loss_and_grads_bf16(p, X, t)
    L0, g0 = mlp.loss_and_grads(p, X, t)
    assert L1 == L0
    for k in mlp.PARAMS:
        assert np.allclose(g1[k], g0[k], rtol=1e-13, atol=1e-15), k
