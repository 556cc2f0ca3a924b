"""Plain FP64 reference of the delayed-acceptance surrogate (test infrastructure only).

Only the tests import this module; the product library never calls it.

The surrogate predicts the log of the trace ratio |T_new / T_old| of a proposed local
update from a feature vector x of a configuration and the move's pair:

    y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3,     W1: [H, n_in], W2: [H, H], w3: [H]

trained on the mean squared error L = (1/B) sum_b (y_b - t_b)^2 with Adam (Kingma & Ba,
"Adam: a method for stochastic optimization", 2015, Algorithm 1: beta1 = 0.9,
beta2 = 0.999, eps = 1e-8, bias-corrected moments). Everything here is written out in
FP64 with numpy products; the backward pass is the chain rule of the three layers.

The network predicts the log trace ratio of INSERTING a pair into the configuration
that does not hold it (the base): for an insertion the base is the current
configuration, for a removal it is the current configuration without the pair, and the
removal's prediction is minus the network's output. The surrogate is then exactly
antisymmetric (a move and its reverse share the features and get opposite
predictions), which is what makes the second delayed-acceptance stage
min(1, R / R~) exact (Christen & Fox: stage 2 carries alpha1(y, x) / alpha1(x, y),
equal to 1 / R~ only for an antisymmetric surrogate).

Features of the base and the pair (a reading of "per-flavor operator counts, a 32-bin
histogram of segment lengths per flavor, and the move type"; the pair is described by
its flavor, length and orientation, because the log ratio depends on it):
    x[f]                      = k_f / 8                 pairs of flavor f in the base
    x[nf + 32 f + b]         += 1/4 for every segment of flavor f in the base (a c^+ to
                                the next c of f, cyclically) whose length l has
                                b = min(floor(32 l / beta), 31)
    x[33 nf]                  = 0 (unused)
    x[33 nf + 1 + f_move]     = 1
    x[34 nf + 1]              = ((t_second - t_first) mod beta) / beta, the distance from
                                the pair's first operator (t1 of an insertion, the chosen
                                operator of a removal) to its partner
    x[34 nf + 2]              = +1 when the first operator is a c^+ (segment), else -1
    x[34 nf + 3 + g]          = the fraction of the pair's interval (from its first
                                operator to its partner, cyclically) during which flavor g
                                is occupied in the base (segments of g as above)
    the rest (up to n_in, a multiple of 16) is 0.
The occupied fractions carry what decides the insertion cost: which other flavors
hold an electron while the pair's flavor changes its occupation.
"""
from __future__ import annotations

import math

import numpy as np

PARAMS = ("W1", "b1", "W2", "b2", "w3", "b3")


def n_inputs(nf: int) -> int:
    n = 35 * nf + 3
    return (n + 15) // 16 * 16


def _overlap(a0: float, a1: float, b0: float, b1: float, beta: float) -> float:
    """Length of the intersection of the cyclic intervals [a0, a0 + a1) and [b0, b0 + b1)
    (start in [0, beta), lengths at most beta)."""
    tot = 0.0
    for k in (-1.0, 0.0, 1.0):
        lo = max(a0, b0 + k * beta)
        hi = min(a0 + a1, b0 + b1 + k * beta)
        tot += max(0.0, hi - lo)
    return tot


def shapes(n_in: int, hidden: int = 256):
    return {"W1": (hidden, n_in), "b1": (hidden,), "W2": (hidden, hidden), "b2": (hidden,), "w3": (hidden,),
            "b3": (1,)}


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in PARAMS])


def unpack(v: np.ndarray, n_in: int, hidden: int = 256) -> dict:
    out, o = {}, 0
    for k, s in shapes(n_in, hidden).items():
        n = int(np.prod(s))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(s)
        o += n
    return out


def init(n_in: int, seed: int, hidden: int = 256) -> dict:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    return {"W1": rng.normal(0.0, math.sqrt(2.0 / n_in), (hidden, n_in)), "b1": np.zeros(hidden),
            "W2": rng.normal(0.0, math.sqrt(2.0 / hidden), (hidden, hidden)), "b2": np.zeros(hidden),
            "w3": rng.normal(0.0, math.sqrt(2.0 / hidden), hidden), "b3": np.zeros(1)}


def forward(p: dict, X: np.ndarray):
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (a1, h1, a2, h2)


def loss_and_grads(p: dict, X: np.ndarray, t: np.ndarray):
    B = X.shape[0]
    y, (a1, h1, a2, h2) = forward(p, X)
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / B
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    da2 = np.outer(dy, p["w3"]) * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    return L, g


def bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16, ties to even, through FP32 (the value is first rounded
    to FP32, as the kernels hold it); returned as float64. bfloat16 is the upper half of an
    IEEE FP32 word, so rounding adds half an ulp of the lower 16 bits (plus the tie bit)."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def from_bf16_bits(b) -> np.ndarray:
    """bfloat16 bit patterns (uint16) as float64."""
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def loss_and_grads_bf16(p: dict, X: np.ndarray, t: np.ndarray):
    """The chain rule of loss_and_grads with the rounding points of a BF16 tensor-core
    implementation: the hidden activations H1 and the back-propagated dZ2 and dZ1 are
    rounded to BF16 (they are the operands of the products), the bias gradients are sums of
    the unrounded values, and everything else stays FP64. The weights and X are used as
    given (pass BF16-representable W1, W2, X). Returns (L, grads, intermediates)."""
    B = X.shape[0]
    a1 = X @ p["W1"].T + p["b1"]
    h1 = bf16(np.maximum(a1, 0.0))
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / B
    e2 = np.outer(dy, p["w3"]) * (a2 > 0)
    dz2 = bf16(e2)
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()]), "b2": e2.sum(axis=0), "W2": dz2.T @ h1}
    dh1 = dz2 @ p["W2"]
    e1 = dh1 * (a1 > 0)
    dz1 = bf16(e1)
    g["b1"] = e1.sum(axis=0)
    g["W1"] = dz1.T @ X
    return L, g, {"a1": a1, "h1": h1, "a2": a2, "h2": h2, "y": y, "dy": dy, "dz2": dz2, "dh1": dh1, "dz1": dz1}


def adam_step(p: dict, g: dict, m: dict, v: dict, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    np_, nm, nv = {}, {}, {}
    for k in PARAMS:
        nm[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
        nv[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k]
        mh = nm[k] / (1.0 - beta1 ** step)
        vh = nv[k] / (1.0 - beta2 ** step)
        np_[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return np_, nm, nv


def base_config(ops, kind: int, flavor: int, t_first: float, t_second: float):
    """The configuration without the move's pair (the current one for an insertion)."""
    if kind == 0:
        return list(ops)
    out, dropped = [], 0
    for t, g, d in ops:
        if g == flavor and (t == t_first or t == t_second) and dropped < 2:
            dropped += 1
            continue
        out.append((t, g, d))
    return out


def features(ops, nf: int, beta: float, kind: int, flavor: int, t_first: float, t_second: float, seg: bool,
             n_in: int | None = None) -> np.ndarray:
    """The surrogate's input for the configuration `ops` and one proposed move."""
    n_in = n_inputs(nf) if n_in is None else n_in
    ops = base_config(ops, kind, flavor, t_first, t_second)
    x = np.zeros(n_in)
    d = t_second - t_first
    if d < 0:
        d += beta
    for f in range(nf):
        mine = [(t, dg) for t, g, dg in ops if g == f]
        x[f] = sum(1 for t, dg in mine if dg == 1) / 8.0
        occ = 0.0
        for i, (t, dg) in enumerate(mine):
            if dg != 1:
                continue
            tn = mine[(i + 1) % len(mine)][0]
            ln = tn - t if tn > t else tn + beta - t
            b = min(int(ln / beta * 32), 31)
            x[nf + 32 * f + b] += 0.25
            occ += _overlap(t, ln, t_first, d, beta)
        if d > 0:
            x[34 * nf + 3 + f] = occ / d
    base = 33 * nf
    x[base + 1 + flavor] = 1.0
    x[base + 1 + nf] = d / beta
    x[base + 2 + nf] = 1.0 if seg else -1.0
    return x
