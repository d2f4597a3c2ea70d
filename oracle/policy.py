"""Oracle of the on-device policy (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module; it shares nothing with the CUDA library.

The policy is the actor of the PPO agent the paper trains (Sec. 5, Table
"PPO hyper-parameters"): a multilayer perceptron from the observation of one
station to one categorical distribution over the action levels of each
charger (the MultiDiscrete action of App. A.2 "Apply Actions").  Written
here in FP64 with the rounding points of the BF16 tensor-core form made
explicit:

    h1 = bf16(relu(W1 bf16(obs) + b1))
    h2 = bf16(relu(W2 h1 + b2))
    logits = W3 h2 + b3                     (row c * L + j: level j of charger c)

``bf16`` is round to nearest, ties to even, to 8 significant bits (pinned
against torch's float32 -> bfloat16 conversion and hand values).  The
sample of a charger is the inverse transform of its softmax: the number of
j < L - 1 whose cumulative probability is <= u.

Exact agreement with the kernel is not expected for the logits: the kernel
accumulates in FP32 in its own order, and an activation whose FP32 value
lands on the other side of a BF16 rounding boundary moves by one BF16 step.
``mlp_bound`` propagates those two effects through the layers as a
first-order worst-case bound per logit (derived in the function).
"""
from __future__ import annotations

import numpy as np

# FP32 accumulation: every partial sum may be rounded, relative error at most
# u = 2^-24 per addition; 2^-23 leaves room for a tensor core that truncates
# instead of rounding.
ACC_UNIT = 2.0 ** -23
# BF16 rounding: |bf16(x) - x| <= 2^-8 |x|.  With 8 significant bits the
# spacing of BF16 numbers in [2^e, 2^(e+1)) is 2^(e-7); half of it is
# 2^(e-8) <= 2^-8 |x|, reached for x just above 2^e (1 + 2^-8 rounds to 1).
BF16_HALF_STEP = 2.0 ** -8


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 number, ties to even (8 significant bits).
    Written from the format: x = m 2^e with m in [0.5, 1); keep 8 bits of
    m.  Overflow and subnormals do not occur for the values used here."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def relu(x):
    return np.maximum(x, 0.0)


def mlp_forward(obs, w):
    """Logits [rows, N * L] for observations [rows, D]; ``w`` has W1 [H, D],
    b1 [H], W2 [H, H], b2 [H], W3 [N * L, H], b3 [N * L] (weights BF16
    values).  Returns (logits, h1, h2)."""
    W1, b1, W2, b2, W3, b3 = (np.asarray(a, np.float64) for a in (w.w1, w.b1, w.w2, w.b2, w.w3, w.b3))
    x = bf16(obs)
    h1 = bf16(relu(x @ W1.T + b1))
    h2 = bf16(relu(h1 @ W2.T + b2))
    return h2 @ W3.T + b3, h1, h2


def mlp_bound(obs, w):
    """Worst-case |kernel logit - oracle logit| to first order.

    For a layer z = W a + b computed in FP32 from the same inputs a, the
    accumulation error is at most g_K * sum_k |W_jk| |a_k| with g_K = K u.
    If the inputs differ by da, z differs by at most sum_k |W_jk| da_k more.
    ReLU does not increase a difference, and BF16 rounding of two values
    that differ by dz gives results that differ by at most
    dz + h (|x| + |x'|) <= dz + 2 h (|x| + dz), h = BF16_HALF_STEP.
    Both parts are reached: an FP32 sum that truncates every partial sum
    loses almost K u of the largest partial sum, and two values on either
    side of a BF16 tie just above a power of two round one step apart."""
    W1, b1, W2, b2, W3, b3 = (np.asarray(a, np.float64) for a in (w.w1, w.b1, w.w2, w.b2, w.w3, w.b3))
    x = bf16(obs)
    A1, A2, A3 = np.abs(W1), np.abs(W2), np.abs(W3)
    z1 = x @ W1.T + b1
    dz1 = W1.shape[1] * ACC_UNIT * (np.abs(x) @ A1.T + np.abs(b1))
    h1 = bf16(relu(z1))
    dh1 = dz1 + 2 * BF16_HALF_STEP * (np.abs(relu(z1)) + dz1)
    z2 = h1 @ W2.T + b2
    dz2 = dh1 @ A2.T + W2.shape[1] * ACC_UNIT * ((np.abs(h1) + dh1) @ A2.T + np.abs(b2))
    h2 = bf16(relu(z2))
    dh2 = dz2 + 2 * BF16_HALF_STEP * (np.abs(relu(z2)) + dz2)
    return dh2 @ A3.T + W3.shape[1] * ACC_UNIT * ((np.abs(h2) + dh2) @ A3.T + np.abs(b3))


def sample(logits, u, n_levels: int):
    """Levels [rows, N] from logits [rows, N * L] and uniforms [rows, N] by
    inverse transform of each charger's softmax.  Also returns the margin:
    the smallest |cumulative probability - u| over the compared boundaries
    (a sample whose margin is below the rounding of the FP32 form may
    legitimately come out one level off)."""
    rows = logits.shape[0]
    lg = np.asarray(logits, np.float64).reshape(rows, -1, n_levels)
    e = np.exp(lg - lg.max(axis=2, keepdims=True))
    cum = np.cumsum(e, axis=2) / e.sum(axis=2, keepdims=True)
    inner = cum[:, :, : n_levels - 1]
    uu = np.asarray(u, np.float64)[:, :, None]
    levels = (inner <= uu).sum(axis=2)
    margin = np.abs(inner - uu).min(axis=2)
    return levels.astype(np.int64), margin
