"""Pins of the policy oracle against what the mathematics fixes: BF16
rounding against a library conversion and hand values, the MLP against
closed forms (bias only, two-hot layers), the sampler against its
closed form for equal logits, a dominant logit and the categorical
frequencies, and the error bound against an independent FP32 evaluation
(sound) and against hand networks on which an adversarial FP32 evaluation
reaches it (tight)."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from oracle import policy as OP
from paper_2507_01522_b300 import inputs as I


def test_bf16_matches_library_conversion():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200_000) * np.exp(rng.uniform(-20, 20, 200_000))).astype(np.float32)
    # exact ties: low 16 bits 0x8000, both parities of bit 16
    u = x.view(np.uint32)
    ties = ((u[:1000] & np.uint32(0xFFFF0000)) | np.uint32(0x8000)).view(np.float32)
    x = np.concatenate([x, ties, np.float32([0.0, -0.0, 1.0, -1.0])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(OP.bf16(x), ref)


def test_bf16_hand_values():
    assert OP.bf16(1.0 + 2.0 ** -8) == 1.0                       # tie, 1.0 is even
    assert OP.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6      # tie, rounds up to even
    assert OP.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert OP.bf16(-3.0) == -3.0
    assert OP.bf16(255.5) == 256.0                               # 8 significant bits


def _weights(H=16, D=12, N=3, L=4, seed=0, **kw):
    return I.policy_weights(D, N, n_levels=L, hidden=H, seed=seed, **kw)


def test_mlp_bias_only():
    w = _weights(bias_scale=1.0, head_gain=1.0)
    w.w3[:] = 0
    obs = np.random.default_rng(1).standard_normal((5, 12)).astype(np.float32)
    logits, _, _ = OP.mlp_forward(obs, w)
    np.testing.assert_array_equal(logits, np.broadcast_to(w.b3.astype(np.float64), logits.shape))


def test_mlp_two_hot_layers():
    """Each layer a "two-hot" matrix (row j has ones at columns p[j] and
    q[j]): every unit is the sum of two rounded inputs plus its bias, so a
    transposed operand, a missing ReLU, a missing or misplaced BF16
    rounding, or a bias in the wrong place gives a different number."""
    H = D = 8
    N, L = 2, 4
    rng = np.random.default_rng(2)
    w = _weights(H=H, D=D, N=N, L=L)
    perms = []
    for W in (w.w1, w.w2, w.w3):
        p, q = rng.permutation(H), np.roll(rng.permutation(H), 1)
        q = np.where(q == p, (q + 1) % H, q)
        W[:] = 0
        W[np.arange(H), p] = 1
        W[np.arange(H), q] = 1
        perms.append((p, q))
    w.b1[:] = np.float32([0.5, -0.25, 1.0, -2.0, 0.125, 3.0, -0.75, 0.0])
    w.b2[:] = np.float32([-0.5, 0.25, 0.75, 1.5, -1.0, 0.0, 2.0, -3.0])
    w.b3[:] = np.float32([1, 2, 3, 4, 5, 6, 7, 8])
    obs = (np.float32([[0.1, -0.3, 1.7, 2.3, -5.1, 0.6, 0.77, 9.3]]) * np.float32(1.0 + 2.0 ** -12))
    logits, _, _ = OP.mlp_forward(obs, w)
    x = [OP.bf16(float(v)) for v in obs[0]]
    (p1, q1), (p2, q2), (p3, q3) = perms
    h1 = [OP.bf16(max(x[p1[j]] + x[q1[j]] + float(w.b1[j]), 0.0)) for j in range(H)]
    h2 = [OP.bf16(max(h1[p2[j]] + h1[q2[j]] + float(w.b2[j]), 0.0)) for j in range(H)]
    expect = [h2[p3[j]] + h2[q3[j]] + float(w.b3[j]) for j in range(H)]
    np.testing.assert_array_equal(logits[0], expect)
    # the rounding points matter for these inputs
    h1_exact = [max(float(obs[0, p1[j]]) + float(obs[0, q1[j]]) + float(w.b1[j]), 0.0) for j in range(H)]
    assert any(OP.bf16(v) != v for v in h1_exact)


def test_sample_tie_counts_as_below():
    """L = 4 equal logits: cumulative probabilities exactly 1/4, 1/2, 3/4.
    u on a boundary counts that boundary (level = #{C_j <= u})."""
    logits = np.zeros((3, 4))
    lv, margin = OP.sample(logits, np.array([[0.25], [0.5], [0.75]]), 4)
    np.testing.assert_array_equal(lv[:, 0], [1, 2, 3])
    np.testing.assert_array_equal(margin[:, 0], [0, 0, 0])


def test_sample_equal_logits_is_floor():
    """Equal logits: cumulative probabilities (j+1)/L, so the level is
    floor(u L) away from the boundaries."""
    L, N = 11, 7
    rng = np.random.default_rng(3)
    u = rng.uniform(0, 1, (1000, N))
    logits = np.full((1000, N * L), 0.37)
    lv, margin = OP.sample(logits, u, L)
    ok = margin > 1e-12
    np.testing.assert_array_equal(lv[ok], np.floor(u[ok] * L).astype(np.int64))


def test_sample_dominant_logit():
    L, N = 11, 4
    rng = np.random.default_rng(4)
    best = rng.integers(0, L, (500, N))
    logits = rng.standard_normal((500, N, L))
    np.put_along_axis(logits, best[:, :, None], 80.0, axis=2)
    lv, _ = OP.sample(logits.reshape(500, -1), rng.uniform(1e-6, 1 - 1e-6, (500, N)), L)
    np.testing.assert_array_equal(lv, best)


def test_sample_frequencies_follow_softmax():
    """Chi-square of 400k draws against the softmax probabilities."""
    L = 11
    rng = np.random.default_rng(5)
    lg = rng.standard_normal(L) * 1.5
    n = 400_000
    lv, _ = OP.sample(np.broadcast_to(lg, (n, L)), rng.uniform(0, 1, (n, 1)), L)
    counts = np.bincount(lv[:, 0], minlength=L)
    p = np.exp(lg - lg.max())
    p /= p.sum()
    chi2 = float(((counts - n * p) ** 2 / (n * p)).sum())
    assert chi2 < 40.0                                           # 10 dof: p ~ 1e-5


def _fp32_forward(obs, w, reverse):
    """The same network in float32 with another summation order."""
    def layer(a, W, b):
        prods = a[:, None, :].astype(np.float32) * W[None, :, :].astype(np.float32)
        if reverse:
            prods = prods[:, :, ::-1]
        acc = np.zeros(prods.shape[:2], np.float32)
        for k in range(prods.shape[2]):
            acc = acc + prods[:, :, k]
        return acc + b.astype(np.float32)
    x = torch.from_numpy(obs.astype(np.float32)).to(torch.bfloat16).float().numpy()
    h1 = torch.from_numpy(np.maximum(layer(x, w.w1, w.b1), 0)).to(torch.bfloat16).float().numpy()
    h2 = torch.from_numpy(np.maximum(layer(h1, w.w2, w.b2), 0)).to(torch.bfloat16).float().numpy()
    return layer(h2, w.w3, w.b3).astype(np.float64)


@pytest.mark.parametrize("reverse", [False, True])
def test_bound_covers_fp32_evaluation(reverse):
    D, N, L, H = 20, 3, 11, 64
    w = _weights(H=H, D=D, N=N, L=L, seed=6, head_gain=1.0, bias_scale=0.5)
    obs = np.random.default_rng(7).uniform(-1, 3, (64, D)).astype(np.float32)
    ref, _, _ = OP.mlp_forward(obs, w)
    bound = OP.mlp_bound(obs, w)
    got = _fp32_forward(obs, w, reverse)
    assert np.all(np.abs(got - ref) <= bound)
    # not vacuous (a worst case over every rounding position: about a tenth
    # of the logits' range for this 64-unit network)
    assert np.all(bound < 0.15 * (np.abs(ref).max() + 1))


def test_policy_uniforms_are_the_policy_philox_words():
    from oracle import philox
    w = I.small_uniform(n_envs=3)
    o = Oracle(w, seed=123)
    o.step()
    o.step()
    n = int(w.stations.n_ports[0])
    u = o.policy_uniforms(n)
    st = o.state()
    for e in range(3):
        for q in range(n):
            words = philox([e, int(st["gstep"][e]), q // 4, 4], [int(st["key0"][e]), int(st["key1"][e])])
            assert u[e, q] == (int(words[q % 4]) >> 8) * 2.0 ** -24


# ----------------------------------------------------------------------------
# tightness of the bound: hand networks on which a legitimate FP32 evaluation
# reaches the worst case the bound allows
# ----------------------------------------------------------------------------

def _rtz32(x: float) -> float:
    """Round a double to FP32 toward zero (a tensor core that truncates)."""
    f = np.float32(x)
    if abs(float(f)) > abs(x):
        f = np.nextafter(f, np.float32(0.0))
    return float(f)


def _truncating_forward(obs, w):
    """FP32 evaluation in which every partial sum is truncated (round toward
    zero), starting from the bias as the kernel does, products exact (BF16
    x BF16 fits FP32), BF16 rounding to nearest even at the same points as
    the oracle.  The bound must cover it (its FP32 unit is 2^-23, room for
    truncation)."""
    def layer(a, W, b):
        out = np.empty((a.shape[0], W.shape[0]))
        for r in range(a.shape[0]):
            for j in range(W.shape[0]):
                acc = float(np.float32(b[j]))
                for k in range(W.shape[1]):
                    acc = _rtz32(acc + float(W[j, k]) * float(a[r, k]))
                out[r, j] = acc
        return out
    x = OP.bf16(obs)
    h1 = OP.bf16(OP.relu(layer(x, w.w1, w.b1)))
    h2 = OP.bf16(OP.relu(layer(h1, w.w2, w.b2)))
    return layer(h2, w.w3, w.b3)


def _net(w1, b1, w2, b2, w3, b3):
    f = lambda a: np.asarray(a, np.float32)
    return I.PolicyWeights(f(w1), f(b1), f(w2), f(b2), f(w3), f(b3))


def test_bound_is_reached_by_bf16_ties():
    """One unit per layer.  Layer 1 sums 1 + 2^-8 (a BF16 tie just above 1)
    and 62 inputs of 2^-30: exactly the sum lies above the tie and rounds up
    to 1 + 2^-7, while the truncating sum drops the small inputs, sits on the
    tie and rounds to 1.  Layer 2 adds 2^-8: 1 + 3 2^-8 is again a tie, which
    rounds up to 1 + 2^-6, and 1 + 2^-8 rounds down to 1.  The logits then
    differ by 2^-6, one step of each rounding; the bound may exceed that only
    by its accumulation terms (a few parts in 1e3)."""
    D = 64
    obs = np.array([[1.0, 2.0 ** -8] + [2.0 ** -30] * (D - 2)])
    w = _net(np.ones((1, D)), [0.0], [[1.0]], [2.0 ** -8], [[1.0]], [0.0])
    ref, h1, h2 = OP.mlp_forward(obs, w)
    assert h1[0, 0] == 1 + 2.0 ** -7 and h2[0, 0] == 1 + 2.0 ** -6
    got = _truncating_forward(obs, w)
    attained = abs(got[0, 0] - ref[0, 0])
    assert attained == 2.0 ** -6
    bound = OP.mlp_bound(obs, w)[0, 0]
    assert attained <= bound <= 1.05 * attained, (attained, bound)


def test_bound_is_reached_by_truncated_accumulation():
    """256 hidden units of 15/128 (biases through identity layers) and a
    logit that starts from a bias of 2^20: each product 15/128 is below the
    FP32 spacing at 2^20 (2^-3), so a truncating sum keeps 2^20 while the
    exact logit is 2^20 + 30.  The bound's accumulation term, 256 2^-23
    (2^20 + 30) = 32.0, must cover the 30 and may exceed it only by that
    term's slack and the small rounding terms of the hidden layers."""
    H, D = 256, 8
    obs = np.zeros((1, D))
    w = _net(np.zeros((H, D)), np.full(H, 15.0 / 128.0), np.eye(H), np.zeros(H), np.ones((1, H)), [2.0 ** 20])
    ref, h1, h2 = OP.mlp_forward(obs, w)
    assert np.all(h2 == 15.0 / 128.0) and ref[0, 0] == 2.0 ** 20 + 30.0
    got = _truncating_forward(obs, w)
    attained = abs(got[0, 0] - ref[0, 0])
    assert attained == 30.0
    bound = OP.mlp_bound(obs, w)[0, 0]
    assert attained <= bound <= 1.25 * attained, (attained, bound)
