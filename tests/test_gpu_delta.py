"""Parity of the Delta-current action form (A.2 "Apply Actions": a level is an
increment of the charger's, or the battery's, last applied power; a
departed car's charger drops to 0) with the oracle, in the charge-only and
V2G modes, plain and fused kernels, through the C interface: events exact,
floats within the tolerances of tests/parity.py."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2507_01522_b300 import inputs as I

from test_gpu_parity import odd_sizes, stressed
from test_gpu_v2g import V2G, check_single_steps, compare_traj

pytestmark = pytest.mark.gpu

BASE = {"odd150": odd_sizes, "stressed": stressed, "hetero64": lambda: I.heterogeneous(n_envs=64)}


def make(name, v2g):
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w = BASE[name]()
    extra = dict(V2G) if v2g else dict(n_levels=21)
    w.params = I.EnvParams(**{**w.params.__dict__, **extra, "action_delta": 1})
    return w, Batch(w), Oracle(w), torch


def small_increments(rng, b, steps, spread=2):
    """Levels within +-spread of the idle level: slow ramps that stay off the
    caps for many steps, so the running sum of increments is exercised."""
    h = (b.workload.params.n_levels - 1) // 2
    return rng.integers(h - spread, h + spread + 1, size=(b.n_actions, steps)).astype(np.int8)


CASES = [("odd150", False), ("stressed", False), ("stressed", True), ("hetero64", True)]


@pytest.mark.parametrize("name,v2g", CASES)
@pytest.mark.parametrize("mode,k", [("plain", 1), ("fused", 24)])
def test_delta_random_levels(cuda_lib, name, v2g, mode, k):
    w, b, o, torch = make(name, v2g)
    n_done = compare_traj(w, b, o, torch, 72, mode=mode, k=k)
    if name == "stressed":
        assert n_done > 0


@pytest.mark.parametrize("name,v2g", CASES)
@pytest.mark.parametrize("mode,k", [("plain", 1), ("fused", 16)])
def test_delta_small_increments(cuda_lib, name, v2g, mode, k):
    w, b, o, torch = make(name, v2g)
    acts = small_increments(np.random.default_rng(12), b, 64)
    compare_traj(w, b, o, torch, 64, mode=mode, k=k, actions=acts)
    pw = b.get_state()["p"]
    assert (pw > 0).any()
    if v2g:
        assert (pw < 0).any()


@pytest.mark.parametrize("v2g", [False, True])
@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_delta_single_step_from_oracle_state(cuda_lib, v2g, mode):
    w, b, o, torch = make("stressed", v2g)
    check_single_steps(w, b, o, torch, mode, np.random.default_rng(13), lambda rng: small_increments(rng, b, 1, 4)[:, 0])


def test_delta_checkpoint_resume_bit_exact(cuda_lib):
    w, b, o, torch = make("odd150", True)
    acts = torch.from_numpy(small_increments(np.random.default_rng(14), b, 40)).cuda()
    b.step_n(10, actions=acts[:, :10].contiguous(), lda=10)
    blob = b.save()
    r1 = torch.zeros(b.E, 30, device="cuda")
    b.step_n(30, actions=acts[:, 10:].contiguous(), reward=r1, lda=30)
    s1 = b.get_state()
    b.load(blob)
    r2 = torch.zeros(b.E, 30, device="cuda")
    b.step_n(30, actions=acts[:, 10:].contiguous(), reward=r2, lda=30)
    assert torch.equal(r1, r2)
    s2 = b.get_state()
    for key in s1:
        np.testing.assert_array_equal(s1[key], s2[key])


def test_delta_rejections(cuda_lib):
    from paper_2507_01522_b300.chargax import CHX_EINVAL, Batch, ChxError
    w = I.small_uniform()
    w.params.action_delta = 1
    w.params.n_levels = 10                                   # increments need an odd count
    with pytest.raises(ChxError) as ei:
        Batch(w)
    assert ei.value.code == CHX_EINVAL
    w.params.n_levels = 11
    b = Batch(w)
    pw = I.policy_weights(8 + 6 * 16, 16)
    with pytest.raises(ChxError) as ei:                      # the on-device policy samples absolute levels
        b.policy_load(pw.w1, pw.b1, pw.w2, pw.b2, pw.w3, pw.b3)
    assert ei.value.code == CHX_EINVAL
    w2 = I.v2g_variant(I.small_uniform())
    w2.params.p_max_dis_kw = (0.0, 50.0)
    with pytest.raises(ChxError) as ei:
        Batch(w2)
    assert ei.value.code == CHX_EINVAL
