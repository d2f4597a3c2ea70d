"""chx_rollout_noalloc, the rollout for callers that cannot allocate device
memory during the call (for example code running under a memory pool it does
not own): it must give the same results as chx_rollout, call after call,
while keeping its scratch in a static device array.

Kept in a file of its own whose name sorts last, so pytest collects it after
every other test: a run that stops at the first failure (-x) has then run all
the other tests before this one.  It does not depend on that order; it passes
alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from parity import STEP_RTOL

pytestmark = pytest.mark.gpu


def _extended():
    """Fig. c trees in V2G mode with increment levels and charge-sensitive
    users: the extended tree instances."""
    from paper_2507_01522_b300 import inputs as I
    w = I.tree_workload(300, seed=8)
    w.params = I.EnvParams(**{**w.params.__dict__, "v2g": 1, "n_levels": 21, "action_delta": 1,
                              "cs_share_256": 128, "soc_target": 0.8})
    return w


@pytest.mark.parametrize("form", ["charge-only", "extended"])
def test_rollout_noalloc_matches_rollout_twice(cuda_lib, form):
    import torch
    from paper_2507_01522_b300 import inputs as I
    from paper_2507_01522_b300.chargax import Batch
    w = I.heterogeneous(n_envs=1000) if form == "charge-only" else _extended()
    a, b = Batch(w), Batch(w)                      # identical batches, identical seeds
    for x in (a, b):
        x.set_launch(steps_per_launch=24, warps_per_block=4)
    n = 100                                         # 5 launches per call
    for call in range(2):                           # the scratch keeps the last call's contents
        ra = torch.zeros(a.E, n, device="cuda")
        da = torch.zeros(a.E, n, dtype=torch.uint8, device="cuda")
        oa = torch.zeros(a.obs_size, device="cuda")
        rb, db, ob = torch.zeros_like(ra), torch.zeros_like(da), torch.zeros_like(oa)
        a.rollout(n, reward=ra, done=da, obs=oa)
        b.rollout_noalloc(n, reward=rb, done=db, obs=ob)
        torch.cuda.synchronize()
        assert torch.equal(da, db), f"done differs on call {call}"
        np.testing.assert_allclose(rb.cpu().numpy(), ra.cpu().numpy(), rtol=STEP_RTOL, atol=1e-6)
        np.testing.assert_allclose(ob.cpu().numpy(), oa.cpu().numpy(), rtol=STEP_RTOL, atol=1e-6)
        sa, sb = a.get_state(), b.get_state()
        for k in ("trem", "tod", "day", "gstep"):
            np.testing.assert_array_equal(sa[k], sb[k], err_msg=f"{k} on call {call}")
        for k in ("soc", "erem", "p"):
            np.testing.assert_allclose(sb[k], sa[k], rtol=STEP_RTOL, atol=1e-6)
        np.testing.assert_array_equal(a.due(), b.due())
        np.testing.assert_allclose(b.battery()["soc"], a.battery()["soc"], rtol=STEP_RTOL, atol=1e-6)


def test_rollout_noalloc_allocates_nothing(cuda_lib):
    """After a first call (which looks up the static array's address), further
    calls with a new step count and new output pointers must leave the device's
    free memory and torch's allocator untouched."""
    import torch
    from paper_2507_01522_b300 import inputs as I
    from paper_2507_01522_b300.chargax import Batch
    b = Batch(I.heterogeneous(n_envs=1000))
    b.set_launch(steps_per_launch=24, warps_per_block=4)
    outs = [(torch.zeros(b.E, n, device="cuda"), torch.zeros(b.E, n, dtype=torch.uint8, device="cuda"),
             torch.zeros(b.obs_size, device="cuda")) for n in (30, 77, 130)]
    b.rollout_noalloc(30, reward=outs[0][0], done=outs[0][1], obs=outs[0][2])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for n, (r, d, o) in zip((77, 130), outs[1:]):
        b.rollout_noalloc(n, reward=r, done=d, obs=o)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    for k in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(k, 0) == stats0.get(k, 0), k


def test_rollout_noalloc_rejects_too_many_launches(cuda_lib):
    import torch
    from paper_2507_01522_b300 import inputs as I
    from paper_2507_01522_b300.chargax import CHX_EINVAL, Batch, ChxError
    w = I.small_uniform()
    b = Batch(w)
    b.set_launch(steps_per_launch=1, warps_per_block=2)
    r = torch.zeros(b.E, 1025, device="cuda")
    with pytest.raises(ChxError) as ei:
        b.rollout_noalloc(1025, reward=r)           # 1025 launches > 1024 counters
    assert ei.value.code == CHX_EINVAL
    assert "at most 1024" in str(ei.value)
    b.rollout_noalloc(1024, reward=r[:, :1024].contiguous())
    torch.cuda.synchronize()
