"""Parity of the on-device policy (3-layer BF16 MLP on the tensor cores with
the sampling fused into its last epilogue) and of the policy rollout.

* Logits: the kernel's against ``oracle.policy.mlp_forward`` of the same FP32
  observations, within ``oracle.policy.mlp_bound`` (first-order worst case
  of FP32 accumulation order and BF16 rounding flips); the typical error
  must also be far below the bound.
* Levels: against the oracle's inverse transform of the KERNEL's logits
  with the oracle's uniforms (same Philox counters): equal wherever the
  sampled uniform is more than MARGIN from a cumulative-probability
  boundary (FP32 rounding of the kernel's softmax), at most one level off
  elsewhere.  Without the kernel's logits (full-size run), the oracle's own
  logits are used and the margin widens by twice the logit bound.
* Rollout: the oracle env replays the kernel's actions: events exact,
  floats within TRAJ_RTOL, observations within OBS_ATOL.
"""
import numpy as np
import pytest

from oracle import Oracle
from oracle import policy as OP
from paper_2507_01522_b300 import inputs as I

from parity import (TRAJ_RTOL, assert_events_equal, assert_reward_close, assert_traj_close, charger_pmax,
                    state_drift, traj_reward_scale)

pytestmark = pytest.mark.gpu

MARGIN = 1e-5
OBS_ATOL = 2e-4


def uniform_workload(n_envs, n_ports, seed=0):
    groups = [8] * (n_ports // 8) + ([n_ports % 8] if n_ports % 8 else [])
    p = I.EnvParams(p_max_kw=(22.0, 150.0))
    st = I.uniform_stations(n_envs, n_ports, groups, 80.0, 9.0 * n_ports)
    exo = I.Exo(I.price_bank(seed=seed), I.arrival_rates([n_ports]))
    return I.Workload(f"uniform-{n_envs}x{n_ports}", p, st, exo, seed)


def batch_with_policy(w, **kw):
    from paper_2507_01522_b300.chargax import Batch
    b = Batch(w)
    N = int(w.stations.n_ports[0])
    pw = I.policy_weights(8 + 6 * N, N, n_levels=w.params.n_levels, **kw)
    b.policy_load(pw.w1, pw.b1, pw.w2, pw.b2, pw.w3, pw.b3)
    return b, pw, N


def check_logits(lg_kernel, obs, pw, where=""):
    ref, _, _ = OP.mlp_forward(obs, pw)
    bound = OP.mlp_bound(obs, pw)
    d = np.abs(lg_kernel.astype(np.float64) - ref)
    bad = d > bound + 1e-6
    assert not bad.any(), (f"logits {where}: {bad.sum()} outside the bound, worst "
                           f"{d[bad].max():.3g} vs {bound[bad][np.argmax(d[bad])]:.3g}")
    assert np.median(d) <= 0.05 * np.median(bound) + 1e-7, (where, np.median(d), np.median(bound))
    return ref, bound


def check_levels(levels, logits, u, n_levels, margin_tol=MARGIN, where=""):
    lv, margin = OP.sample(logits, u, n_levels)
    lv_k = levels.astype(np.int64)
    sure = margin > margin_tol
    mism = sure & (lv_k != lv)
    assert not mism.any(), f"levels {where}: {mism.sum()} mismatches away from boundaries"
    assert np.all(np.abs(lv_k - lv) <= 1), f"levels {where}: more than one level off"
    assert np.all((lv_k >= 0) & (lv_k < n_levels))
    return sure.mean()


@pytest.mark.parametrize("N", [32, 16, 5])
def test_policy_act_matches_oracle(cuda_lib, N):
    """Ragged tiles (300 envs = 128 + 128 + 44), charger counts whose
    logit and observation widths are not whole tiles."""
    import torch
    w = uniform_workload(300, N, seed=N)
    b, pw, _ = batch_with_policy(w, seed=N, head_gain=1.0, bias_scale=0.5)
    o = Oracle(w)
    rng = np.random.default_rng(N)
    D, L = 8 + 6 * N, w.params.n_levels
    obs = rng.uniform(-1.0, 3.0, (b.E, D)).astype(np.float32)
    obs[:, :8] = np.float32([0.3, -0.9, 0.12, 0.75, 0.5, 0.1, 0.2, 1.0])
    before = b.get_state()
    acts = torch.zeros(b.E, N, dtype=torch.int8, device="cuda")
    logits = torch.zeros(b.E, N * L, device="cuda")
    b.policy_act(torch.from_numpy(obs).cuda(), acts, logits)
    b.check()
    lg = logits.cpu().numpy()
    check_logits(lg, obs, pw, where=f"N={N}")
    frac = check_levels(acts.cpu().numpy(), lg, o.policy_uniforms(N), L, where=f"N={N}")
    assert frac > 0.99
    after = b.get_state()
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    # deterministic: a second call gives the same bits
    acts2 = torch.zeros_like(acts)
    logits2 = torch.zeros_like(logits)
    b.policy_act(torch.from_numpy(obs).cuda(), acts2, logits2)
    assert torch.equal(acts, acts2) and torch.equal(logits, logits2)


def test_policy_act_without_logits_and_ppo_init(cuda_lib):
    """The rollout's configuration: PPO initialisation (near-uniform
    policy), no logits output, observations of the environment itself."""
    import torch
    w = uniform_workload(260, 32, seed=3)
    b, pw, N = batch_with_policy(w, seed=3)
    o = Oracle(w)
    b.step_n(20)
    for _ in range(20):
        o.step()
    obs_t = torch.zeros(b.obs_size, device="cuda")
    b.observe(obs_t)
    obs = obs_t.cpu().numpy().reshape(b.E, -1)
    acts = torch.zeros(b.E, N, dtype=torch.int8, device="cuda")
    b.policy_act(obs_t, acts)
    b.check()
    ref, _, _ = OP.mlp_forward(obs, pw)
    bound = OP.mlp_bound(obs, pw)
    np.testing.assert_array_equal(b.get_state()["gstep"], o.state()["gstep"])
    check_levels(acts.cpu().numpy(), ref, o.policy_uniforms(N), w.params.n_levels,
                 margin_tol=MARGIN + 2 * bound.max(), where="ppo init")


def run_policy_rollout(w, b, pw, N, T, with_logits=True, form=0):
    import torch
    E, D, L = b.E, 8 + 6 * N, w.params.n_levels
    obs = torch.zeros(T, E, D, device="cuda")
    acts = torch.zeros(T, E, N, dtype=torch.int8, device="cuda")
    rew = torch.zeros(T, E, device="cuda")
    done = torch.zeros(T, E, dtype=torch.uint8, device="cuda")
    logits = torch.zeros(T, E, N * L, device="cuda") if with_logits else None
    b.policy_rollout(T, obs, acts, rew, done, logits, form=form)
    b.check()
    return obs, acts, rew, done, logits


def replay_in_oracle(w, b, o, pw, N, T, obs, acts, rew, done, logits, where=""):
    """Step the oracle with the kernel's actions and compare everything the
    rollout wrote; returns the number of episode ends.  The state drift at
    the start is measured on both sides (the second of back-to-back calls
    starts from where the first left the two)."""
    L = w.params.n_levels
    n_done = 0
    d0 = state_drift(b.get_state(), o.state())
    recs = []
    for t in range(T):
        oo = o.observe().reshape(b.E, -1)
        np.testing.assert_allclose(obs[t], oo, rtol=0, atol=OBS_ATOL, err_msg=f"obs step {t} {where}")
        check_logits(logits[t], obs[t], pw, where=f"step {t} {where}")
        check_levels(acts[t], logits[t], o.policy_uniforms(N), L, where=f"step {t} {where}")
        before = o.state()
        ro, do = o.step(acts[t].reshape(-1))
        recs.append((ro, o.info(), before))
        np.testing.assert_array_equal(done[t], do, err_msg=f"done step {t} {where}")
        n_done += int(do.sum())
    gs, os_ = b.get_state(), o.state()
    d1 = state_drift(gs, os_)
    for t, (ro, info, before) in enumerate(recs):
        assert_reward_close(rew[t], ro, traj_reward_scale(w, info, before, d0, d1, T), TRAJ_RTOL,
                            where=f"step {t} {where}")
    assert_events_equal(gs, os_, where=f"after rollout {where}")
    assert_traj_close(gs, os_, charger_pmax(w), TRAJ_RTOL, where=f"after rollout {where}")
    stg, sto = b.stats(), o.stats()
    np.testing.assert_array_equal(stg["arrived"], sto["arrived"].astype(np.uint32))
    np.testing.assert_array_equal(stg["rejected"], sto["rejected"].astype(np.uint32))
    np.testing.assert_array_equal(stg["n_episodes"], sto["n_episodes"])
    return n_done


def stressed_uniform(n_envs, n_ports, seed):
    """Uniform charger count, but per-station random group layouts (4..9
    chargers), 30 % DC ports, efficiencies below 1, tight group and grid
    limits, every reward term on, a 16-step episode and heavy traffic."""
    rng = np.random.default_rng(seed)
    p = I.EnvParams(p_max_kw=(22.0, 150.0))
    p.alpha_con, p.alpha_sat, p.alpha_decl, p.c_fixed = 0.05, 0.2, 0.3, 0.01
    p.soc_target, p.eta_port, p.ep_len, p.stay_steps = 0.85, (0.95, 0.9), 16, (2, 20)
    st = I.mixed_stations(rng, np.full(n_envs, n_ports), p.p_max_kw, p_dc=0.3, grid_kw_per_port=6.0,
                          group_frac=0.35, class_sizes=[n_ports], group_lo=4, group_hi=9)
    st.group_eta[:] = rng.uniform(0.8, 1.0, st.group_eta.shape).astype(np.float32)
    st.grid_eta[:] = rng.uniform(0.85, 1.0, st.grid_eta.shape).astype(np.float32)
    exo = I.Exo(I.price_bank(n_days=9, ep_len=16, seed=seed), I.arrival_rates([n_ports], ep_len=16, base=2.5))
    return I.Workload(f"stressed-{n_envs}x{n_ports}", p, st, exo, seed)


@pytest.mark.parametrize("form", [0, 1], ids=["fused", "split"])
def test_policy_rollout_matches_oracle(cuda_lib, form):
    w = uniform_workload(200, 32, seed=9)
    w.params.ep_len = 16                                   # cross an episode end
    w.exo = I.Exo(I.price_bank(n_days=5, ep_len=16, seed=9), I.arrival_rates([32], ep_len=16, base=2.0))
    b, pw, N = batch_with_policy(w, seed=9, head_gain=1.0, bias_scale=0.5)
    o = Oracle(w)
    T, L = 24, w.params.n_levels
    out = [x.cpu().numpy() for x in run_policy_rollout(w, b, pw, N, T, form=form)]
    n_done = replay_in_oracle(w, b, o, pw, N, T, *out)
    assert n_done == b.E                                   # every env ended its 16-step episode once
    assert len(np.unique(out[1])) == L                     # a spread of levels was sampled


@pytest.mark.parametrize("N,E", [(20, 300), (8, 130), (32, 129), (13, 70)])
def test_fused_rollout_stressed(cuda_lib, N, E):
    """Padding charger slots (N = 20 in the 32 class), a small class (N = 8),
    ragged tiles, per-station group layouts, every reward term; two
    rollouts back to back (the second starts from the first one's state).
    N = 13 (a row length of 86 floats) takes the kernel's other observation
    path: rows written from the observation pass in 8-byte pairs, the
    operand rebuilt from the state, instead of 32-byte sectors and parked
    operand rows from the environment step."""
    w = stressed_uniform(E, N, seed=N)
    b, pw, _ = batch_with_policy(w, seed=N, head_gain=1.0, bias_scale=0.5)
    o = Oracle(w)
    for rep in range(2):
        T = 21 if rep == 0 else 13
        out = [x.cpu().numpy() for x in run_policy_rollout(w, b, pw, N, T, form=0)]
        n_done = replay_in_oracle(w, b, o, pw, N, T, *out, where=f"rollout {rep}")
        assert n_done > 0


@pytest.mark.parametrize("form", [0, 1], ids=["fused", "split"])
def test_policy_rollout_replay_is_deterministic(cuda_lib, form):
    """Same start state -> bit-identical rollout buffers (the split form
    replays its captured graph on the second call); loading new weights with
    the same shape keeps a captured graph valid and changes the actions."""
    import torch
    w = uniform_workload(150, 32, seed=4)
    b, pw, N = batch_with_policy(w, seed=4, head_gain=1.0, bias_scale=0.5)
    blob = b.save()
    T = 12
    first = [x.clone() for x in run_policy_rollout(w, b, pw, N, T, with_logits=False, form=form)[:4]]
    end_state = b.get_state()
    E, D = b.E, 8 + 6 * N
    bufs = (torch.zeros(T, E, D, device="cuda"), torch.zeros(T, E, N, dtype=torch.int8, device="cuda"),
            torch.zeros(T, E, device="cuda"), torch.zeros(T, E, dtype=torch.uint8, device="cuda"))
    for _ in range(2):
        b.load(blob)
        b.policy_rollout(T, *bufs, form=form)
        b.check()
        for x, y in zip(first, bufs):
            assert torch.equal(x, y)
        again = b.get_state()
        for k in end_state:
            np.testing.assert_array_equal(end_state[k], again[k])
    pw2 = I.policy_weights(D, N, seed=5, head_gain=1.0, bias_scale=0.5)
    b.policy_load(pw2.w1, pw2.b1, pw2.w2, pw2.b2, pw2.w3, pw2.b3)
    b.load(blob)
    b.policy_rollout(T, *bufs, form=form)
    b.check()
    assert not torch.equal(first[1], bufs[1])


def test_fused_and_split_rollouts_agree(cuda_lib):
    """Same start state: identical events while the levels agree; the
    sampled levels differ only where the two FP32 computations straddle a
    sampling boundary (rare), so compare the first steps before divergence."""
    import torch
    w = uniform_workload(256, 32, seed=12)
    b, pw, N = batch_with_policy(w, seed=12, head_gain=1.0, bias_scale=0.5)
    blob = b.save()
    T = 8
    fa = [x.cpu().numpy() for x in run_policy_rollout(w, b, pw, N, T, form=0)]
    b.load(blob)
    sa = [x.cpu().numpy() for x in run_policy_rollout(w, b, pw, N, T, form=1)]
    same_env = np.all(fa[1].reshape(T, b.E, -1) == sa[1].reshape(T, b.E, -1), axis=(0, 2))
    assert same_env.mean() > 0.9
    for t in range(T):
        np.testing.assert_allclose(fa[0][t][same_env], sa[0][t][same_env], rtol=0, atol=OBS_ATOL)
        np.testing.assert_array_equal(fa[3][t][same_env], sa[3][t][same_env])


def test_policy_rejects_unsupported_batches(cuda_lib):
    from paper_2507_01522_b300.chargax import CHX_EINVAL, Batch, ChxError
    w = I.heterogeneous(n_envs=64)                          # mixed charger counts
    b = Batch(w)
    pw = I.policy_weights(8 + 6 * 8, 8)
    with pytest.raises(ChxError) as ei:
        b.policy_load(pw.w1, pw.b1, pw.w2, pw.b2, pw.w3, pw.b3)
    assert ei.value.code == CHX_EINVAL
    w = uniform_workload(10, 33)                            # more than 32 chargers
    b = Batch(w)
    pw = I.policy_weights(8 + 6 * 33, 33)
    with pytest.raises(ChxError) as ei:
        b.policy_load(pw.w1, pw.b1, pw.w2, pw.b2, pw.w3, pw.b3)
    assert ei.value.code == CHX_EINVAL
    import torch
    with pytest.raises(ChxError) as ei:                     # no policy loaded
        b.policy_act(torch.zeros(10, 206, device="cuda"), torch.zeros(10, 33, dtype=torch.int8, device="cuda"))
    assert ei.value.code == CHX_EINVAL
    w = uniform_workload(10, 32)                            # 32 x 12 logits: split form only
    w.params.n_levels = 12
    b, pw, N = batch_with_policy(w)
    acts = torch.zeros(2, 10, 32, dtype=torch.int8, device="cuda")
    obs = torch.zeros(2, 10, 200, device="cuda")
    with pytest.raises(ChxError) as ei:
        b.policy_rollout(2, obs, acts, form=0)
    assert ei.value.code == CHX_EINVAL
    b.policy_rollout(2, obs, acts, form=1)
    b.check()
    assert int(acts.max()) <= 11
    # buffers off a 16-byte boundary are refused before any launch
    w = uniform_workload(10, 32)
    b, pw, N = batch_with_policy(w)
    big = torch.zeros(2 * 10 * 200 + 1, device="cuda")
    skewed = big[1:].view(2, 10, 200)                       # 4 bytes past the allocation's start
    for form in (0, 1):
        with pytest.raises(ChxError) as ei:
            b.policy_rollout(2, skewed, acts, form=form)
        assert ei.value.code == CHX_EINVAL
    with pytest.raises(ChxError) as ei:
        b.policy_act(skewed[0], acts[0])
    assert ei.value.code == CHX_EINVAL


def test_policy_rollout_fullsize_sampled(cuda_lib):
    """16384 stations x 32 chargers, 128-step buffer, PPO initialisation,
    no logits output (the benchmark's launch configuration).  Rewards and
    done flags of every env at every step against the oracle replay;
    observations, and levels against the oracle's own logits, on sampled
    envs and steps."""
    w = I.rollout_stations()
    b, pw, N = batch_with_policy(w, seed=0)
    o = Oracle(w)
    T, L = 128, w.params.n_levels
    obs, acts, rew, done, _ = run_policy_rollout(w, b, pw, N, T, with_logits=False, form=0)
    obs, acts, rew, done = (x.cpu().numpy() for x in (obs, acts, rew, done))
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(b.E, 256, replace=False))
    recs = []
    for t in range(T):
        if t % 16 == 0 or t == T - 1:
            oo = o.observe().reshape(b.E, -1)
            np.testing.assert_allclose(obs[t][sample], oo[sample], rtol=0, atol=OBS_ATOL, err_msg=f"obs step {t}")
            ref, _, _ = OP.mlp_forward(obs[t][sample], pw)
            bound = OP.mlp_bound(obs[t][sample], pw)
            u = o.policy_uniforms(N)[sample]
            check_levels(acts[t][sample], ref, u, L, margin_tol=MARGIN + 2 * bound.max(), where=f"step {t}")
        before = o.state()
        ro, do = o.step(acts[t].reshape(-1))
        recs.append((ro, o.info(), before))
        np.testing.assert_array_equal(done[t], do, err_msg=f"done step {t}")
    gs, os_ = b.get_state(), o.state()
    d0, d1 = state_drift(None, None, b.P), state_drift(gs, os_)
    for t, (ro, info, before) in enumerate(recs):
        assert_reward_close(rew[t], ro, traj_reward_scale(w, info, before, d0, d1, T), TRAJ_RTOL, where=f"step {t}")
    assert_events_equal(gs, os_, where="after rollout")
    assert_traj_close(gs, os_, charger_pmax(w), TRAJ_RTOL, where="after rollout")


def test_bounded_wait_gives_up_and_context_survives(cuda_lib):
    """The tensor-core kernels' bounded wait, run on a barrier nothing
    releases: it gives up after its limit (2^31 cycles), raises the fault
    flag (chx_check: CHX_ETIMEOUT, once) and the context keeps working (a
    policy rollout afterwards equals one on a fresh batch)."""
    import torch
    from paper_2507_01522_b300.chargax import CHX_ETIMEOUT, Batch, ChxError
    w = uniform_workload(200, 16)
    b, ref = Batch(w), Batch(w)
    gave_up, mcycles = b.selftest_wait()
    assert gave_up and 2048 <= mcycles < 4096
    with pytest.raises(ChxError) as ei:
        b.check()
    assert ei.value.code == CHX_ETIMEOUT
    b.check()
    N = int(w.stations.n_ports[0])
    D, L = 8 + 6 * N, w.params.n_levels
    pw = I.policy_weights(D, N, n_levels=L, seed=3)
    outs = []
    for bb in (b, ref):
        bb.policy_load(pw.w1, pw.b1, pw.w2, pw.b2, pw.w3, pw.b3)
        obs = torch.zeros(4, bb.E, D, device="cuda")
        acts = torch.zeros(4, bb.E, N, dtype=torch.int8, device="cuda")
        rew = torch.zeros(4, bb.E, device="cuda")
        bb.policy_rollout(4, obs, acts, rew)
        torch.cuda.synchronize()
        bb.check()
        outs.append((obs.cpu().numpy(), acts.cpu().numpy(), rew.cpu().numpy()))
    for x, y in zip(*outs):
        np.testing.assert_array_equal(x, y)
