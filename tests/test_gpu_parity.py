"""Parity of the CUDA library with the CPU oracle, through the C interface.

Events bit-exact, floats within the tolerances stated in tests/parity.py.
Workloads are small enough for the oracle (seconds) but span several warp
tiles of every size class, ragged station counts and charger counts that are
not powers of two; the full-size workloads are checked on sampled stations.
"""
import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_2507_01522_b300 import inputs as I

from parity import (RETURN_RTOL, STEP_RTOL, TRAJ_RTOL, assert_events_equal, assert_floats_close,
                    assert_reward_close, assert_traj_close, charger_pmax, reward_scale, state_drift,
                    to_f32_state, traj_reward_scale, widen)

pytestmark = pytest.mark.gpu


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def odd_sizes(n_envs=150, seed=7):
    """Stations of 1..128 chargers including every class edge (1, 8, 9, 16,
    17, 32, 33, 64, 65, 128), groups of 4..16, mixed AC/DC."""
    rng = np.random.default_rng(seed)
    edges = [1, 5, 8, 9, 13, 16, 17, 31, 32, 33, 63, 64, 65, 100, 127, 128]
    sizes = np.array([edges[i % len(edges)] for i in range(n_envs)], np.int32)
    rng.shuffle(sizes)
    p = I.EnvParams(p_max_kw=(11.0, 150.0))
    classes = sorted(set(int(s) for s in sizes))
    st = I.mixed_stations(rng, sizes, p.p_max_kw, class_sizes=classes)
    exo = I.Exo(I.price_bank(seed=seed), I.arrival_rates(classes))
    return I.Workload("odd", p, st, exo, seed)


def stressed(n_envs=96, seed=11):
    """Every reward term on: node efficiencies below 1, constraint penalty,
    partial charging targets, fixed cost, distinct AC/DC efficiency, a short
    episode and heavy traffic."""
    w = odd_sizes(n_envs, seed)
    p = w.params
    p.alpha_con = 0.05
    p.alpha_sat = 0.2
    p.alpha_decl = 0.3
    p.c_fixed = 0.01
    p.soc_target = 0.85
    p.eta_port = (0.95, 0.9)
    p.ep_len = 37
    p.stay_steps = (2, 20)
    rng = np.random.default_rng(seed + 1)
    st = w.stations
    st.group_eta[:] = rng.uniform(0.8, 1.0, st.group_eta.shape).astype(np.float32)
    st.grid_eta[:] = rng.uniform(0.85, 1.0, st.grid_eta.shape).astype(np.float32)
    classes = sorted(set(int(s) for s in st.n_ports))
    w.exo = I.Exo(I.price_bank(n_days=9, ep_len=37, seed=seed), I.arrival_rates(classes, ep_len=37, base=1.5))
    return w


WORKLOADS = {
    "uniform16": lambda: I.small_uniform(),
    "fixed203": lambda: I.fixed_station(n_envs=203),
    "hetero64": lambda: I.heterogeneous(n_envs=64),
    "odd150": lambda: odd_sizes(),
    "stressed": lambda: stressed(),
}


def make(name):
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w = WORKLOADS[name]()
    return w, Batch(w), Oracle(w), torch


# ----------------------------------------------------------------------------
# trajectories
# ----------------------------------------------------------------------------

def compare_traj(w, b, o, torch, steps, mode="plain", k=1, actions=None):
    """Run both sides for `steps` steps and compare after every step (plain)
    or every launch (fused)."""
    E = b.E
    params = w.params
    returns_g, returns_o = np.zeros(E), np.zeros(E)
    reward = torch.zeros(E, k, device="cuda")
    done = torch.zeros(E, k, dtype=torch.uint8, device="cuda")
    n_done = 0
    d0 = state_drift(None, None, w.stations.total_ports)
    for s0 in range(0, steps, k):
        kk = min(k, steps - s0)
        if mode == "plain":
            a = None if actions is None else torch.from_numpy(np.ascontiguousarray(actions[:, s0])).cuda()
            b.step(actions=a, reward=reward.view(-1), done=done.view(-1))
        else:
            a = None if actions is None else torch.from_numpy(np.ascontiguousarray(actions[:, s0:s0 + kk])).cuda()
            b.step_n(kk, actions=a, reward=reward, done=done, lda=kk, ld_out=k)
        torch.cuda.synchronize()
        rg = reward.cpu().numpy()
        dg = done.cpu().numpy()
        recs = []
        for j in range(kk):
            before = o.state()
            ro, do = o.step(None if actions is None else actions[:, s0 + j])
            recs.append((ro, o.info(), before))
            np.testing.assert_array_equal(dg[:, j], do, err_msg=f"done step {s0 + j}")
            n_done += int(do.sum())
        gs, os_ = b.get_state(), o.state()
        d1 = state_drift(gs, os_)
        for j, (ro, info, before) in enumerate(recs):
            assert_reward_close(rg[:, j], ro, traj_reward_scale(w, info, before, d0, d1, kk), TRAJ_RTOL,
                                where=f"step {s0 + j}")
        d0 = d1
        assert_events_equal(gs, os_, where=f"after step {s0 + kk}")
        assert_traj_close(gs, os_, charger_pmax(w), TRAJ_RTOL, where=f"after step {s0 + kk}")
        stg, sto = b.stats(), o.stats()
        np.testing.assert_array_equal(stg["arrived"], sto["arrived"].astype(np.uint32))
        np.testing.assert_array_equal(stg["rejected"], sto["rejected"].astype(np.uint32))
        np.testing.assert_array_equal(stg["n_episodes"], sto["n_episodes"])
    stg, sto = b.stats(), o.stats()
    fin = sto["n_episodes"] > 0
    if fin.any():
        d = np.abs(stg["last_ret"][fin] - sto["last_ret"][fin])
        tol = RETURN_RTOL * np.maximum(np.abs(sto["last_ret"][fin]), 1.0)
        assert np.all(d <= tol), (d.max(), tol[np.argmax(d - tol)])
    np.testing.assert_allclose(stg["missing"], sto["missing"], rtol=1e-3, atol=1e-2)
    np.testing.assert_allclose(stg["charged"], sto["charged"], rtol=1e-3, atol=1e-2)
    return n_done


@pytest.mark.parametrize("name,steps", [("uniform16", 300), ("fixed203", 60), ("hetero64", 60),
                                        ("odd150", 80), ("stressed", 90)])
def test_plain_random_actions(cuda_lib, name, steps):
    w, b, o, torch = make(name)
    n_done = compare_traj(w, b, o, torch, steps, mode="plain")
    if name in ("uniform16", "stressed"):
        assert n_done > 0                  # crossed episode ends


@pytest.mark.parametrize("name,steps,k", [("uniform16", 300, 32), ("fixed203", 64, 16), ("hetero64", 64, 7),
                                          ("odd150", 96, 24), ("stressed", 111, 37), ("odd150", 20, 1)])
def test_fused_random_actions(cuda_lib, name, steps, k):
    w, b, o, torch = make(name)
    compare_traj(w, b, o, torch, steps, mode="fused", k=k)


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_given_actions(cuda_lib, mode):
    w, b, o, torch = make("odd150")
    rng = np.random.default_rng(5)
    steps = 48
    acts = I.random_actions(rng, w.stations.total_ports, steps=steps)
    compare_traj(w, b, o, torch, steps, mode=mode, k=1 if mode == "plain" else 16, actions=acts)


# ----------------------------------------------------------------------------
# one step from a shared mid-episode state (1e-5)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["odd150", "stressed", "fixed203"])
@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_single_step_from_oracle_state(cuda_lib, name, mode):
    w, b, o, torch = make(name)
    rng = np.random.default_rng(3)
    for _ in range(29):
        o.step(None)
    for trial in range(3):
        s32 = to_f32_state(o.state())
        o.set_state(widen(s32))
        b.set_state(s32)
        acts = I.random_actions(rng, w.stations.total_ports)
        reward = torch.zeros(b.E, device="cuda")
        done = torch.zeros(b.E, dtype=torch.uint8, device="cuda")
        a = torch.from_numpy(acts).cuda()
        if mode == "plain":
            b.step(actions=a, reward=reward, done=done)
        else:
            b.step_n(1, actions=a, reward=reward, done=done, lda=1, ld_out=1)
        ro, do = o.step(acts)
        info = o.info()
        gs, os_ = b.get_state(), o.state()
        assert_events_equal(gs, os_, where=f"trial {trial}")
        assert_floats_close(gs, os_, STEP_RTOL, where=f"trial {trial}", cap_hi=w.params.cap_kwh[1])
        assert_reward_close(reward.cpu().numpy(), ro, reward_scale(info, w.params), STEP_RTOL, where=f"trial {trial}")
        np.testing.assert_array_equal(done.cpu().numpy(), do)
        for _ in range(7):
            o.step(None)


# ----------------------------------------------------------------------------
# observation, reset, checkpoint, host API, launch paths
# ----------------------------------------------------------------------------

def test_observation(cuda_lib):
    w, b, o, torch = make("odd150")
    for _ in range(41):
        o.step(None)
    s32 = to_f32_state(o.state())
    o.set_state(widen(s32))
    b.set_state(s32)
    obs = torch.zeros(b.obs_size, device="cuda")
    b.observe(obs)
    og = obs.cpu().numpy().astype(np.float64)
    oo = o.observe()
    np.testing.assert_allclose(og, oo, rtol=2e-6, atol=2e-6)


def test_fused_obs_matches_observe(cuda_lib):
    w, b, o, torch = make("odd150")
    obs1 = torch.zeros(b.obs_size, device="cuda")
    obs2 = torch.zeros(b.obs_size, device="cuda")
    b.step_n(13, obs=obs1)
    b.observe(obs2)
    assert torch.equal(obs1, obs2)


def test_reset_subset(cuda_lib):
    w, b, o, torch = make("odd150")
    for _ in range(20):
        b.step()
        o.step(None)
    ids = np.array([0, 3, 17, 64, 149], np.int32)
    b.reset(torch.from_numpy(ids).cuda(), seed=1234)
    o.reset(ids, seed=1234)
    assert_events_equal(b.get_state(), o.state(), "after reset")
    compare_traj(w, b, o, torch, 30, mode="fused", k=10)


def test_checkpoint_resume_bit_exact(cuda_lib):
    w, b, o, torch = make("odd150")
    for _ in range(15):
        b.step()
    blob = b.save()
    r1 = torch.zeros(b.E, 40, device="cuda")
    b.step_n(40, reward=r1)
    s1 = b.get_state()
    b.load(blob)
    r2 = torch.zeros(b.E, 40, device="cuda")
    b.step_n(40, reward=r2)
    s2 = b.get_state()
    assert torch.equal(r1, r2)
    for k in s1:
        np.testing.assert_array_equal(s1[k], s2[k])


def test_rollout_graph_equals_chunks(cuda_lib):
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w = odd_sizes()
    b1, b2 = Batch(w), Batch(w)
    b1.set_launch(steps_per_launch=16, warps_per_block=4)
    n = 50
    r1 = torch.zeros(b1.E, n, device="cuda")
    d1 = torch.zeros(b1.E, n, dtype=torch.uint8, device="cuda")
    b1.rollout(n, reward=r1, done=d1)
    r2 = torch.zeros(b2.E, n, device="cuda")
    for k0 in range(0, n, 16):
        kk = min(16, n - k0)
        tmp = torch.zeros(b2.E, kk, device="cuda")
        b2.step_n(kk, reward=tmp)
        r2[:, k0:k0 + kk] = tmp
    torch.cuda.synchronize()
    assert torch.equal(r1, r2)
    # a second replay of the captured graph continues the trajectory
    b1.rollout(n, reward=r1, done=d1)
    b2.step_n(n, reward=r2)
    torch.cuda.synchronize()
    s1, s2 = b1.get_state(), b2.get_state()
    for k in ("trem", "tod", "gstep"):
        np.testing.assert_array_equal(s1[k], s2[k])


def test_autotune_keeps_state(cuda_lib):
    w, b, o, torch = make("hetero64")
    b.step_n(5)
    before = b.get_state()
    k, wpb = b.autotune(64)
    assert k >= 1 and 1 <= wpb <= 8
    after = b.get_state()
    for key in before:
        np.testing.assert_array_equal(before[key], after[key])


@pytest.mark.parametrize("n,pinned", [(20, False), (7, False), (3, False), (1, False), (20, True), (7, True)])
def test_host_api_matches_device(cuda_lib, n, pinned):
    """The host-call rollout (step-major outputs, launches whose copies
    overlap the next) equals the device rollout, bit for bit, with pageable
    and with pinned host buffers."""
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w = odd_sizes()
    b1, b2 = Batch(w), Batch(w)

    def host(n_items, dtype):
        if not pinned:
            return np.zeros(n_items, dtype)
        t = torch.zeros(n_items, dtype={np.float32: torch.float32, np.uint8: torch.uint8}[dtype], pin_memory=True)
        return t.numpy()

    hr = host(b1.E * n, np.float32)
    hd = host(b1.E * n, np.uint8)
    ho = host(b1.obs_size, np.float32)
    for _ in range(2):                                  # back-to-back calls continue the episode
        b1.rollout_host(n, hr, hd, ho)
        r = torch.zeros(b2.E, n, device="cuda")
        d = torch.zeros(b2.E, n, dtype=torch.uint8, device="cuda")
        ob = torch.zeros(b2.obs_size, device="cuda")
        b2.rollout(n, reward=r, done=d, obs=ob)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(hr.reshape(n, b1.E), r.cpu().numpy().T)
        np.testing.assert_array_equal(hd.reshape(n, b1.E), d.cpu().numpy().T)
        np.testing.assert_array_equal(ho, ob.cpu().numpy())
    if n != 20:
        return
    # plain step with host buffers
    acts = I.random_actions(np.random.default_rng(1), b1.P)
    hr1 = np.zeros(b1.E, np.float32)
    hd1 = np.zeros(b1.E, np.uint8)
    b1.step_host(acts, hr1, hd1, ho)
    r1 = torch.zeros(b2.E, device="cuda")
    b2.step(actions=torch.from_numpy(acts).cuda(), reward=r1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hr1, r1.cpu().numpy())


@pytest.mark.parametrize("n,v2g", [(30, False), (5, False), (1, False), (26, True), (61, False)])
def test_host_actions_rollout(cuda_lib, n, v2g):
    """The host-actions rollout (step-major host levels in, launches whose
    copies in and out overlap their neighbours) equals the device fused form
    given the same levels (charger-major, one launch), bit for bit, on the
    class-edge stations (128-charger class beside the others), and matches the
    oracle step by step; two calls in a row continue the episode."""
    import torch
    from paper_2507_01522_b300.chargax import Batch
    from test_gpu_v2g import v2g_scale
    w = odd_sizes()
    if v2g:
        w = I.v2g_variant(w)
    b1, b2, o = Batch(w), Batch(w), Oracle(w)
    E, P = b1.E, b1.P
    n_act = P + (E if v2g else 0)
    rng = np.random.default_rng(17 + n)
    hr = torch.zeros(n * E, dtype=torch.float32, pin_memory=True).numpy()
    hd = torch.zeros(n * E, dtype=torch.uint8, pin_memory=True).numpy()
    ho = torch.zeros(b1.obs_size, dtype=torch.float32, pin_memory=True).numpy()
    d0 = state_drift(None, None, P)
    for call in range(2):
        acts = rng.integers(0, w.params.n_levels, size=(n, n_act), dtype=np.int8)     # step-major
        ha = torch.from_numpy(acts.reshape(-1)).pin_memory().numpy()
        b1.rollout_host_actions(n, ha, hr, hd, ho)
        r = torch.zeros(E, n, device="cuda")
        d = torch.zeros(E, n, dtype=torch.uint8, device="cuda")
        ob = torch.zeros(b2.obs_size, device="cuda")
        b2.step_n(n, actions=torch.from_numpy(np.ascontiguousarray(acts.T)).cuda(), reward=r, done=d, obs=ob)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(hr.reshape(n, E), r.cpu().numpy().T, err_msg=f"reward, call {call}")
        np.testing.assert_array_equal(hd.reshape(n, E), d.cpu().numpy().T, err_msg=f"done, call {call}")
        np.testing.assert_array_equal(ho, ob.cpu().numpy(), err_msg=f"observation, call {call}")
        recs = []
        for k in range(n):
            before, bb = o.state(), o.battery()
            ro, do = o.step(acts[k])
            recs.append((ro, o.info(), o.info_v2g(), before, bb))
            np.testing.assert_array_equal(hd[k * E:(k + 1) * E], do)
        gs, os_ = b1.get_state(), o.state()
        d1 = state_drift(gs, os_, None, b1.battery(), o.battery())
        for k, (ro, info, vi, before, bb) in enumerate(recs):
            sc = v2g_scale(w, info, vi, before, d0, d1, n, bb) if v2g else traj_reward_scale(w, info, before, d0, d1, n)
            assert_reward_close(hr[k * E:(k + 1) * E], ro, sc, TRAJ_RTOL, where=f"call {call} step {k}")
        d0 = d1
        assert_events_equal(gs, os_, where=f"after call {call}")
        assert_traj_close(gs, os_, charger_pmax(w), TRAJ_RTOL, where=f"after call {call}")
    b1.check()


@pytest.mark.parametrize("n,v2g,n_envs", [(30, False, 150), (7, False, 151), (26, True, 150)])
def test_host_levels4_rollout_equals_int8(cuda_lib, n, v2g, n_envs):
    """Levels packed two per byte (chx_rollout_host_levels4) give bit for bit
    what the int8 host-actions rollout gives on the same levels (itself
    checked against the oracle above), on the class-edge stations, over two
    calls in a row (151 stations: an odd number of action slots, so each
    step's row ends in a half-used byte); a nibble of n_levels or more is
    flagged."""
    import torch
    from paper_2507_01522_b300.chargax import CHX_EFAULT, Batch, ChxError, pack_levels4
    from paper_2507_01522_b300.chargax import CHX_EINVAL
    w = odd_sizes(n_envs=n_envs)
    if v2g:
        w = I.v2g_variant(w)                                # 21 levels: too many for a nibble
        with pytest.raises(ChxError) as ei:
            Batch(w).rollout_host_levels4(1, np.zeros(w.stations.n_ports.sum() + n_envs, np.uint8))
        assert ei.value.code == CHX_EINVAL
        w.params.n_levels = 15
    b1, b2 = Batch(w), Batch(w)
    E, P = b1.E, b1.P
    n_act = P + (E if v2g else 0)
    rng = np.random.default_rng(29 + n)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    out = [[pin(np.zeros(n * E, np.float32)), pin(np.zeros(n * E, np.uint8)), pin(np.zeros(b1.obs_size, np.float32))]
           for _ in range(2)]
    for call in range(2):
        acts = rng.integers(0, w.params.n_levels, size=(n, n_act), dtype=np.int8)
        packed = pack_levels4(acts)
        assert packed.shape == (n, (n_act + 1) // 2)
        b1.rollout_host_actions(n, pin(acts.reshape(-1)), *out[0])
        b2.rollout_host_levels4(n, pin(packed.reshape(-1)), *out[1])
        for x, y, name in zip(out[0], out[1], ("reward", "done", "observation")):
            np.testing.assert_array_equal(x, y, err_msg=f"{name}, call {call}")
        s1, s2 = b1.get_state(), b2.get_state()
        for k in s1:
            np.testing.assert_array_equal(s1[k], s2[k], err_msg=f"state {k}, call {call}")
    b2.check()
    bad = packed.copy()
    bad[0, 0] = 0xF0 | (bad[0, 0] & 0x0F)             # slot 1 of step 0 at level 15
    b2.rollout_host_levels4(n, pin(bad.reshape(-1)), *out[1])
    with pytest.raises(ChxError) as ei:
        b2.check()
    assert ei.value.code == CHX_EFAULT


def test_host_actions_rollout_rejects_null_actions(cuda_lib):
    from paper_2507_01522_b300.chargax import CHX_EINVAL, Batch, ChxError
    b = Batch(I.small_uniform())
    with pytest.raises(ChxError) as ei:
        b.rollout_host_actions(4, None, np.zeros(4 * b.E, np.float32))
    assert ei.value.code == CHX_EINVAL


def test_action_out_of_range_is_flagged(cuda_lib):
    from paper_2507_01522_b300.chargax import CHX_EFAULT, ChxError
    w, b, o, torch = make("fixed203")
    b.step()
    b.step()
    acts = torch.full((b.P,), 11, dtype=torch.int8, device="cuda")
    b.step(actions=acts)
    with pytest.raises(ChxError) as ei:
        b.check()
    assert ei.value.code == CHX_EFAULT
    b.check()                               # flag cleared


def test_invalid_configuration_rejected(cuda_lib):
    from paper_2507_01522_b300.chargax import CHX_EINVAL, Batch, ChxError
    w = I.small_uniform()
    w.stations.group_size[0] = 15           # groups no longer cover the chargers
    with pytest.raises(ChxError) as ei:
        Batch(w)
    assert ei.value.code == CHX_EINVAL


# ----------------------------------------------------------------------------
# full-size workloads, in the launch configuration the benchmark times
# ----------------------------------------------------------------------------

def sampled_oracle(w, ids):
    sub = I.Workload(w.name, w.params, w.stations.subset(ids), w.exo, w.seed)
    return Oracle(sub, streams=ids), sub


def test_fullsize_heterogeneous_sampled(cuda_lib):
    """65536 mixed stations in the benchmark's launch shape (autotuned fused
    kernel, CUDA-graph rollout): two rollouts of 287 steps, so the second one
    crosses an episode end; 192 sampled stations re-simulated by the oracle;
    invariants checked on every station."""
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w = I.heterogeneous(n_envs=65536)
    b = Batch(w)
    T = w.params.ep_len
    b.autotune(T)
    n = T - 1
    r = torch.zeros(b.E, n, device="cuda")
    d = torch.zeros(b.E, n, dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(0)
    ids = np.sort(rng.choice(w.stations.n_envs, 192, replace=False)).astype(np.int64)
    o, ws = sampled_oracle(w, ids)
    po = w.stations.port_off
    sel = np.concatenate([np.arange(po[e], po[e + 1]) for e in ids])
    d0 = state_drift(None, None, len(sel))
    for rep in range(2):
        b.rollout(n, reward=r, done=d)
        torch.cuda.synchronize()
        gs = b.get_state()
        rg, dg = r.cpu().numpy()[ids], d.cpu().numpy()[ids]
        recs = []
        for j in range(n):
            before = o.state()
            ro, do = o.step(None)
            recs.append((ro, o.info(), before))
            np.testing.assert_array_equal(dg[:, j], do)
        sub = {k: (v[sel] if v.shape[0] == b.P else v[ids]) for k, v in gs.items()}
        os_ = o.state()
        d1 = state_drift(sub, os_)
        for j, (ro, inf, before) in enumerate(recs):
            assert_reward_close(rg[:, j], ro, traj_reward_scale(ws, inf, before, d0, d1, n), TRAJ_RTOL,
                                where=f"rep {rep} step {j}")
        d0 = d1
        assert_events_equal(sub, os_, f"sampled rep {rep}")
        assert_traj_close(sub, os_, charger_pmax(ws), TRAJ_RTOL, f"sampled rep {rep}")
        np.testing.assert_allclose(sub["ep_ret"], os_["ep_ret"], rtol=RETURN_RTOL, atol=1e-3)
        # invariants on all stations
        assert np.all((gs["soc"] >= 0) & (gs["soc"] <= 1))
        assert np.all(gs["erem"] >= 0)
        assert np.all(gs["trem"] <= w.params.stay_steps[1])
        occ = np.add.reduceat((gs["trem"] > 0).astype(np.int64), po[:-1])
        assert np.all(occ <= w.stations.n_ports)
        pw = gs["p"].astype(np.float64)
        assert np.all(np.add.reduceat(pw, po[:-1]) <= w.stations.grid_limit_kw * (1 + 1e-5) + 1e-4)
    sg, so = b.stats(), o.stats()
    np.testing.assert_array_equal(sg["n_episodes"][ids], so["n_episodes"])
    np.testing.assert_allclose(sg["last_ret"][ids], so["last_ret"], rtol=RETURN_RTOL, atol=1e-3)
    np.testing.assert_array_equal(sg["arrived"][ids], so["arrived"].astype(np.uint32))
    np.testing.assert_array_equal(sg["rejected"][ids], so["rejected"].astype(np.uint32))


def test_fullsize_fixed_station_plain_sampled(cuda_lib):
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w = I.fixed_station(n_envs=4096)
    b = Batch(w)
    r = torch.zeros(b.E, device="cuda")
    for _ in range(100):
        b.step(reward=r)
    torch.cuda.synchronize()
    ids = np.arange(0, 4096, 37)
    o, ws = sampled_oracle(w, ids)
    for _ in range(99):
        o.step(None)
    before = o.state()
    ro, _ = o.step(None)
    info = o.info()
    gs = b.get_state()
    po = w.stations.port_off
    sel = np.concatenate([np.arange(po[e], po[e + 1]) for e in ids])
    sub = {k: (v[sel] if v.shape[0] == b.P else v[ids]) for k, v in gs.items()}
    assert_events_equal(sub, o.state(), "sampled")
    assert_traj_close(sub, o.state(), charger_pmax(ws), TRAJ_RTOL, "sampled")
    d1 = state_drift(sub, o.state())
    assert_reward_close(r.cpu().numpy()[ids], ro,
                        traj_reward_scale(ws, info, before, state_drift(None, None, len(sel)), d1, 100), TRAJ_RTOL)


def test_fullsize_heterogeneous_plain_sampled(cuda_lib):
    """The benchmark's plain leg: 65536 mixed stations, one launch per step,
    290 steps (past the episode end at 288); 64 stations of each size class
    and the first and last re-simulated by the oracle: every step's reward
    and done flag, the final state, the episode returns and counters."""
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w = I.heterogeneous(n_envs=65536)
    b = Batch(w)
    T = 290
    r = torch.zeros(T, b.E, device="cuda")
    d = torch.zeros(T, b.E, dtype=torch.uint8, device="cuda")
    for k in range(T):
        b.step(reward=r[k], done=d[k])
    torch.cuda.synchronize()
    b.check()
    n = w.stations.n_ports
    rng = np.random.default_rng(5)
    ids = np.unique(np.concatenate([rng.choice(np.flatnonzero(n == c), 64, replace=False) for c in (8, 16, 32, 64)]
                                   + [np.array([0, b.E - 1])]))
    o, ws = sampled_oracle(w, ids)
    rg, dg = r.cpu().numpy()[:, ids], d.cpu().numpy()[:, ids]
    recs = []
    for k in range(T):
        before = o.state()
        ro, do = o.step(None)
        recs.append((ro, o.info(), before))
        np.testing.assert_array_equal(dg[k], do, err_msg=f"done step {k}")
    gs = b.get_state()
    po = w.stations.port_off
    sel = np.concatenate([np.arange(po[e], po[e + 1]) for e in ids])
    sub = {key: (v[sel] if v.shape[0] == b.P else v[ids]) for key, v in gs.items()}
    d0, d1 = state_drift(None, None, len(sel)), state_drift(sub, o.state())
    for k, (ro, info, before) in enumerate(recs):
        assert_reward_close(rg[k], ro, traj_reward_scale(ws, info, before, d0, d1, T), TRAJ_RTOL, where=f"step {k}")
    assert_events_equal(sub, o.state(), "sampled")
    assert_traj_close(sub, o.state(), charger_pmax(ws), TRAJ_RTOL, "sampled")
    stg, sto = b.stats(), o.stats()
    np.testing.assert_array_equal(stg["arrived"][ids], sto["arrived"].astype(np.uint32))
    np.testing.assert_array_equal(stg["rejected"][ids], sto["rejected"].astype(np.uint32))
    np.testing.assert_array_equal(stg["n_episodes"][ids], sto["n_episodes"])
    assert np.all(sto["n_episodes"] == 1)
    dret = np.abs(stg["last_ret"][ids] - sto["last_ret"])
    assert np.all(dret <= RETURN_RTOL * np.maximum(np.abs(sto["last_ret"]), 1.0)), dret.max()


def test_reset_list_out_of_range_and_empty(cuda_lib):
    """chx_reset with a list: ids outside 0..n_envs-1 are skipped (nothing
    outside the batch is written), the valid ones are reset exactly as the
    oracle resets them, and the next chx_check reports CHX_EFAULT once; an
    empty list changes nothing."""
    from paper_2507_01522_b300.chargax import CHX_EFAULT, ChxError
    w, b, o, torch = make("odd150")
    for _ in range(20):
        b.step()
        o.step(None)
    before = b.get_state()
    b.reset(torch.zeros(0, dtype=torch.int32, device="cuda"), seed=5)
    b.check()
    after = b.get_state()
    for key in before:
        np.testing.assert_array_equal(after[key], before[key], err_msg=key)
    ids = np.array([3, b.E, -1, 1 << 30, 17, -(1 << 31)], np.int32)
    b.reset(torch.from_numpy(ids).cuda(), seed=99)
    with pytest.raises(ChxError) as ei:
        b.check()
    assert ei.value.code == CHX_EFAULT and "env id" in str(ei.value)
    b.check()                               # flag cleared
    o.reset(np.array([3, 17]), seed=99)
    assert_events_equal(b.get_state(), o.state(), "after reset")
    compare_traj(w, b, o, torch, 20, mode="fused", k=10)


def one_station(n_ports, group_sizes, group_limit=50.0, grid_limit=100.0):
    st = I.Stations(
        n_ports=np.array([n_ports], np.int32), port_type=np.zeros(max(n_ports, 0), np.uint8),
        n_groups=np.array([len(group_sizes)], np.int32), group_size=np.array(group_sizes, np.int32),
        group_limit_kw=np.full(len(group_sizes), group_limit, np.float32),
        group_eta=np.ones(len(group_sizes), np.float32), grid_limit_kw=np.array([grid_limit], np.float32),
        grid_eta=np.ones(1, np.float32), arrival_class=np.zeros(1, np.int32))
    base = I.small_uniform()
    return I.Workload("degenerate", base.params, st, base.exo, 0)


@pytest.mark.parametrize("case,reason", [
    ("no stations", "n_envs out of range"),
    ("129 chargers", "n_ports out of 1..128"),
    ("0 chargers", "n_ports out of 1..128"),
    ("empty group", "empty group"),
    ("groups short", "do not cover"),
    ("group limit 0", "group limit must be > 0"),
    ("grid limit 0", "grid limit must be > 0"),
    ("33 groups", "n_groups out of"),
])
def test_degenerate_configurations_rejected(cuda_lib, case, reason):
    """Configurations outside the documented ranges fail with CHX_EINVAL
    and the reason, before anything is allocated."""
    from paper_2507_01522_b300.chargax import CHX_EINVAL, Batch, ChxError
    if case == "no stations":
        base = I.small_uniform()
        w = I.Workload(base.name, base.params, base.stations.subset(np.array([], np.int64)), base.exo, 0)
    else:
        w = {"129 chargers": lambda: one_station(129, [64, 65]),
             "0 chargers": lambda: one_station(0, [1]),
             "empty group": lambda: one_station(8, [8, 0]),
             "groups short": lambda: one_station(8, [4, 3]),
             "group limit 0": lambda: one_station(8, [8], group_limit=0.0),
             "grid limit 0": lambda: one_station(8, [8], grid_limit=0.0),
             "33 groups": lambda: one_station(66, [2] * 33)}[case]()
    with pytest.raises(ChxError) as ei:
        Batch(w)
    assert ei.value.code == CHX_EINVAL and reason in str(ei.value), str(ei.value)


def test_degenerate_launch_arguments_rejected(cuda_lib):
    """Zero steps, a launch shape outside 1..8 warps, and a negative reset
    count fail with CHX_EINVAL and leave the state as it was; the smallest
    valid station (one charger, one group) steps like the oracle."""
    from paper_2507_01522_b300.chargax import CHX_EINVAL, ChxError
    w, b, o, torch = make("odd150")
    b.step()
    o.step(None)
    before = b.get_state()
    r = torch.zeros(b.E, device="cuda")
    for call in (lambda: b.step_n(0, reward=r), lambda: b.rollout(0, reward=r),
                 lambda: b.set_launch(0, 9)):
        with pytest.raises(ChxError) as ei:
            call()
        assert ei.value.code == CHX_EINVAL
    from paper_2507_01522_b300 import chargax
    assert chargax.load_library().chx_reset(b.h, None, -1, 0, None) == CHX_EINVAL
    after = b.get_state()
    for key in before:
        np.testing.assert_array_equal(after[key], before[key], err_msg=key)
    w1 = one_station(1, [1], group_limit=5.0, grid_limit=7.0)
    from paper_2507_01522_b300.chargax import Batch
    b1, o1 = Batch(w1), Oracle(w1)
    compare_traj(w1, b1, o1, torch, 300, mode="fused", k=100)
