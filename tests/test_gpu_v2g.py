"""Parity of the vehicle-to-grid mode (signed levels, station battery,
sell-back price, degradation penalty) with the oracle, through the C
interface: events exact, floats within the tolerances of tests/parity.py
(the reward scale adds the battery's and the discharge terms), battery state
within the same relative bounds."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2507_01522_b300 import inputs as I

from parity import (RETURN_RTOL, STEP_RTOL, TRAJ_RTOL, assert_events_equal, assert_floats_close,
                    assert_reward_close, assert_traj_close, charger_pmax, reward_scale, state_drift,
                    to_f32_state, traj_reward_scale, widen)
from test_gpu_parity import odd_sizes, stressed

pytestmark = pytest.mark.gpu

V2G = dict(v2g=1, n_levels=21, sell_grid_ratio=0.8, alpha_degrad=0.02, batt_cap_kwh=150.0, batt_rate_kw=60.0,
           batt_tau=0.7, batt_soc0=0.5, p_max_dis_kw=(9.0, 100.0))


def v2g(w):
    w.params = I.EnvParams(**{**w.params.__dict__, **V2G})
    return w


WORKLOADS = {
    "odd150": lambda: v2g(odd_sizes()),
    "stressed": lambda: v2g(stressed()),
    "hetero64": lambda: v2g(I.heterogeneous(n_envs=64)),
}


def make(name):
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w = WORKLOADS[name]()
    return w, Batch(w), Oracle(w), torch


def v2g_scale(w, info, vi, before=None, d0=None, d1=None, kk=1, b_before=None):
    """Reward scale of the V2G mode: the charge-only terms, the battery's
    energy and the discharge, degradation and feed-in terms of the step;
    with a state before the step and drifts (see tests/parity.py), the
    trajectory allowance for the drift of the FP32 state (chargers and
    battery); without, one step from a shared state."""
    p = w.params
    base = (traj_reward_scale(w, info, before, d0, d1, kk, b_before) if before is not None
            else reward_scale(info, p))
    return (base + np.abs(info["price"]) * (np.abs(vi["e_b"]) + np.abs(vi["e_to"]))
            + p.alpha_degrad * np.abs(vi["degrad"]) + np.abs(p.sell_grid_ratio * info["price"] * vi["e_grid_net"]))


def v2g_drift(gs, os_, gb, ob, n=None):
    return state_drift(gs, os_, n, gb, ob)


def assert_battery_close(bg, bo, w, rtol, where=""):
    np.testing.assert_allclose(bg["soc"], bo["soc"], rtol=0, atol=rtol, err_msg=f"battery SoC {where}")
    np.testing.assert_allclose(bg["p"], bo["p"], rtol=0, atol=rtol * w.params.batt_rate_kw, err_msg=f"battery power {where}")


def compare_traj(w, b, o, torch, steps, mode="plain", k=1, actions=None):
    E = b.E
    reward = torch.zeros(E, k, device="cuda")
    done = torch.zeros(E, k, dtype=torch.uint8, device="cuda")
    n_done = 0
    d0 = v2g_drift(None, None, None, None, w.stations.total_ports)
    for s0 in range(0, steps, k):
        kk = min(k, steps - s0)
        if mode == "plain":
            a = None if actions is None else torch.from_numpy(np.ascontiguousarray(actions[:, s0])).cuda()
            b.step(actions=a, reward=reward.view(-1), done=done.view(-1))
        else:
            a = None if actions is None else torch.from_numpy(np.ascontiguousarray(actions[:, s0:s0 + kk])).cuda()
            b.step_n(kk, actions=a, reward=reward, done=done, lda=kk, ld_out=k)
        torch.cuda.synchronize()
        rg, dg = reward.cpu().numpy(), done.cpu().numpy()
        recs = []
        for j in range(kk):
            before, bb = o.state(), o.battery()
            ro, do = o.step(None if actions is None else actions[:, s0 + j])
            recs.append((ro, o.info(), o.info_v2g(), before, bb))
            np.testing.assert_array_equal(dg[:, j], do, err_msg=f"done step {s0 + j}")
            n_done += int(do.sum())
        gs, os_ = b.get_state(), o.state()
        d1 = v2g_drift(gs, os_, b.battery(), o.battery())
        for j, (ro, info, vi, before, bb) in enumerate(recs):
            assert_reward_close(rg[:, j], ro, v2g_scale(w, info, vi, before, d0, d1, kk, bb), TRAJ_RTOL,
                                where=f"step {s0 + j}")
        d0 = d1
        assert_events_equal(gs, os_, where=f"after step {s0 + kk}")
        assert_traj_close(gs, os_, charger_pmax(w), TRAJ_RTOL, where=f"after step {s0 + kk}")
        assert_battery_close(b.battery(), o.battery(), w, TRAJ_RTOL, where=f"after step {s0 + kk}")
    stg, sto = b.stats(), o.stats()
    np.testing.assert_array_equal(stg["arrived"], sto["arrived"].astype(np.uint32))
    np.testing.assert_array_equal(stg["n_episodes"], sto["n_episodes"])
    fin = sto["n_episodes"] > 0
    if fin.any():
        d = np.abs(stg["last_ret"][fin] - sto["last_ret"][fin])
        assert np.all(d <= RETURN_RTOL * np.maximum(np.abs(sto["last_ret"][fin]), 1.0))
    return n_done


def v2g_actions(rng, b, steps):
    return rng.integers(0, b.workload.params.n_levels, size=(b.n_actions, steps)).astype(np.int8)


@pytest.mark.parametrize("name,steps", [("odd150", 70), ("stressed", 80), ("hetero64", 60)])
def test_v2g_plain_random_actions(cuda_lib, name, steps):
    w, b, o, torch = make(name)
    n_done = compare_traj(w, b, o, torch, steps, mode="plain")
    if name == "stressed":
        assert n_done > 0


@pytest.mark.parametrize("name,steps,k", [("odd150", 72, 24), ("stressed", 74, 37), ("hetero64", 64, 16)])
def test_v2g_fused_random_actions(cuda_lib, name, steps, k):
    w, b, o, torch = make(name)
    compare_traj(w, b, o, torch, steps, mode="fused", k=k)


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_v2g_given_actions_discharge(cuda_lib, mode):
    """Given levels biased to discharge (and the battery cycling both ways),
    so the negative branch, the sell-back price and degradation all occur."""
    w, b, o, torch = make("stressed")
    rng = np.random.default_rng(8)
    steps = 48
    acts = v2g_actions(rng, b, steps)
    acts = np.where(rng.random(acts.shape) < 0.6, acts // 3, acts).astype(np.int8)   # mostly below idle (10)
    compare_traj(w, b, o, torch, steps, mode=mode, k=1 if mode == "plain" else 12, actions=acts)


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_v2g_single_step_from_oracle_state(cuda_lib, mode):
    w, b, o, torch = make("stressed")
    check_single_steps(w, b, o, torch, mode, np.random.default_rng(9), lambda rng: v2g_actions(rng, b, 1)[:, 0])


def check_single_steps(w, b, o, torch, mode, rng, draw, trials=3):
    """From the oracle's state rounded to FP32 (shared by both sides), one
    step with the levels draw(rng): events exact, floats within STEP_RTOL."""
    for _ in range(21):
        o.step(None)
    for trial in range(trials):
        s32 = to_f32_state(o.state())
        bo = o.battery()
        bs, bpw = bo["soc"].astype(np.float32), bo["p"].astype(np.float32)
        o.set_state(widen(s32))
        o.set_battery(bs.astype(np.float64), bpw.astype(np.float64))
        b.set_state(s32)
        b.set_battery(bs, bpw)
        acts = draw(rng)
        reward = torch.zeros(b.E, device="cuda")
        done = torch.zeros(b.E, dtype=torch.uint8, device="cuda")
        a = torch.from_numpy(acts).cuda()
        if mode == "plain":
            b.step(actions=a, reward=reward, done=done)
        else:
            b.step_n(1, actions=a, reward=reward, done=done, lda=1, ld_out=1)
        ro, do = o.step(acts)
        info, vi = o.info(), o.info_v2g()
        gs, os_ = b.get_state(), o.state()
        assert_events_equal(gs, os_, where=f"trial {trial}")
        # SoC after a discharge is SoC - |dE|/C: in FP32 its rounding error is
        # one step of the PREVIOUS SoC, which can be far larger than the result
        # (a car emptied to ~0), so its tolerance floor is the previous value
        prev = s32["soc"].astype(np.float64)
        d = np.abs(gs["soc"].astype(np.float64) - os_["soc"])
        tol = STEP_RTOL * np.maximum(np.maximum(np.abs(os_["soc"]), np.abs(prev)), 1e-3)
        assert np.all(d <= tol), (int(np.argmax(d - tol)), d.max())
        gs2 = dict(gs, soc=os_["soc"].astype(np.float32))
        assert_floats_close(gs2, os_, STEP_RTOL, where=f"trial {trial}", cap_hi=w.params.cap_kwh[1])
        sc = reward_scale(info, w.params) + np.abs(info["price"] * vi["e_grid_net"]) + w.params.alpha_degrad * vi["degrad"]
        assert_reward_close(reward.cpu().numpy(), ro, sc, STEP_RTOL, where=f"trial {trial}")
        np.testing.assert_array_equal(done.cpu().numpy(), do)
        assert_battery_close(b.battery(), o.battery(), w, STEP_RTOL, where=f"trial {trial}")
        for _ in range(5):
            o.step(None)


def test_v2g_observation(cuda_lib):
    w, b, o, torch = make("odd150")
    for _ in range(23):
        o.step(None)
    s32 = to_f32_state(o.state())
    bo = o.battery()
    o.set_state(widen(s32))
    o.set_battery(bo["soc"].astype(np.float32).astype(np.float64), bo["p"].astype(np.float32).astype(np.float64))
    b.set_state(s32)
    b.set_battery(bo["soc"].astype(np.float32), bo["p"].astype(np.float32))
    obs = torch.zeros(b.obs_size, device="cuda")
    assert b.obs_size == 10 * b.E + 6 * b.P
    b.observe(obs)
    np.testing.assert_allclose(obs.cpu().numpy().astype(np.float64), o.observe(), rtol=2e-6, atol=2e-6)
    # the fused kernel writes the same observation after its last step
    obs2 = torch.zeros(b.obs_size, device="cuda")
    b.step_n(9, obs=obs2)
    b.observe(obs)
    assert torch.equal(obs, obs2)


def test_v2g_reduces_to_charge_only_on_gpu(cuda_lib):
    """Non-negative levels and an idle battery: the V2G kernels give the
    charge-only kernels' rewards and state (within rounding)."""
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w0 = stressed()
    w1 = v2g(stressed())
    b0, b1 = Batch(w0), Batch(w1)
    rng = np.random.default_rng(10)
    st = w0.stations
    for mode in ("plain", "fused"):
        for step in range(30):
            lv = rng.integers(0, 11, st.total_ports).astype(np.int8)
            av = np.concatenate([np.append(lv[st.port_off[e]:st.port_off[e + 1]] + 10, 10) for e in range(st.n_envs)])
            r0 = torch.zeros(b0.E, device="cuda")
            r1 = torch.zeros(b1.E, device="cuda")
            a0, a1 = torch.from_numpy(lv).cuda(), torch.from_numpy(av.astype(np.int8)).cuda()
            if mode == "plain":
                b0.step(actions=a0, reward=r0)
                b1.step(actions=a1, reward=r1)
            else:
                b0.step_n(1, actions=a0, reward=r0, lda=1, ld_out=1)
                b1.step_n(1, actions=a1, reward=r1, lda=1, ld_out=1)
            np.testing.assert_allclose(r1.cpu().numpy(), r0.cpu().numpy(), rtol=1e-6, atol=1e-6,
                                       err_msg=f"{mode} step {step}")
        s0, s1 = b0.get_state(), b1.get_state()
        for k in s0:
            np.testing.assert_allclose(s1[k].astype(np.float64), s0[k].astype(np.float64), rtol=1e-6, atol=1e-6,
                                       err_msg=f"{mode} {k}")
    np.testing.assert_array_equal(b1.battery()["soc"], np.full(b1.E, np.float32(0.5)))


def test_v2g_autotune_keeps_battery_state(cuda_lib):
    w, b, o, torch = make("odd150")
    for _ in range(7):
        b.step()
    before, bt = b.get_state(), b.battery()
    b.autotune(40)
    after, bt2 = b.get_state(), b.battery()
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    for k in bt:
        np.testing.assert_array_equal(bt[k], bt2[k])


def test_v2g_checkpoint_resume_bit_exact(cuda_lib):
    w, b, o, torch = make("odd150")
    for _ in range(11):
        b.step()
    blob = b.save()
    r1 = torch.zeros(b.E, 30, device="cuda")
    b.step_n(30, reward=r1)
    s1, bt1 = b.get_state(), b.battery()
    b.load(blob)
    r2 = torch.zeros(b.E, 30, device="cuda")
    b.step_n(30, reward=r2)
    assert torch.equal(r1, r2)
    s2, bt2 = b.get_state(), b.battery()
    for k in s1:
        np.testing.assert_array_equal(s1[k], s2[k])
    for k in bt1:
        np.testing.assert_array_equal(bt1[k], bt2[k])


def test_v2g_fullsize_heterogeneous_sampled(cuda_lib):
    """The 65536-station benchmark batch in V2G mode through the CUDA-graph
    rollout (Philox levels for chargers and batteries), 160 sampled stations
    re-simulated by the oracle, invariants on all."""
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w = v2g(I.heterogeneous(n_envs=65536))
    b = Batch(w)
    n = 150
    b.autotune(n)
    r = torch.zeros(b.E, n, device="cuda")
    d = torch.zeros(b.E, n, dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(1)
    ids = np.sort(rng.choice(w.stations.n_envs, 160, replace=False)).astype(np.int64)
    sub = I.Workload(w.name, w.params, w.stations.subset(ids), w.exo, w.seed)
    o = Oracle(sub, streams=ids)
    po = w.stations.port_off
    sel = np.concatenate([np.arange(po[e], po[e + 1]) for e in ids])
    b.rollout(n, reward=r, done=d)
    torch.cuda.synchronize()
    rg = r.cpu().numpy()[ids]
    recs = []
    for j in range(n):
        before, bb = o.state(), o.battery()
        ro, do = o.step(None)
        recs.append((ro, o.info(), o.info_v2g(), before, bb))
    gs = b.get_state()
    s = {k: (v[sel] if v.shape[0] == b.P else v[ids]) for k, v in gs.items()}
    os_ = o.state()
    d0 = v2g_drift(None, None, None, None, len(sel))
    d1 = v2g_drift(s, os_, {k: v[ids] for k, v in b.battery().items()}, o.battery())
    for j, (ro, info, vi, before, bb) in enumerate(recs):
        assert_reward_close(rg[:, j], ro, v2g_scale(sub, info, vi, before, d0, d1, n, bb), TRAJ_RTOL,
                            where=f"step {j}")
    assert_events_equal(s, os_, "sampled")
    assert_traj_close(s, os_, charger_pmax(sub), TRAJ_RTOL, "sampled")
    bt = b.battery()
    assert_battery_close({k: v[ids] for k, v in bt.items()}, o.battery(), w, TRAJ_RTOL, "sampled")
    assert np.all((gs["soc"] >= 0) & (gs["soc"] <= 1)) and np.all((bt["soc"] >= 0) & (bt["soc"] <= 1))
    pw = gs["p"].astype(np.float64)
    assert np.all(np.abs(np.add.reduceat(pw, po[:-1]) + bt["p"]) <= w.stations.grid_limit_kw * (1 + 1e-5) + 1e-4)
    assert (pw < 0).any() and (bt["p"] < 0).any()             # discharge happened


def test_v2g_rejections(cuda_lib):
    from paper_2507_01522_b300.chargax import CHX_EINVAL, Batch, ChxError, Server
    w = v2g(I.small_uniform())
    w.params.n_levels = 20                                  # must be odd
    with pytest.raises(ChxError) as ei:
        Batch(w)
    assert ei.value.code == CHX_EINVAL
    w.params.n_levels = 21
    b = Batch(w)
    with pytest.raises(ChxError) as ei:
        b.set_battery(soc=np.full(b.E, 1.5, np.float32))
    assert ei.value.code == CHX_EINVAL
    pw = I.policy_weights(8 + 6 * 16, 16, n_levels=21)
    with pytest.raises(ChxError) as ei:                     # the on-device policy is charge-only
        b.policy_load(pw.w1, pw.b1, pw.w2, pw.b2, pw.w3, pw.b3)
    assert ei.value.code == CHX_EINVAL
    with pytest.raises(ChxError) as ei:                     # so is the serving loop
        Server(w.params, w.exo, (16, 16, 16, 16, 16))
    assert ei.value.code == CHX_EINVAL
