"""Parity of deeper architecture trees (Fig. charge-tree c: nodes above the
groups, Eq. ArchConst at every node, proportional rescale deepest first)
with the oracle, through the C interface: plain and fused kernels, charge-
only and V2G, with charge-sensitive users and the Delta form, every penalty
on; events exact, floats within the tolerances of tests/parity.py."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2507_01522_b300 import inputs as I

from parity import STEP_RTOL, assert_events_equal, assert_floats_close, assert_reward_close, reward_scale, to_f32_state, widen
from test_gpu_parity import compare_traj
from test_gpu_v2g import V2G, compare_traj as compare_traj_v2g
from test_gpu_cs import CS, compare_cs

pytestmark = pytest.mark.gpu


def make(n_envs=96, seed=4, **extra):
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w = I.tree_workload(n_envs, seed=seed)
    kw = dict(alpha_con=0.05, alpha_sat=0.1, alpha_decl=0.2, c_fixed=0.01)
    kw.update(extra)
    w.params = I.EnvParams(**{**w.params.__dict__, **kw})
    return w, Batch(w), Oracle(w), torch


@pytest.mark.parametrize("mode,k", [("plain", 1), ("fused", 24)])
def test_tree_random_levels(cuda_lib, mode, k):
    w, b, o, torch = make()
    compare_traj(w, b, o, torch, 96, mode=mode, k=k)


@pytest.mark.parametrize("mode,k", [("plain", 1), ("fused", 16)])
def test_tree_given_levels(cuda_lib, mode, k):
    w, b, o, torch = make(n_envs=64, seed=9)
    rng = np.random.default_rng(1)
    acts = rng.integers(0, 11, size=(b.P, 64)).astype(np.int8)
    compare_traj(w, b, o, torch, 64, mode=mode, k=k, actions=acts)


@pytest.mark.parametrize("mode,k", [("plain", 1), ("fused", 24)])
def test_tree_v2g(cuda_lib, mode, k):
    w, b, o, torch = make(**V2G)
    compare_traj_v2g(w, b, o, torch, 72, mode=mode, k=k)


@pytest.mark.parametrize("mode,k", [("plain", 1), ("fused", 32)])
def test_tree_with_charge_sensitive_users_and_delta(cuda_lib, mode, k):
    w, b, o, torch = make(**CS, action_delta=1, n_levels=21)
    compare_cs(w, b, o, torch, 96, mode=mode, k=k)


def test_tree_fused_two_episodes(cuda_lib):
    w, b, o, torch = make(n_envs=384, seed=12)
    compare_traj(w, b, o, torch, 2 * 288, mode="fused", k=96)


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_tree_single_step_from_oracle_state(cuda_lib, mode):
    w, b, o, torch = make()
    rng = np.random.default_rng(6)
    for _ in range(25):
        o.step(None)
    for trial in range(3):
        s32 = to_f32_state(o.state())
        o.set_state(widen(s32))
        b.set_state(s32)
        acts = rng.integers(0, 11, b.P).astype(np.int8)
        reward = torch.zeros(b.E, device="cuda")
        a = torch.from_numpy(acts).cuda()
        if mode == "plain":
            b.step(actions=a, reward=reward)
        else:
            b.step_n(1, actions=a, reward=reward, lda=1, ld_out=1)
        ro, _ = o.step(acts)
        gs, os_ = b.get_state(), o.state()
        assert_events_equal(gs, os_, where=f"trial {trial}")
        assert_floats_close(gs, os_, STEP_RTOL, where=f"trial {trial}", cap_hi=w.params.cap_kwh[1])
        assert_reward_close(reward.cpu().numpy(), ro, reward_scale(o.info(), w.params), STEP_RTOL, where=f"trial {trial}")
        for _ in range(5):
            o.step(None)


def test_tree_rejections(cuda_lib):
    from paper_2507_01522_b300.chargax import CHX_EINVAL, Batch, ChxError
    w = I.tree_workload(4, seed=1)
    st = w.stations
    bad = [
        dict(upper_parent=np.where(np.arange(len(st.upper_parent)) == 0, 0, st.upper_parent)),   # a cycle
        dict(group_parent=np.full_like(st.group_parent, 99)),                                      # out of range
        dict(upper_limit_kw=np.zeros_like(st.upper_limit_kw)),                                     # limit 0
    ]
    for change in bad:
        w2 = I.Workload(w.name, w.params, I.Stations(**{**st.__dict__, **change}), w.exo, 0)
        with pytest.raises(ChxError) as ei:
            Batch(w2)
        assert ei.value.code == CHX_EINVAL
    # groups of one node that are not consecutive
    from test_oracle_tree_pins import tree_station
    w3 = tree_station([2, 2, 2], [50.0] * 3, [0, -1, 0], [-1], [60.0])
    with pytest.raises(ChxError) as ei:
        Batch(w3)
    assert ei.value.code == CHX_EINVAL
    # four levels above the groups
    w4 = tree_station([2], [50.0], [3], [-1, 0, 1, 2], [60.0] * 4)
    with pytest.raises(ChxError) as ei:
        Batch(w4)
    assert ei.value.code == CHX_EINVAL
    b = Batch(w)
    pw = I.policy_weights(8 + 6 * 63, 63)
    with pytest.raises(ChxError):
        b.policy_load(pw.w1, pw.b1, pw.w2, pw.b2, pw.w3, pw.b3)


def test_tree_fullsize_sampled(cuda_lib):
    """The benchmark's Fig. c leg: 65536 tree stations through the rollout in
    the benchmark's launch shape (one 288-step launch, 8 warps per block);
    160 sampled stations re-simulated by the oracle, every node's constraint
    checked on all stations."""
    import torch
    from paper_2507_01522_b300.chargax import Batch
    from parity import TRAJ_RTOL, assert_traj_close, charger_pmax, state_drift, traj_reward_scale
    w = I.tree_workload(65536, seed=0)
    b = Batch(w)
    b.set_launch(288, 8)
    n = 287                                             # one launch; the state is mid-episode at the end
    r = torch.zeros(b.E, n, device="cuda")
    rng = np.random.default_rng(3)
    ids = np.sort(rng.choice(w.stations.n_envs, 160, replace=False)).astype(np.int64)
    sub = I.Workload(w.name, w.params, w.stations.subset(ids), w.exo, w.seed)
    o = Oracle(sub, streams=ids)
    b.rollout(n, reward=r)
    torch.cuda.synchronize()
    rg = r.cpu().numpy()[ids]
    recs = []
    for j in range(n):
        before = o.state()
        ro, _ = o.step(None)
        recs.append((ro, o.info(), before))
    st = w.stations
    po = st.port_off
    sel = np.concatenate([np.arange(po[e], po[e + 1]) for e in ids])
    gs = b.get_state()
    s = {k: (v[sel] if v.shape[0] == b.P else v[ids]) for k, v in gs.items()}
    d0, d1 = state_drift(None, None, len(sel)), state_drift(s, o.state())
    for j, (ro, info, before) in enumerate(recs):
        assert_reward_close(rg[:, j], ro, traj_reward_scale(sub, info, before, d0, d1, n), TRAJ_RTOL,
                            where=f"step {j}")
    assert_events_equal(s, o.state(), "sampled")
    assert_traj_close(s, o.state(), charger_pmax(sub), TRAJ_RTOL, "sampled")
    # every upper node within eta x I on all stations (last step's power)
    pw = gs["p"].astype(np.float64)
    go, uo = st.group_off, st.upper_off
    gstart = np.concatenate([[0], np.cumsum(st.group_size)[:-1]])
    gsum = np.add.reduceat(pw, gstart)
    gcap = st.group_eta.astype(np.float64) * st.group_limit_kw
    assert np.all(gsum <= gcap * (1 + 1e-5) + 1e-4)
    for e in rng.choice(st.n_envs, 2000, replace=False):
        gpar, upar = st.group_parent[go[e]:go[e + 1]], st.upper_parent[uo[e]:uo[e + 1]]
        for u in range(st.n_upper[e]):
            under = np.zeros(go[e + 1] - go[e], bool)
            for g in range(len(under)):
                a = gpar[g]
                while a >= 0 and a != u:
                    a = upar[a]
                under[g] = a == u
            cap = float(st.upper_eta[uo[e] + u]) * float(st.upper_limit_kw[uo[e] + u])
            assert gsum[go[e]:go[e + 1]][under].sum() <= cap * (1 + 1e-5) + 1e-4


def test_extended_reset_subset_and_host_step(cuda_lib):
    """A subset reset and the host-buffer step on Fig. c trees in V2G mode
    with increment levels and charge-sensitive users: the reset stations
    start over (empty, battery at its initial SoC, no Delta t_remain left)
    exactly as in the oracle, and the host step (charger and battery levels
    copied in) equals the device step."""
    w, b, o, torch = make(n_envs=64, seed=13, **V2G, **CS, action_delta=1)
    for _ in range(20):
        b.step()
        o.step(None)
    ids = np.array([0, 5, 17, 40, 63], np.int32)
    b.reset(torch.from_numpy(ids).cuda(), seed=77)
    o.reset(ids, seed=77)
    gs = b.get_state()
    assert_events_equal(gs, o.state(), "after reset")
    po = w.stations.port_off
    for e in ids:
        assert np.all(gs["trem"][po[e]:po[e + 1]] == 0) and np.all(b.due()[po[e]:po[e + 1]] == 0)
    np.testing.assert_allclose(b.battery()["soc"][ids], w.params.batt_soc0, rtol=0, atol=0)
    np.testing.assert_allclose(b.battery()["soc"], o.battery()["soc"], rtol=0, atol=2e-4)
    compare_cs(w, b, o, torch, 24, mode="fused", k=8)
    # host step = device step, on two identical batches
    from paper_2507_01522_b300.chargax import Batch
    b1, b2 = Batch(w), Batch(w)
    rng = np.random.default_rng(3)
    for _ in range(5):
        acts = rng.integers(0, 21, b1.n_actions).astype(np.int8)
        hr = np.zeros(b1.E, np.float32)
        hd = np.zeros(b1.E, np.uint8)
        ho = np.zeros(b1.obs_size, np.float32)
        b1.step_host(acts, hr, hd, ho)
        r2 = torch.zeros(b2.E, device="cuda")
        d2 = torch.zeros(b2.E, dtype=torch.uint8, device="cuda")
        o2 = torch.zeros(b2.obs_size, device="cuda")
        b2.step(actions=torch.from_numpy(acts).cuda(), reward=r2, done=d2)
        b2.observe(o2)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(hr, r2.cpu().numpy())
        np.testing.assert_array_equal(hd, d2.cpu().numpy())
        np.testing.assert_array_equal(ho, o2.cpu().numpy())


def wrap_tree(st, frac=0.6):
    """Upper nodes over stations that had none: every station one node over
    all its groups (frac of the summed group limits), every second station
    also a node over its first half of the groups, every third one a node
    above all (uneven depth up to three levels)."""
    go = st.group_off
    n_upper, gpar, upar, ulim = [], [], [], []
    for e in range(st.n_envs):
        G = int(st.n_groups[e])
        glim = st.group_limit_kw[go[e]:go[e + 1]].astype(np.float64)
        nodes = []                                         # (parent, limit)
        top = -1
        if e % 3 == 0:
            nodes.append((-1, 0.9 * frac * glim.sum()))
            top = 0
        nodes.append((top, frac * glim.sum()))
        all_node = len(nodes) - 1
        parents = [all_node] * G
        if e % 2 == 0 and G >= 2:
            nodes.append((all_node, frac * glim[:G // 2].sum()))
            parents[:G // 2] = [len(nodes) - 1] * (G // 2)
        n_upper.append(len(nodes))
        gpar.extend(parents)
        upar.extend(p for p, _ in nodes)
        ulim.extend(l for _, l in nodes)
    return I.Stations(**{**st.__dict__, "n_upper": np.array(n_upper, np.int32),
                         "group_parent": np.array(gpar, np.int32), "upper_parent": np.array(upar, np.int32),
                         "upper_limit_kw": np.array(ulim, np.float32),
                         "upper_eta": np.full(len(ulim), 0.97, np.float32)})


@pytest.mark.parametrize("mode,k", [("plain", 1), ("fused", 24)])
def test_tree_on_every_class_edge(cuda_lib, mode, k):
    """Stations of 1, 8, 9, 16, 17, 32, 33, 64, 65 and 128 chargers (padding
    chargers, both kernel size ranges) with upper nodes of uneven depth."""
    import torch
    from paper_2507_01522_b300.chargax import Batch
    from test_gpu_parity import odd_sizes
    w = odd_sizes()
    w.stations = wrap_tree(w.stations)
    w.params = I.EnvParams(**{**w.params.__dict__, "alpha_con": 0.05})
    b, o = Batch(w), Oracle(w)
    compare_traj(w, b, o, torch, 72, mode=mode, k=k)
