"""The serving loop (chx_srv_*): parity with the oracle through requests,
results independent of what shares a tick ("alone vs in the mix"), per-station
ordering, admission by HBM budget, errors, and the simulated actors."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2507_01522_b300 import inputs as I

from parity import TRAJ_RTOL, assert_reward_close, state_drift, traj_reward_scale
from test_gpu_parity import odd_sizes

pytestmark = pytest.mark.gpu

CAP = (64, 64, 64, 64, 64)


def server_for(w, **kw):
    from paper_2507_01522_b300.chargax import Server
    kw.setdefault("max_tick_obs_floats", 8 * w.stations.n_envs + 6 * w.stations.total_ports)
    return Server(w.params, w.exo, kw.pop("cap", CAP), **kw)


def partition(rng, n, max_size=40):
    perm = rng.permutation(n)
    out, i = [], 0
    while i < n:
        k = int(rng.integers(1, max_size + 1))
        out.append(perm[i:i + k])
        i += k
    return out


def obs_of(w, o_obs, envs):
    po = w.stations.port_off
    return np.concatenate([o_obs[8 * e + 6 * po[e]: 8 * (e + 1) + 6 * po[e + 1]] for e in envs])


def test_serving_matches_oracle():
    from paper_2507_01522_b300.chargax import CHX_SRV_RESET
    w = odd_sizes()
    srv = server_for(w)
    ids = srv.admit(w.stations, seed=5)
    assert len(set(ids.tolist())) == w.stations.n_envs
    o = Oracle(w, seed=5, streams=ids)
    rng = np.random.default_rng(1)
    po = w.stations.port_off
    for rnd in range(40):
        given = rnd % 3 == 2
        acts = I.random_actions(rng, w.stations.total_ports) if given else None
        if rnd == 25:                                   # a round of resets for a subset
            sub = np.sort(rng.choice(w.stations.n_envs, 30, replace=False))
            t = srv.submit(ids[sub], kind=CHX_SRV_RESET, seed=77)
            srv.wait(t)
            o.reset(sub, seed=77)
        reqs = []
        for part in partition(rng, w.stations.n_envs):
            r = np.zeros(len(part), np.float32)
            d = np.zeros(len(part), np.uint8)
            n_ch = int(sum(po[e + 1] - po[e] for e in part))
            ob = np.zeros(8 * len(part) + 6 * n_ch, np.float32)
            a = None if acts is None else np.concatenate([acts[po[e]:po[e + 1]] for e in part])
            reqs.append((part, r, d, ob, srv.submit(ids[part], actions=a, reward=r, done=d, obs=ob)))
        for _, _, _, _, t in reqs:
            srv.wait(t)
        before = o.state()
        ro, do = o.step(acts)
        info = o.info()
        # the pool's state is not read back: the drift allowance is the
        # per-step bound over the rounds so far (tests/parity.py)
        zero = state_drift(None, None, w.stations.total_ports)
        scale = traj_reward_scale(w, info, before, zero, zero, rnd + 1)
        oo = o.observe()
        for part, r, d, ob, _ in reqs:
            assert_reward_close(r, ro[part], scale[part], TRAJ_RTOL, where=f"round {rnd}")
            np.testing.assert_array_equal(d, do[part])
            exp = obs_of(w, oo, part)
            np.testing.assert_allclose(ob, exp, rtol=0, atol=2e-4, err_msg=f"obs round {rnd}")
            # events: occupancy and remaining stay are exact
            port_blocks = []
            k = 0
            for e in part:
                n = po[e + 1] - po[e]
                port_blocks.append(ob[k + 8: k + 8 + 6 * n].reshape(n, 6))
                k += 8 + 6 * n
            pb = np.concatenate(port_blocks)
            trem_o = o.state()["trem"][np.concatenate([np.arange(po[e], po[e + 1]) for e in part])]
            np.testing.assert_array_equal(np.rint(pb[:, 2] * w.params.stay_steps[1]).astype(int), trem_o)
            np.testing.assert_array_equal(pb[:, 0], (trem_o > 0).astype(np.float32))
    st = srv.stats()
    assert st["env_steps"] == 40 * w.stations.n_envs
    srv.stop()


def run_rounds(srv, ids, w, rounds, mix, seed=3):
    """Queue `rounds` rounds of steps (random partitions, some rounds with
    given actions, one reset round).  mix=False: every request alone (submit,
    wait).  mix=True: everything submitted at once, then waited."""
    from paper_2507_01522_b300.chargax import CHX_SRV_RESET
    rng = np.random.default_rng(seed)
    po = w.stations.port_off
    out, tickets = [], []
    for rnd in range(rounds):
        acts = I.random_actions(rng, w.stations.total_ports) if rnd % 2 else None
        parts = partition(rng, w.stations.n_envs, 25)
        for part in parts:
            r = np.zeros(len(part), np.float32)
            d = np.zeros(len(part), np.uint8)
            n_ch = int(sum(po[e + 1] - po[e] for e in part))
            ob = np.zeros(8 * len(part) + 6 * n_ch, np.float32)
            a = None if acts is None else np.concatenate([acts[po[e]:po[e + 1]] for e in part])
            t = srv.submit(ids[part], actions=a, reward=r, done=d, obs=ob)
            out.append((r, d, ob))
            tickets.append(t)
            if not mix:
                srv.wait(t)
        if rnd == 4:
            t = srv.submit(ids[parts[0]], kind=CHX_SRV_RESET, seed=9)
            tickets.append(t)
            if not mix:
                srv.wait(t)
    for t in tickets:
        if mix:
            srv.wait(t)
    return out


def test_serving_alone_equals_mix():
    """Each request's reward, done flags and observation are the same when it
    runs alone and when it shares ticks with others (here: bit-identical),
    with several rounds for the same stations queued at once (so per-station
    submission order must be kept)."""
    w = odd_sizes()
    a, b = server_for(w), server_for(w, n_streams=3)
    ia, ib = a.admit(w.stations, seed=2), b.admit(w.stations, seed=2)
    assert np.array_equal(ia, ib)
    alone = run_rounds(a, ia, w, 12, mix=False)
    mixed = run_rounds(b, ib, w, 12, mix=True)
    assert len(alone) == len(mixed)
    for (r1, d1, o1), (r2, d2, o2) in zip(alone, mixed):
        assert np.array_equal(r1, r2)
        assert np.array_equal(d1, d2)
        assert np.array_equal(o1, o2)
    sa, sb = a.stats(), b.stats()
    assert sb["n_ticks"] < sb["n_requests"]          # requests really shared ticks
    assert sa["n_ticks"] == sa["n_requests"]
    a.stop()
    b.stop()


def test_serving_admission_budget_and_errors():
    from paper_2507_01522_b300.chargax import CHX_EINVAL, CHX_ENOMEM, ChxError
    w = I.fixed_station(n_envs=12)
    one = 16 * 33.0 + 128.0
    srv = server_for(w, cap=(0, 11, 0, 0, 0), hbm_budget_bytes=10 * one + 1)
    ids = srv.admit(w.stations.subset(range(10)))
    with pytest.raises(ChxError) as ei:                  # budget
        srv.admit(w.stations.subset([10]))
    assert ei.value.code == CHX_ENOMEM
    srv.evict(ids[:2])
    more = srv.admit(w.stations.subset([10, 11]))
    assert srv.stats()["resident"] == 10
    small = server_for(w, cap=(0, 2, 0, 0, 0))
    with pytest.raises(ChxError) as ei:                  # class capacity (2 slots)
        small.admit(w.stations.subset([0, 1, 2]))
    assert ei.value.code == CHX_ENOMEM
    assert small.stats()["resident"] == 0                # all or nothing
    small.admit(w.stations.subset([0, 1]))
    small.stop()
    assert set(more.tolist()) == set(ids[:2].tolist())   # freed slots are reused
    srv.evict(more[1:2])
    for bad_id in (more[1:2], np.array([10 ** 6])):      # evicted / never admitted
        with pytest.raises(ChxError) as ei:
            srv.submit(bad_id)
        assert ei.value.code == CHX_EINVAL
    with pytest.raises(ChxError) as ei:                  # duplicate station
        srv.submit(np.array([more[0], more[0]]))
    assert ei.value.code == CHX_EINVAL
    bad = np.full(16, 11, np.int8)
    with pytest.raises(ChxError) as ei:                  # action level out of range
        srv.submit(more[:1], actions=bad)
    assert ei.value.code == CHX_EINVAL
    # a station with a queued request cannot be evicted
    r = np.zeros(1, np.float32)
    t = srv.submit(more[:1], reward=r)
    try:
        srv.evict(more[:1])
        evicted = True
    except ChxError as e:
        evicted = False
        assert e.code == CHX_EINVAL
    srv.wait(t)
    if evicted:                                          # it may have finished first
        return
    srv.evict(more[:1])
    srv.stop()


def test_serving_full_record_table_refuses():
    """Ticket t uses record t mod 65536: with 65536 tickets unreleased, the
    next submission returns CHX_ENOMEM at once without taking a ticket; once
    one ticket is released the submission goes through."""
    import time
    from paper_2507_01522_b300.chargax import CHX_ENOMEM, ChxError
    w = I.fixed_station(n_envs=4)
    srv = server_for(w, cap=(0, 4, 0, 0, 0))
    ids = srv.admit(w.stations)
    tickets = [srv.submit(ids[i % 4:i % 4 + 1]) for i in range(65536)]
    t0 = time.perf_counter()
    with pytest.raises(ChxError) as ei:
        srv.submit(ids[:1])
    assert ei.value.code == CHX_ENOMEM
    assert time.perf_counter() - t0 < 0.1
    srv.wait(tickets[0])                                 # releases the record the next ticket uses
    t = srv.submit(ids[:1])
    assert t == tickets[-1] + 1
    for k in tickets[1:] + [t]:
        srv.wait(k)
    srv.stop()


def test_serving_simulation_reports_latency():
    w = I.serving_pool(n_envs=2048, seed=1)
    cap = [int(np.sum((w.stations.n_ports > (4 << c)) & (w.stations.n_ports <= (8 << c)))) for c in range(5)]
    cap[0] += int(np.sum(w.stations.n_ports <= 4))
    srv = server_for(w, cap=cap, max_tick_obs_floats=0, max_tick_envs=4096)
    ids = srv.admit(w.stations)
    res = srv.simulate(ids, n_actors=64, envs_per_actor=32, mean_think_us=200.0, duration_s=0.5, warmup_s=0.2,
                       n_threads=4, reset_every=10)
    assert res["n_requests"] > 100
    assert 0 < res["p50_us"] <= res["p99_us"] <= res["max_us"]
    assert res["env_steps_per_s"] > 0
    assert res["mean_tick_envs"] > 0
    srv.stop()


def test_serving_wait_timeout():
    """A wait that runs out of time returns CHX_ETIMEOUT and leaves the ticket
    valid; a later wait collects it."""
    from paper_2507_01522_b300.chargax import CHX_ETIMEOUT, ChxError
    w = I.serving_pool(n_envs=4096, seed=3)
    n = w.stations.n_ports
    cap = [int(np.sum(n <= 8))] + [int(np.sum((n > (4 << c)) & (n <= (8 << c)))) for c in range(1, 5)]
    srv = server_for(w, cap=cap, max_tick_obs_floats=0, max_tick_envs=4096)
    ids = srv.admit(w.stations)
    seen = False
    for _ in range(5):
        r = np.zeros(len(ids), np.float32)
        t = srv.submit(ids, reward=r)
        try:
            srv.wait(t, timeout_us=0)
        except ChxError as e:
            assert e.code == CHX_ETIMEOUT
            seen = True
        else:
            continue                                     # finished before the zero-time wait
        lat = srv.wait(t)
        assert lat > 0 and np.all(np.isfinite(r))
    assert seen
    srv.stop()


def test_serving_fullsize_sampled():
    """The benchmark's serving pool: 1,048,576 resident stations of 8-128
    chargers (log-uniform, about 45 M chargers), admitted with the
    benchmark's class capacities and tick size.  Rounds that step every
    station (requests of 256 stations, Philox actions) alternate with rounds
    that step only a sample (64 stations of each size class, the first and
    the last admitted) in random partitions, with observations, given
    actions and one reset; the oracle runs the sample alone, on the same
    Philox streams, and must agree on every sampled reward, done flag,
    observation and occupancy."""
    from paper_2507_01522_b300.chargax import CHX_SRV_RESET, Server
    w = I.serving_pool(1 << 20, seed=0)
    st = w.stations
    n = st.n_ports
    cap = [int(np.sum(n <= 8))] + [int(np.sum((n > (4 << c)) & (n <= (8 << c)))) for c in range(1, 5)]
    rng = np.random.default_rng(12)
    bounds = [(1, 8), (9, 16), (17, 32), (33, 64), (65, 128)]
    sample = np.unique(np.concatenate(
        [rng.choice(np.flatnonzero((n >= lo) & (n <= hi)), 64, replace=False) for lo, hi in bounds]
        + [np.array([0, st.n_envs - 1])]))
    sub = st.subset(sample)
    obs_floats = 8 * len(sample) + 6 * int(sub.total_ports)
    srv = Server(w.params, w.exo, cap, hbm_budget_bytes=150e9, max_tick_envs=65536, n_streams=2,
                 max_tick_obs_floats=obs_floats)
    seed = 2000
    ids = srv.admit(st, seed=seed)
    assert len(np.unique(ids)) == st.n_envs
    ws = I.Workload(w.name, w.params, sub, w.exo, w.seed)
    o = Oracle(ws, seed=seed, streams=ids[sample])
    po = sub.port_off
    active = []

    def compare(rnd, r_s, d_s, ob_parts=None):
        before = o.state()
        ro, do = o.step(acts)
        info = o.info()
        zero = state_drift(None, None, ws.stations.total_ports)
        scale = traj_reward_scale(ws, info, before, zero, zero, rnd + 1)
        assert_reward_close(r_s, ro, scale, TRAJ_RTOL, where=f"round {rnd}")
        np.testing.assert_array_equal(d_s, do, err_msg=f"done round {rnd}")
        active.append((int(np.count_nonzero(ro)), int(np.count_nonzero(o.state()["trem"]))))
        if ob_parts is None:
            return
        oo = o.observe()
        trem_o = o.state()["trem"]
        for part, ob in ob_parts:
            np.testing.assert_allclose(ob, obs_of(ws, oo, part), rtol=0, atol=2e-4, err_msg=f"obs round {rnd}")
            blocks, k = [], 0
            for e in part:
                m = po[e + 1] - po[e]
                blocks.append(ob[k + 8: k + 8 + 6 * m].reshape(m, 6))
                k += 8 + 6 * m
            pb = np.concatenate(blocks)
            tr = trem_o[np.concatenate([np.arange(po[e], po[e + 1]) for e in part])]
            np.testing.assert_array_equal(np.rint(pb[:, 2] * ws.params.stay_steps[1]).astype(int), tr)

    for rnd in range(9):
        acts = None
        if rnd in (0, 1, 8):                               # every resident station, 4096 requests of 256
            r_all = np.zeros(st.n_envs, np.float32)
            d_all = np.zeros(st.n_envs, np.uint8)
            perm = rng.permutation(st.n_envs)
            reqs = []
            for j in range(0, st.n_envs, 256):
                part = perm[j:j + 256]
                r = np.zeros(len(part), np.float32)
                d = np.zeros(len(part), np.uint8)
                reqs.append((part, r, d, srv.submit(ids[part], reward=r, done=d)))
            for part, r, d, t in reqs:
                srv.wait(t)
                r_all[part] = r
                d_all[part] = d
            compare(rnd, r_all[sample], d_all[sample])
            continue
        if rnd == 5:                                       # a reset for a third of the sample
            rs = np.sort(rng.choice(len(sample), len(sample) // 3, replace=False))
            srv.wait(srv.submit(ids[sample[rs]], kind=CHX_SRV_RESET, seed=77))
            o.reset(rs, seed=77)
        if rnd % 2:
            acts = I.random_actions(rng, int(sub.total_ports))
        r_s = np.zeros(len(sample), np.float32)
        d_s = np.zeros(len(sample), np.uint8)
        reqs = []
        for part in partition(rng, len(sample)):
            r = np.zeros(len(part), np.float32)
            d = np.zeros(len(part), np.uint8)
            ob = np.zeros(8 * len(part) + 6 * int(sum(po[e + 1] - po[e] for e in part)), np.float32)
            a = None if acts is None else np.concatenate([acts[po[e]:po[e + 1]] for e in part])
            reqs.append((part, r, d, ob, srv.submit(ids[sample[part]], actions=a, reward=r, done=d, obs=ob)))
        for part, r, d, ob, t in reqs:
            srv.wait(t)
            r_s[part] = r
            d_s[part] = d
        compare(rnd, r_s, d_s, [(part, ob) for part, _, _, ob, _ in reqs])
    stats = srv.stats()
    assert stats["env_steps"] == 3 * st.n_envs + 6 * len(sample)
    # the sample was busy: most stations earn a reward and hold cars in the later rounds
    assert min(a for a, _ in active[2:]) > len(sample) // 2 and min(c for _, c in active[2:]) > len(sample)
    srv.stop()
