"""Pins of the oracle's charge-sensitive users (u = 1; A.1 User Profiles,
A.2 "Departure of Cars", A.3 c_Sat,1) against what the paper and arithmetic
fix: departure steps of a car charged at a known rate (early and overdue)
with c_Sat,1 read from the reward difference, the remaining-demand
threshold on hand-built remainders, a never-charged car staying to the
episode end, instant departure of a car whose demand is met on arrival,
the share of charge-sensitive users (binomial test), the observation, and
invariants along random trajectories."""

import numpy as np
import pytest
from scipy import stats

from oracle import Oracle
from paper_2507_01522_b300 import inputs as I

from test_oracle_pins import hand_workload, park

CS = 255   # trem of a port holding a charge-sensitive car

def park_cs(o, port, due, **kw):
    park(o, port, trem=CS, **kw)
    d = o.due()
    d[port] = due
    o.set_due(d)

def run_levels(o, level, n):
    rew, occ = [], []
    for _ in range(n):
        r, _ = o.step(np.array([level] * o.P, np.int8))
        rew.append(r[0]); occ.append(o.state()["trem"].copy())
    return np.array(rew), occ

@pytest.mark.parametrize("due,early", [(10, True), (3, False)])
def test_departure_when_charged_and_csat1(due, early):
    """5 kWh of demand at 11 kW (rbar) on a 22 kW charger: 11/12 kWh per
    step, so the demand is met in step ceil(5 / (11/12)) = 6 (the last one
    capped by the demand); the car leaves at its end with Delta t_remain =
    due - 6: c_Sat,1 = -beta x 4 (early) or 3 (overdue), seen as the reward
    difference between alpha_sat1 = 0 and 0.2."""
    out = {}
    for a in (0.0, 0.2):
        w = hand_workload(n_ports=1, cs_share_256=256, alpha_sat1=a, beta_early=0.5, alpha_sat=0.3,
                          alpha_decl=0.0)
        o = Oracle(w)
        park_cs(o, 0, due, soc=0.5, cap=50.0, rbar=11.0, erem=5.0)
        out[a] = run_levels(o, 10, 8)
    (r0, occ), (r1, _) = out[0.0], out[0.2]
    assert [int(x[0]) for x in occ] == [CS] * 5 + [0, 0, 0]
    d = due - 6
    csat1 = max(0, -d) - 0.5 * max(0, d)
    expect = np.zeros(8)
    expect[5] = -0.2 * csat1
    np.testing.assert_allclose(r1 - r0, expect, rtol=0, atol=1e-12)
    assert (csat1 < 0) == early
    # a time-sensitive user with the same profile leaves at its stay instead,
    # with its missing energy as c_Sat,0
    w = hand_workload(n_ports=1, alpha_sat=0.3, alpha_decl=0.0)
    o = Oracle(w)
    park(o, 0, soc=0.5, cap=50.0, rbar=11.0, trem=due, erem=5.0)
    rts, occ = run_levels(o, 10, due)
    assert int(occ[due - 1][0]) == 0 and all(int(x[0]) > 0 for x in occ[:due - 1])

def test_demand_met_threshold():
    """Capacity 50 kWh: the demand counts as met at 1e-3 x 50 = 0.05 kWh.
    At 0.06 kW (0.005 kWh per step) a car with 0.0512 kWh left ends at
    0.0462 and leaves; one with 0.0562 ends at 0.0512, stays, and leaves a
    step later."""
    w = hand_workload(n_ports=2, cs_share_256=256, alpha_sat=0.0, alpha_decl=0.0)
    o = Oracle(w)
    park_cs(o, 0, 50, soc=0.5, cap=50.0, rbar=0.06, erem=0.0512)
    park_cs(o, 1, 50, soc=0.5, cap=50.0, rbar=0.06, erem=0.0562)
    o.step(np.array([10, 10], np.int8))
    s = o.state()
    assert list(s["trem"]) == [0, CS]
    np.testing.assert_allclose(s["erem"][1], 0.0512, rtol=1e-12)
    np.testing.assert_allclose(o.info_cs()["margin"][0], 0.0012 / 0.05, rtol=1e-9)
    o.step(np.array([10, 10], np.int8))
    assert list(o.state()["trem"]) == [0, 0]


def test_threshold_reached_under_a_group_limit():
    """Two charge-sensitive cars with 1 kWh left (capacity 50 kWh) in a
    2.304 kW group: the proportional rescale gives each 1.152 kW, 0.096 kWh
    per step, so 1 - 0.096 k remains; at k = 10 that is 0.04 kWh, below
    1e-3 x 50, and both leave a step before the demand cap would finish
    them."""
    w = hand_workload(n_ports=2, cs_share_256=256, group_limit=2.304, alpha_sat=0.0, alpha_decl=0.0)
    o = Oracle(w)
    for q in (0, 1):
        park_cs(o, q, 50, soc=0.5, cap=50.0, rbar=50.0, erem=1.0)
    glim = float(np.float32(2.304))                       # limits are stored in FP32
    for k in range(1, 10):
        o.step(np.array([10, 10], np.int8))
        s = o.state()
        assert list(s["trem"]) == [CS, CS]
        np.testing.assert_allclose(s["erem"], 1.0 - k * glim / 24.0, rtol=1e-12)
    o.step(np.array([10, 10], np.int8))
    assert list(o.state()["trem"]) == [0, 0]


def test_uncharged_car_stays_to_episode_end():
    """Level 0 never charges: the charge-sensitive car stays past its due
    time (Delta t_remain counts down through 0 into overdue steps) until the
    episode ends, which clears it without a satisfaction penalty."""
    w = hand_workload(n_ports=1, cs_share_256=256, ep_len=30, alpha_sat1=1.0, alpha_decl=0.0, c_fixed=0.0)
    o = Oracle(w)
    park_cs(o, 0, 5, soc=0.3, cap=50.0, rbar=11.0, erem=20.0)
    for t in range(29):
        r, d = o.step(np.array([0], np.int8))
        assert o.state()["trem"][0] == CS and o.due()[0] == 5 - (t + 1)
        assert r[0] == 0.0 and d[0] == 0
    r, d = o.step(np.array([0], np.int8))
    assert d[0] == 1 and r[0] == 0.0
    assert o.state()["trem"][0] == 0 and o.due()[0] == 0

def test_met_demand_leaves_after_one_step():
    """With the target SoC below every arrival SoC the demand is 0 on
    arrival: every admitted charge-sensitive car leaves at the end of its
    first step (its early-leave bonus is beta x (stay - 1))."""
    w = hand_workload(n_ports=16, cs_share_256=256, lam=3.0, soc_target=0.05, alpha_sat=0.0, alpha_decl=0.0,
                      alpha_sat1=0.1, beta_early=0.5)
    o = Oracle(w)
    prev_adm = 0
    total = 0
    for t in range(40):
        r, _ = o.step(None)
        inf = o.info()
        assert inf["departed"][0] == prev_adm
        s = o.state()
        assert np.all((s["trem"] == 0) | (s["trem"] == CS))
        # the bonus: beta x the steps left, over the cars that left now
        assert o.info_cs()["csat1"][0] <= 0.0
        prev_adm = inf["admitted"][0]
        total += prev_adm
    assert total > 50

def test_share_of_charge_sensitive_users():
    """cs_share_256 = 96: each admitted user is charge-sensitive with
    probability 96/256 (binomial two-sided test on the arrivals)."""
    w = I.heterogeneous(n_envs=64, seed=5)
    w.params.cs_share_256 = 96
    w.params.ep_len = 60
    w.exo = I.Exo(I.price_bank(n_days=3, ep_len=60, seed=5), I.arrival_rates([8, 16, 32, 64], ep_len=60, base=1.0))
    o = Oracle(w)
    n_cs = n_all = 0
    prev = o.state()
    for _ in range(50):
        o.step(None)
        cur = o.state()
        # a port holds a new car if it was free or its car's capacity changed
        fresh = (cur["trem"] > 0) & ((prev["trem"] == 0) | (cur["cap"] != prev["cap"]))
        n_all += int(fresh.sum()); n_cs += int((cur["trem"][fresh] == CS).sum())
        prev = cur
    assert n_all > 2000
    p = stats.binomtest(n_cs, n_all, 96 / 256).pvalue
    assert p > 1e-3, (n_cs, n_all)

def test_observation_port_features():
    w = hand_workload(n_ports=3, cs_share_256=256, alpha_decl=0.0)
    o = Oracle(w)
    assert o.obs_port_features == 7
    park_cs(o, 0, 7, soc=0.4, cap=50.0, rbar=11.0, erem=20.0)
    park(o, 1, soc=0.3, cap=60.0, rbar=11.0, trem=12)
    ob = o.observe()
    F, mx = 8, w.params.stay_steps[1]
    assert ob.size == F + 7 * 3
    np.testing.assert_allclose(ob[F:F + 7], [1.0, 0.4, 7 / mx, 11.0 / 22.0, 0.0, 20.0 / w.params.cap_kwh[1], 1.0])
    np.testing.assert_allclose(ob[F + 7:F + 14], [1.0, 0.3, 12 / mx, 11.0 / 22.0, 0.0, 0.7 * 60 / w.params.cap_kwh[1], 0.0])
    np.testing.assert_array_equal(ob[F + 14:], 0.0)
    for _ in range(9):
        o.step(np.array([0, 0, 0], np.int8))
    assert o.observe()[F + 2] == pytest.approx(-2 / mx)          # overdue: negative Delta t_remain

def test_cs_invariants_along_random_trajectories():
    """Half charge-sensitive users, every penalty on: each step a
    charge-sensitive car either stays, its remaining demand above the
    threshold and Delta t_remain one lower, or leaves with its demand met;
    time-sensitive cars keep their stay rule; SoC and demand domains hold."""
    w = I.heterogeneous(n_envs=32, seed=7)
    p = w.params
    p.cs_share_256, p.alpha_sat1, p.beta_early, p.soc_target = 128, 0.05, 0.5, 0.8
    p.ep_len = 80
    w.exo = I.Exo(I.price_bank(n_days=3, ep_len=80, seed=7), I.arrival_rates([8, 16, 32, 64], ep_len=80, base=1.0))
    o = Oracle(w)
    rng = np.random.default_rng(3)
    seen_cs_leave = 0
    for t in range(160):
        s0, d0 = o.state(), o.due()
        _, done = o.step(rng.integers(0, 11, o.P).astype(np.int8))
        s1, d1 = o.state(), o.due()
        if done.any():
            continue
        cs0 = s0["trem"] == CS
        stay = cs0 & (s1["trem"] == CS) & (s1["cap"] == s0["cap"])
        assert np.all(d1[stay] == d0[stay] - 1)
        assert np.all(s1["erem"][stay] > p.eps_cap * s1["cap"][stay])
        left = cs0 & ((s1["trem"] != CS) | (s1["cap"] != s0["cap"]))
        seen_cs_leave += int(left.sum())
        assert np.all((s1["soc"] >= 0) & (s1["soc"] <= 1)) and np.all(s1["erem"] >= 0)
        ts = (s0["trem"] > 0) & (s0["trem"] != CS)
        moved = ts & (s1["trem"] != 0) & (s1["trem"] != CS) & (s1["cap"] == s0["cap"])
        assert np.all(s1["trem"][moved] == s0["trem"][moved] - 1)
    assert seen_cs_leave > 20


def test_user_draw_from_the_pinned_generator():
    """The n-th car of a station takes its profile from the Philox block
    (stream, n, 0, purpose 1) of the known-answer-pinned generator: its user
    is charge-sensitive iff the low byte of word 0 is below the share, and
    its stay (time-sensitive: remaining steps; charge-sensitive: Delta
    t_remain) is stay_lo + the high word of word 2 x the span."""
    import oracle
    w = hand_workload(n_ports=16, cs_share_256=128, lam=2.0, alpha_decl=0.0, stay_steps=(2, 8), soc_target=0.55)
    o = Oracle(w)
    p = w.params
    lo, span = p.stay_steps[0], p.stay_steps[1] - p.stay_steps[0] + 1
    checked = n_cs = 0
    for _ in range(30):
        s0 = o.state()
        o.step(np.full(16, 10, np.int8))
        s1, due = o.state(), o.due()
        n0, n1 = int(s0["ncar"][0]), int(s1["ncar"][0])
        new = np.flatnonzero((s1["trem"] > 0) & ((s0["trem"] <= 1) | (s1["cap"] != s0["cap"])))
        new = [i for i in new if s1["cap"][i] != s0["cap"][i]]
        assert len(new) == n1 - n0
        for j, i in enumerate(sorted(new)):
            wd = oracle.philox([0, n0 + j, 0, 1], [int(s1["key0"][0]), int(s1["key1"][0])])
            cs = (int(wd[0]) & 0xFF) < 128
            stay = lo + ((int(wd[2]) * span) >> 32)
            if cs:
                assert s1["trem"][i] == CS and due[i] == stay
                n_cs += 1
            else:
                assert s1["trem"][i] == stay and due[i] == 0
            checked += 1
    assert checked > 30 and 0 < n_cs < checked


def test_charge_sensitive_departure_carries_no_csat0():
    """A charge-sensitive car leaving with 0.0462 kWh still due (below its
    threshold) adds nothing to c_Sat,0, the time-sensitive users' term: the
    reward does not move with alpha_sat."""
    out = []
    for a in (0.0, 1.0):
        w = hand_workload(n_ports=1, cs_share_256=256, alpha_sat=a, alpha_decl=0.0)
        o = Oracle(w)
        park_cs(o, 0, 50, soc=0.5, cap=50.0, rbar=0.06, erem=0.0512)
        r, _ = o.step(np.array([10], np.int8))
        assert o.state()["trem"][0] == 0
        out.append(r[0])
    assert out[0] == out[1]
