"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks the oracle against something it cannot simply repeat: the
published Philox known-answer values, the exact Poisson CDF, closed-form
single-car trajectories (taper, Appendix A.1), hand-computed clipping cases
(Eq. ArchConst), conservation laws and state-domain invariants (Appendix A.2,
"State summary"), and the sampling distributions of the workload.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import Oracle
from paper_2507_01522_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# helpers: tiny hand-built workloads
# ----------------------------------------------------------------------------

def hand_workload(n_ports=1, groups=None, group_limit=1e9, grid_limit=1e9, port_types=None,
                  lam=0.0, price=0.2, ep_len=288, n_days=1, group_eta=None, grid_eta=1.0, **pkw):
    groups = groups or [n_ports]
    types = port_types if port_types is not None else [I.AC] * n_ports
    glim = group_limit if isinstance(group_limit, (list, tuple)) else [group_limit] * len(groups)
    geta = group_eta if group_eta is not None else [1.0] * len(groups)
    st = I.Stations(
        n_ports=np.array([n_ports], np.int32), port_type=np.array(types, np.uint8),
        n_groups=np.array([len(groups)], np.int32), group_size=np.array(groups, np.int32),
        group_limit_kw=np.array(glim, np.float32), group_eta=np.array(geta, np.float32),
        grid_limit_kw=np.array([grid_limit], np.float32), grid_eta=np.array([grid_eta], np.float32),
        arrival_class=np.array([0], np.int32))
    pr = np.full((n_days, ep_len), price, np.float32) if np.isscalar(price) else np.asarray(price, np.float32)
    exo = I.Exo(pr, np.full((1, ep_len), lam, np.float32))
    params = I.EnvParams(ep_len=ep_len, **pkw)
    return I.Workload("hand", params, st, exo, 0)


def park(o: Oracle, port, soc, cap, rbar, trem, erem=None, target=1.0):
    s = o.state()
    s["soc"][port] = soc
    s["cap"][port] = cap
    s["rbar"][port] = rbar
    s["trem"][port] = trem
    s["erem"][port] = (target - soc) * cap if erem is None else erem
    o.set_state(s)


# ----------------------------------------------------------------------------
# Philox4x32-10: published known-answer values
# ----------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# ----------------------------------------------------------------------------
# Poisson arrivals: exact inverse CDF
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("lam", [0.0, 0.03, 0.5, 1.0, 2.7, 8.0])
def test_poisson_matches_exact_inverse_cdf(lam):
    lam32 = float(np.float32(lam))
    rng = np.random.default_rng(1)
    words = rng.integers(0, 2 ** 32, size=4000, dtype=np.uint64)
    cdf = stats.poisson.cdf(np.arange(0, 200), lam32) if lam32 > 0 else np.ones(200)
    n_checked = 0
    for w in words:
        u = (int(w) >> 8) / 2.0 ** 24
        k = oracle.poisson(lam32, int(w))
        # exact inverse transform: smallest k with u < F(k); FP32 may differ
        # only when u sits within rounding distance of a CDF boundary
        k_exact = int(np.searchsorted(cdf, u, side="right"))
        if np.min(np.abs(cdf[:60] - u)) > 1e-5:
            assert k == k_exact, (lam, u, k, k_exact)
            n_checked += 1
    assert n_checked > 3500


def test_poisson_distribution_over_all_u():
    # sweep u over a fine regular grid: the histogram is the pmf
    lam = float(np.float32(3.25))
    n = 1 << 16
    words = (np.arange(n, dtype=np.uint64) << np.uint64(16)) + np.uint64(1 << 15)
    ks = np.array([oracle.poisson(lam, int(w)) for w in words])
    hist = np.bincount(ks, minlength=30)[:30] / n
    pmf = stats.poisson.pmf(np.arange(30), lam)
    assert np.max(np.abs(hist - pmf)) < 2.0 / n + 1e-6


def test_poisson_zero_rate_and_cap():
    assert oracle.poisson(0.0, 0xFFFFFFFF) == 0
    assert oracle.poisson(100.0, 0xFFFFFFFF) <= 127


# ----------------------------------------------------------------------------
# taper (Appendix A.1) and the closed-form single-car trajectory
# ----------------------------------------------------------------------------

def test_taper_shape():
    assert oracle.taper(0.3, 22.0, 0.8) == 22.0
    assert oracle.taper(0.8, 22.0, 0.8) == 22.0
    assert abs(oracle.taper(1.0, 22.0, 0.8)) < 1e-12
    assert abs(oracle.taper(0.9, 22.0, 0.8) - 11.0) < 1e-12      # halfway down the line
    assert abs(oracle.taper(0.8 + 1e-9, 22.0, 0.8) - 22.0) < 1e-6  # continuous at tau


def closed_form_soc(soc0, C, rbar, dt, tau, n):
    """SoC after n full-power steps: linear bulk phase, then geometric decay
    of (1 - SoC) with ratio 1 - dt*rbar/((1-tau) C)."""
    d = rbar * dt / C
    n_bulk = 0
    s = soc0
    # bulk steps happen while SoC <= tau at the start of the step
    n_bulk = int(math.floor((tau - soc0) / d)) + 1 if soc0 <= tau else 0
    out = []
    rho = 1.0 - dt * rbar / ((1.0 - tau) * C)
    for k in range(1, n + 1):
        if k <= n_bulk:
            out.append(soc0 + k * d)
        else:
            s_b = soc0 + n_bulk * d
            out.append(1.0 - (1.0 - s_b) * rho ** (k - n_bulk))
    return np.array(out)


@pytest.mark.parametrize("eta", [1.0, 0.95])
def test_single_car_closed_form(eta):
    p_buy, C, soc0, rbar = float(np.float32(0.2)), 50.0, 0.2, 22.0   # price table is float32
    w = hand_workload(n_ports=1, price=p_buy, eta_port=(eta, eta), alpha_sat=0.0, alpha_decl=0.0)
    o = Oracle(w)
    park(o, 0, soc=soc0, cap=C, rbar=rbar, trem=200)
    n = 60
    socs, rews = [], []
    for _ in range(n):
        r, d = o.step(np.array([10], np.int8))
        socs.append(o.state()["soc"][0])
        rews.append(r[0])
    expect = closed_form_soc(soc0, C, rbar, w.params.dt_h, w.params.tau, n)
    np.testing.assert_allclose(socs, expect, rtol=0, atol=1e-12)
    assert abs(socs[16] - 0.8233333333333333) < 1e-12          # 17 bulk steps
    dsoc = np.diff(np.concatenate([[soc0], expect]))
    expect_r = (0.75 - p_buy / eta) * C * dsoc                  # sells kWh, buys kWh/eta
    np.testing.assert_allclose(rews, expect_r, rtol=1e-12, atol=1e-12)
    # return of the absorption phase is a geometric sum
    s_b = expect[16]
    rho = 1.0 - w.params.dt_h * rbar / ((1 - w.params.tau) * C)
    tail = (0.75 - p_buy / eta) * C * (1 - s_b) * (1 - rho ** (n - 17))
    assert abs(sum(rews[17:]) - tail) < 1e-10


def test_short_stay_missing_energy_penalty():
    # stay of 5 steps: the car leaves after exactly 5 charging steps and the
    # missing energy C (1 - SoC_5) is charged at alpha_sat
    C, soc0, rbar, asat = 50.0, 0.2, 22.0, 0.3
    w = hand_workload(n_ports=1, price=0.2, alpha_sat=asat, alpha_decl=0.0)
    o = Oracle(w)
    park(o, 0, soc=soc0, cap=C, rbar=rbar, trem=5)
    rews = [o.step(np.array([10], np.int8))[0][0] for _ in range(6)]
    d = rbar * w.params.dt_h / C
    soc5 = soc0 + 5 * d
    missing = C * (1 - soc5)
    profit = (0.75 - float(np.float32(0.2)) / 0.95) * C * d
    np.testing.assert_allclose(rews[:4], [profit] * 4, rtol=1e-12)
    assert abs(rews[4] - (profit - asat * missing)) < 1e-10
    assert rews[5] == 0.0                                  # port now empty
    s = o.state()
    assert s["trem"][0] == 0 and s["cap"][0] == 0.0 and s["soc"][0] == 0.0


def test_demand_cap_binds():
    # a user wanting only 5 kWh at a DC charger: one step delivers exactly it
    w = hand_workload(n_ports=1, port_types=[I.DC], price=0.1, alpha_sat=0, alpha_decl=0)
    o = Oracle(w)
    park(o, 0, soc=0.2, cap=50.0, rbar=100.0, trem=50, erem=5.0)
    o.step(np.array([10], np.int8))
    s = o.state()
    assert abs(s["p"][0] - 5.0 / w.params.dt_h) < 1e-9     # 60 kW, not 100 or 150
    assert abs(s["erem"][0]) < 1e-12
    assert abs(s["soc"][0] - 0.3) < 1e-12
    o.step(np.array([10], np.int8))
    assert o.state()["p"][0] == 0.0


def test_soc_cap_binds():
    # near full: (1 - SoC) C / dt is below the taper rate and the port maximum
    w = hand_workload(n_ports=1, port_types=[I.DC], tau=0.5)
    o = Oracle(w)
    park(o, 0, soc=0.95, cap=40.0, rbar=150.0, trem=50)
    o.step(np.array([10], np.int8))
    s = o.state()
    # taper (1-0.95)*150/0.5 = 15 kW; soc cap = 0.05*40*12 = 24 kW -> taper binds
    assert abs(s["p"][0] - 15.0) < 1e-9
    o2 = Oracle(w)
    park(o2, 0, soc=0.99, cap=40.0, rbar=150.0, trem=50)
    w.params.tau = 0.999
    o3 = Oracle(w)
    park(o3, 0, soc=0.99, cap=40.0, rbar=150.0, trem=50, erem=10.0)
    o3.step(np.array([10], np.int8))
    # taper is flat until 0.999 -> 150 kW; the demand allows 10*12 = 120 kW;
    # the soc cap 0.01*40*12 = 4.8 kW binds
    assert abs(o3.state()["p"][0] - 4.8) < 1e-9
    assert abs(o3.state()["soc"][0] - 1.0) < 1e-12
    assert abs(o3.state()["erem"][0] - (10.0 - 0.4)) < 1e-12


# ----------------------------------------------------------------------------
# architecture clip, Eq. (ArchConst)
# ----------------------------------------------------------------------------

def full_station(w, levels, rbar=22.0, soc=0.3):
    o = Oracle(w)
    n = w.stations.total_ports
    for i in range(n):
        park(o, i, soc=soc, cap=80.0, rbar=rbar, trem=100)
    o.step(np.asarray(levels, np.int8))
    return o


def test_grid_clip_uniform():
    w = hand_workload(n_ports=16, grid_limit=150.0, group_limit=1e6)
    o = full_station(w, [10] * 16)
    np.testing.assert_allclose(o.power(), 150.0 / 16, rtol=1e-12)
    info = o.info()
    assert abs(info["ccon"][0] - (16 * 22.0 - 150.0)) < 1e-9


def test_group_then_grid_clip():
    w = hand_workload(n_ports=16, groups=[8, 8], group_limit=80.0, grid_limit=150.0)
    o = full_station(w, [10] * 16)
    np.testing.assert_allclose(o.power(), 9.375, rtol=1e-12)         # 80/8 = 10, then 150/160


def test_asymmetric_levels():
    w = hand_workload(n_ports=16, groups=[8, 8], group_limit=80.0, grid_limit=150.0)
    o = full_station(w, [10] * 8 + [2] * 8)
    # group A: 176 kW -> 80 (10 each); group B: 8 x 4.4 = 35.2 untouched; root 115.2 ok
    np.testing.assert_allclose(o.power()[:8], 10.0, rtol=1e-12)
    np.testing.assert_allclose(o.power()[8:], 4.4, rtol=1e-12)
    assert abs(o.info()["ccon"][0] - 96.0) < 1e-9                    # 176 - 80
    o = full_station(w, [10] * 8 + [5] * 8)
    # group B: 88 -> 80; root 160 -> 150
    np.testing.assert_allclose(o.power(), 9.375, rtol=1e-12)


def test_node_efficiency_and_mixed_groups():
    w = hand_workload(n_ports=6, groups=[2, 4], group_limit=[30.0, 1000.0], grid_limit=1000.0,
                      group_eta=[0.9, 1.0], port_types=[I.DC, I.DC, I.AC, I.AC, I.AC, I.AC])
    o = full_station(w, [10, 5, 10, 10, 0, 3], rbar=100.0)
    # DC ports request 100 (rbar) and 75 -> 175 vs 0.9*30 = 27 -> scale 27/175
    # AC ports: 22, 22, 0, 6.6 (level 3 of 22)
    p = o.power()
    eta32 = float(np.float32(0.9))                                    # inputs are float32
    np.testing.assert_allclose(p[:2], np.array([100.0, 75.0]) * eta32 * 30.0 / 175.0, rtol=1e-12)
    np.testing.assert_allclose(p[2:], [22.0, 22.0, 0.0, 6.6], rtol=1e-12)


def test_grid_efficiency():
    w = hand_workload(n_ports=4, grid_limit=50.0, grid_eta=0.8)
    o = full_station(w, [10] * 4)
    np.testing.assert_allclose(o.power(), float(np.float32(0.8)) * 50.0 / 4, rtol=1e-12)  # 0.8 * 50 shared


# ----------------------------------------------------------------------------
# trajectory invariants and distributions on the workload generators
# ----------------------------------------------------------------------------

def run_invariants(w, steps, actions_seed=None):
    o = Oracle(w)
    st = w.stations
    po, go = st.port_off, st.group_off
    p = w.params
    rng = np.random.default_rng(actions_seed) if actions_seed is not None else None
    arrival_step = {}
    for step in range(steps):
        s0 = o.state()
        acts = I.random_actions(rng, st.total_ports) if rng is not None else None
        r, d = o.step(acts)
        s1 = o.state()
        inf = o.info()
        pw = o.power()
        pmax = np.asarray(p.p_max_kw)[st.port_type]
        eta = np.asarray(p.eta_port)[st.port_type]
        occ0 = s0["trem"] > 0
        # power only where a car was, within port and car limits
        assert np.all(pw[~occ0] == 0.0)
        assert np.all(pw <= pmax * (1 + 1e-12))
        rb = s0["rbar"]
        rhat = np.where(s0["soc"] <= p.tau, rb, (1 - s0["soc"]) * rb / (1 - p.tau))
        assert np.all(pw <= rhat + 1e-9)
        for e in range(st.n_envs):
            if d[e]:
                continue                               # state already reset for a new episode
            sl = slice(po[e], po[e + 1])
            # group and root limits
            o_ = po[e]
            for g in range(go[e], go[e + 1]):
                n = st.group_size[g]
                assert pw[o_:o_ + n].sum() <= float(st.group_eta[g]) * float(st.group_limit_kw[g]) * (1 + 1e-9) + 1e-9
                o_ += n
            assert pw[sl].sum() <= float(st.grid_eta[e]) * float(st.grid_limit_kw[e]) * (1 + 1e-9) + 1e-9
            # energy: delivered energy equals the SoC gain of cars that stayed,
            # grid energy adds the port loss
            stay = occ0[sl] & (s1["trem"][sl] == s0["trem"][sl] - 1) & (s0["trem"][sl] > 1)
            gain = (s1["soc"][sl] - s0["soc"][sl]) * s0["cap"][sl]
            dE = pw[sl] * p.dt_h
            np.testing.assert_allclose(gain[stay], dE[stay], rtol=1e-9, atol=1e-9)
            np.testing.assert_allclose((s0["erem"][sl] - s1["erem"][sl])[stay], dE[stay], rtol=1e-9, atol=1e-9)
            assert abs(inf["enet"][e] - dE.sum()) < 1e-9
            assert abs(inf["egrid"][e] - (dE / eta[sl]).sum()) < 1e-9
            # arrivals: admitted + rejected = M, clipped by free ports
            free = st.n_ports[e] - int((occ0[sl] & (s0["trem"][sl] > 1)).sum())
            assert inf["admitted"][e] == min(inf["M"][e], free) or d[e]
        # state domains
        assert np.all((s1["soc"] >= 0) & (s1["soc"] <= 1))
        assert np.all(s1["erem"] >= 0)
        assert np.all(s1["trem"] >= 0) and np.all(s1["trem"] <= p.stay_steps[1])
        # stays: a port that received a car departs exactly `stay` steps later
        for i in np.nonzero((s0["trem"] == 1))[0]:
            if i in arrival_step:
                a_step, stay_len = arrival_step.pop(i)
                assert step - a_step == stay_len
        for e in np.nonzero(d)[0]:                      # episode end clears the station
            for i in range(po[e], po[e + 1]):
                arrival_step.pop(i, None)
        new = (s1["trem"] > 0) & ((s0["trem"] <= 1))
        for i in np.nonzero(new)[0]:
            arrival_step[i] = (step, int(s1["trem"][i]))
    return o


def test_invariants_fixed_station():
    w = I.fixed_station(n_envs=12)
    run_invariants(w, 300, actions_seed=3)


def test_invariants_heterogeneous_random_actions():
    w = I.heterogeneous(n_envs=16)
    run_invariants(w, 120)


def test_arrival_rate_statistics():
    # empirical mean arrivals per step-of-day bin vs lambda(t) within 4 sigma
    w = I.fixed_station(n_envs=256)
    w.params.stay_steps = (1, 1)       # free ports each step
    o = Oracle(w)
    T = w.params.ep_len
    sums = np.zeros(T)
    for t in range(T):
        o.step(np.zeros(w.stations.total_ports, np.int8))
        sums[t] = o.info()["M"].sum()
    lam = w.exo.arrival_rate[0].astype(np.float64)
    # aggregate in 24 one-hour bins
    mb = sums.reshape(24, 12).sum(1)
    lb = lam.reshape(24, 12).sum(1) * 256
    z = (mb - lb) / np.sqrt(lb)
    assert np.all(np.abs(z) < 4.5), z


def test_profile_distributions():
    w = I.heterogeneous(n_envs=64)
    w.exo.arrival_rate[:] = 30.0    # fill every free port every step
    w.params.stay_steps = (1, 1)
    o = Oracle(w)
    caps, socs, rb_ac, rb_dc = [], [], [], []
    types = w.stations.port_type
    for _ in range(40):
        o.step(np.zeros(w.stations.total_ports, np.int8))
        s = o.state()
        occ = s["trem"] > 0
        caps.append(s["cap"][occ]); socs.append(s["soc"][occ])
        rb_ac.append(s["rbar"][occ & (types == 0)]); rb_dc.append(s["rbar"][occ & (types == 1)])
    caps, socs = np.concatenate(caps), np.concatenate(socs)
    rb_ac, rb_dc = np.concatenate(rb_ac), np.concatenate(rb_dc)
    assert stats.kstest(caps, stats.uniform(40, 60).cdf).pvalue > 1e-4
    assert stats.kstest(socs, stats.uniform(0.1, 0.4).cdf).pvalue > 1e-4
    assert stats.kstest(rb_ac, stats.uniform(7, 15).cdf).pvalue > 1e-4
    assert stats.kstest(rb_dc, stats.uniform(50, 100).cdf).pvalue > 1e-4
    # the profile fields are independent draws
    assert abs(np.corrcoef(caps, socs)[0, 1]) < 0.05


def test_stay_range_inclusive_and_uniform():
    w = I.fixed_station(n_envs=64)
    w.exo.arrival_rate[:] = 30.0
    o = Oracle(w)
    stays = []
    prev = o.state()["trem"]
    for _ in range(100):
        o.step(np.zeros(w.stations.total_ports, np.int8))
        cur = o.state()["trem"]
        stays.append(cur[(cur > 0) & (prev <= 1)])
        prev = cur
    stays = np.concatenate(stays)
    assert stays.min() == 12 and stays.max() == 96
    counts = np.bincount(stays - 12, minlength=85)
    chi = stats.chisquare(counts)
    assert chi.pvalue > 1e-4


def test_random_actions_uniform():
    w = I.fixed_station(n_envs=4)
    o = Oracle(w)
    ks = [o.random_action(e, g, q) for e in range(4) for g in range(64) for q in range(16)]
    counts = np.bincount(ks, minlength=11)
    assert len(counts) == 11
    assert stats.chisquare(counts).pvalue > 1e-4


# ----------------------------------------------------------------------------
# special cases
# ----------------------------------------------------------------------------

def test_zero_actions_keep_soc_and_cost_only():
    w = I.fixed_station(n_envs=8)
    w.params.c_fixed = 0.7
    w.params.alpha_decl = 0.0
    w.params.alpha_sat = 0.0
    o = Oracle(w)
    z = np.zeros(w.stations.total_ports, np.int8)
    for _ in range(40):
        s0 = o.state()
        r, d = o.step(z)
        s1 = o.state()
        np.testing.assert_allclose(r, -0.7, rtol=0, atol=1e-15)
        keep = (s0["trem"] > 1)
        assert np.all(s1["soc"][keep] == s0["soc"][keep])


def test_no_arrivals_zero_reward():
    w = I.fixed_station(n_envs=4)
    w.exo.arrival_rate[:] = 0.0
    o = Oracle(w)
    for _ in range(300):
        r, d = o.step(None)
        assert np.all(r == 0.0)
    assert np.all(o.state()["trem"] == 0)


def test_small_station_saturates_and_rejects():
    w = I.heterogeneous(n_envs=8, classes=(8,))
    w.exo.arrival_rate[:] = 2.0
    o = Oracle(w)
    rej = 0
    for _ in range(100):
        o.step(None)
        inf = o.info()
        rej += int((inf["M"] - inf["admitted"]).sum())
        assert np.all(inf["M"] - inf["admitted"] >= 0)
    assert rej > 0
    st = o.stats()
    assert st["rejected"].sum() == rej


def test_decline_penalty_value():
    # all-zero actions, no fixed cost: the reward is exactly -alpha_decl * rejected
    w = I.heterogeneous(n_envs=8, classes=(8,))
    w.exo.arrival_rate[:] = 3.0
    w.params.alpha_decl = 0.5
    w.params.alpha_sat = 0.0
    o = Oracle(w)
    z = np.zeros(w.stations.total_ports, np.int8)
    for _ in range(50):
        r, _ = o.step(z)
        inf = o.info()
        np.testing.assert_allclose(r, -0.5 * (inf["M"] - inf["admitted"]), atol=1e-15)


def test_fcfs_first_free_ports():
    w = I.fixed_station(n_envs=32)
    w.exo.arrival_rate[:] = 6.0
    o = Oracle(w)
    po = w.stations.port_off
    seen = 0
    for _ in range(40):
        s0 = o.state()
        o.step(None)
        s1 = o.state()
        inf = o.info()
        for e in range(w.stations.n_envs):
            sl = slice(po[e], po[e + 1])
            free_after_departure = np.nonzero(s0["trem"][sl] <= 1)[0]
            got = np.nonzero((s1["trem"][sl] > 0) & (s0["trem"][sl] <= 1))[0]
            m = inf["admitted"][e]
            assert np.array_equal(got, free_after_departure[:m])
            seen += m
    assert seen > 100


def test_price_lookup_and_episode_end():
    T, D = 12, 5
    price = np.arange(D * T, dtype=np.float32).reshape(D, T) / 1000.0
    w = hand_workload(n_ports=4, price=price, ep_len=T, n_days=D, lam=1.5)
    o = Oracle(w)
    total = 0.0
    for k in range(3 * T):
        s0 = o.state()
        r, d = o.step(None)
        inf = o.info()
        assert inf["price"][0] == pytest.approx(price[s0["day"][0], s0["tod"][0]], abs=0)
        total += r[0]
        if (k + 1) % T == 0:
            assert d[0] == 1
            s1 = o.state()
            assert s1["tod"][0] == 0 and np.all(s1["trem"] == 0) and np.all(s1["p"] == 0)
            assert o.stats()["last_ret"][0] == pytest.approx(total, abs=1e-12)
            total = 0.0
        else:
            assert d[0] == 0
    assert o.stats()["n_episodes"][0] == 3


def test_reset_day_uniform():
    w = I.fixed_station(n_envs=4000)
    o = Oracle(w)
    days = o.state()["day"]
    assert days.min() >= 0 and days.max() < 365
    assert stats.chisquare(np.bincount(days // 73, minlength=5)).pvalue > 1e-4


def test_observation_hand_values():
    T = 288
    w = hand_workload(n_ports=2, port_types=[I.AC, I.DC], price=0.25, ep_len=T)
    o = Oracle(w)
    park(o, 1, soc=0.9, cap=50.0, rbar=100.0, trem=48)
    s = o.state(); s["tod"][0] = 72; s["day"][0] = 0; o.set_state(s)
    ob = o.observe()
    assert ob.shape == (8 + 12,)
    np.testing.assert_allclose(ob[:8], [1.0, 0.0, 0.25, 0.75, 0.5, 0.0, 0.25, 1.0], atol=1e-12)
    np.testing.assert_allclose(ob[8:14], 0.0)
    # DC port: occupied, soc 0.9, 48/96, taper (0.1*100/0.2 = 50)/150, p 0, erem 5/100
    np.testing.assert_allclose(ob[14:20], [1.0, 0.9, 0.5, 50.0 / 150.0, 0.0, 5.0 / 100.0], atol=1e-12)
    # weekday flag: days 0..4 of each week are weekdays, 5 and 6 are not
    wk = []
    w2 = hand_workload(n_ports=1, n_days=14, ep_len=T)
    o2 = Oracle(w2)
    for day in range(14):
        s = o2.state(); s["day"][0] = day; o2.set_state(s)
        wk.append(o2.observe()[7])
    assert wk == [1.0] * 5 + [0.0] * 2 + [1.0] * 5 + [0.0] * 2


def test_reset_subset_and_determinism():
    w = I.fixed_station(n_envs=6)
    a, b = Oracle(w), Oracle(w)
    for _ in range(30):
        ra, _ = a.step(None)
        rb, _ = b.step(None)
        assert np.array_equal(ra, rb)
    # the car count is the number of cars admitted since the last reset
    np.testing.assert_array_equal(a.state()["ncar"], a.stats()["arrived"].astype(np.uint32))
    a.reset([1, 4], seed=99)
    sa = a.state()
    assert sa["ncar"][1] == 0 and sa["ncar"][4] == 0 and sa["ncar"][0] == a.stats()["arrived"][0]
    assert sa["gstep"][1] == 0 and sa["gstep"][4] == 0 and sa["gstep"][0] == 30
    assert np.all(sa["trem"][16:32] == 0) and sa["key0"][1] == 99
