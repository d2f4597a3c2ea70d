"""Pins of the oracle's vehicle-to-grid mode (signed levels, station battery,
sell-back price, degradation penalty) against what the paper's formulas and
mathematics fix: the reduction to the (separately pinned) charge-only mode,
closed-form discharge and battery trajectories with their rewards, the
signed architecture limits on hand-computed cases, and invariants along
random trajectories."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2507_01522_b300 import inputs as I

from test_oracle_pins import hand_workload, park

V2G = dict(v2g=1, n_levels=21)


def v2g_actions(rng, st, n_levels=21, steps=None):
    """Levels for every port plus one battery level per station (V2G layout:
    the station's ports, then its battery)."""
    n = st.total_ports + st.n_envs
    return rng.integers(0, n_levels, size=(n,) if steps is None else (n, steps)).astype(np.int8)


def with_battery_slots(st, port_levels, battery_levels):
    """Interleave per-port levels (batch order) with one battery level per station."""
    out = []
    for e in range(st.n_envs):
        out.extend(port_levels[st.port_off[e]:st.port_off[e + 1]])
        out.append(battery_levels[e])
    return np.array(out, np.int8)


def test_v2g_reduces_to_charge_only():
    """Non-negative levels (k >= h) and an idle battery (k = h): the V2G mode
    gives the charge-only mode's trajectory exactly (every reward term on)."""
    w0 = I.heterogeneous(n_envs=24, seed=3)
    p = w0.params
    p.alpha_con, p.alpha_sat, p.alpha_decl, p.c_fixed, p.ep_len = 0.05, 0.2, 0.3, 0.01, 40
    p.eta_port = (0.95, 0.9)
    w0.exo = I.Exo(I.price_bank(n_days=5, ep_len=40, seed=3), I.arrival_rates([8, 16, 32, 64], ep_len=40, base=1.5))
    w1 = I.Workload(w0.name, I.EnvParams(**{**p.__dict__, **V2G}), w0.stations, w0.exo, w0.seed)
    o0, o1 = Oracle(w0), Oracle(w1)
    st = w0.stations
    rng = np.random.default_rng(4)
    for step in range(90):
        lv = rng.integers(0, 11, st.total_ports).astype(np.int8)
        r0, d0 = o0.step(lv)
        r1, d1 = o1.step(with_battery_slots(st, lv + 10, np.full(st.n_envs, 10)))
        np.testing.assert_array_equal(r0, r1, err_msg=f"step {step}")
        np.testing.assert_array_equal(d0, d1)
    s0, s1 = o0.state(), o1.state()
    for k in s0:
        np.testing.assert_array_equal(s0[k], s1[k], err_msg=k)
    np.testing.assert_array_equal(o1.battery()["soc"], np.full(st.n_envs, p.batt_soc0))
    ob0, ob1 = o0.observe(), o1.observe()
    F0, F1 = 8, 10
    for e in range(st.n_envs):
        a0 = F0 * e + 6 * st.port_off[e]
        a1 = F1 * e + 6 * st.port_off[e]
        n = int(st.n_ports[e])
        np.testing.assert_array_equal(ob0[a0:a0 + 8], ob1[a1:a1 + 8])
        np.testing.assert_array_equal(ob0[a0 + 8:a0 + 8 + 6 * n], ob1[a1 + 10:a1 + 10 + 6 * n])


def closed_form_discharge(soc0, C, rbar, dt, tau, n):
    """SoC after n full-discharge steps along the flipped curve r_hat(1 - SoC):
    linear while 1 - SoC <= tau, then geometric decay of SoC with ratio
    1 - dt * rbar / ((1 - tau) C)."""
    d = rbar * dt / C
    n_bulk = int(math.floor((soc0 - (1.0 - tau)) / d)) + 1 if soc0 >= 1.0 - tau else 0
    rho = 1.0 - dt * rbar / ((1.0 - tau) * C)
    out = []
    for k in range(1, n + 1):
        if k <= n_bulk:
            out.append(soc0 - k * d)
        else:
            out.append((soc0 - n_bulk * d) * rho ** (k - n_bulk))
    return np.array(out)


@pytest.mark.parametrize("eta", [1.0, 0.9])
def test_single_car_discharge_closed_form(eta):
    price, C, soc0, rbar, ratio = float(np.float32(0.2)), 50.0, 0.6, 20.0, 0.8
    w = hand_workload(n_ports=1, price=price, eta_port=(eta, eta), alpha_sat=0.0, alpha_decl=0.0,
                      sell_grid_ratio=ratio, alpha_degrad=0.03, **V2G)
    o = Oracle(w)
    park(o, 0, soc=soc0, cap=C, rbar=rbar, trem=250, erem=5.0)
    n = 80
    socs, erems, rews = [], [], []
    for _ in range(n):
        r, _ = o.step(np.array([0, 10], np.int8))            # full discharge, battery idle
        s = o.state()
        socs.append(s["soc"][0]); erems.append(s["erem"][0]); rews.append(r[0])
    dt = w.params.dt_h
    expect = closed_form_discharge(soc0, C, rbar, dt, w.params.tau, n)
    np.testing.assert_allclose(socs, expect, rtol=0, atol=1e-12)
    # 13 bulk steps of 20 kW (SoC 0.6 -> 0.2 at 1/30 per step), then geometric
    assert abs(socs[11] - (0.6 - 12 * dt * rbar / C)) < 1e-12
    dE = -C * np.diff(np.concatenate([[soc0], expect]))     # energy taken out of the car, > 0
    np.testing.assert_allclose(erems, 5.0 + np.cumsum(dE), rtol=1e-12, atol=1e-9)
    # revenue: the station pays the user p_sell per kWh taken, sells eta x that
    # to the grid at ratio x p_buy, and pays the degradation cost on eta x kWh
    expect_r = -0.75 * dE + ratio * price * eta * dE - 0.03 * eta * dE
    np.testing.assert_allclose(rews, expect_r, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("tau", [0.8, 0.65])
def test_battery_closed_form_and_two_case_profit(tau):
    """No cars: the battery charges at its full rate from the grid (buy
    price), then discharges (sell-back price, degradation cost); its SoC
    follows the bulk/taper closed forms in both directions, with the
    battery's own taper knee (0.65 differs from the cars' 0.8)."""
    price, ratio, Cb, rate = float(np.float32(0.3)), 0.7, 200.0, 60.0
    w = hand_workload(n_ports=2, price=price, alpha_sat=0.0, alpha_decl=0.0, c_fixed=0.01, sell_grid_ratio=ratio,
                      alpha_degrad=0.05, batt_cap_kwh=Cb, batt_rate_kw=rate, batt_tau=tau, batt_soc0=0.5, **V2G)
    o = Oracle(w)
    dt = w.params.dt_h
    socs, rews = [], []
    for _ in range(40):
        r, _ = o.step(np.array([10, 10, 20], np.int8))      # ports idle, battery +100 %
        socs.append(o.battery()["soc"][0]); rews.append(r[0])
    # charging: 60 kW while SoC <= 0.8 (0.025 per step: 13 steps from 0.5),
    # then 1 - SoC decays by 1 - rate dt / ((1 - tau) Cb) per step
    expect = []
    s = 0.5
    for k in range(40):
        s = s + rate * dt / Cb if s <= tau else 1.0 - (1.0 - s) * (1.0 - rate * dt / ((1 - tau) * Cb))
        expect.append(s)
    np.testing.assert_allclose(socs, expect, rtol=0, atol=1e-12)
    e_b = Cb * np.diff(np.concatenate([[0.5], expect]))
    np.testing.assert_allclose(rews, -price * e_b - 0.01, rtol=1e-12, atol=1e-12)
    # discharge to empty: the flipped curve, sell-back price and degradation
    socs, rews = [], []
    for _ in range(120):
        r, _ = o.step(np.array([10, 10, 0], np.int8))
        socs.append(o.battery()["soc"][0]); rews.append(r[0])
    s0 = expect[-1]
    e_b = Cb * np.diff(np.concatenate([[s0], socs]))        # < 0
    np.testing.assert_allclose(rews, -ratio * price * e_b - 0.01 - 0.05 * (-e_b), rtol=1e-12, atol=1e-12)
    d = rate * dt / Cb
    assert abs(socs[0] - (s0 - d)) < 1e-12                   # bulk: 1 - SoC <= tau
    tail = [x for x in socs if x < 1 - tau - 1e-12]
    ratios = np.array(tail[1:]) / np.array(tail[:-1])
    np.testing.assert_allclose(ratios, 1 - rate * dt / ((1 - tau) * Cb), rtol=1e-9)
    assert socs[-1] >= 0.0


def test_signed_group_and_root_limits():
    """Two cars in one group: opposite flows cancel inside the limit; two
    discharging cars beyond |I_H| are scaled down; the battery counts at the
    root."""
    w = hand_workload(n_ports=2, groups=[2], group_limit=30.0, grid_limit=25.0, alpha_sat=0.0, alpha_decl=0.0,
                      alpha_con=1.0, batt_rate_kw=60.0, **V2G)
    o = Oracle(w)
    for port in (0, 1):
        park(o, port, soc=0.5, cap=100.0, rbar=22.0, trem=100)
    # +22 and -22 kW: net 0 within both limits; battery idle
    o.step(np.array([20, 0, 10], np.int8))
    np.testing.assert_allclose(o.power(), [22.0, -22.0], rtol=1e-12)
    assert o.info()["ccon"][0] == 0.0
    # -22 and -22: |-44| > 30 in the group -> x 30/44; root |-30| > 25 -> x 25/30
    o.step(np.array([0, 0, 10], np.int8))
    np.testing.assert_allclose(o.power(), [-12.5, -12.5], rtol=1e-12)
    assert abs(o.info()["ccon"][0] - 19.0) < 1e-12           # max(44 - 30, 44 - 25)
    # battery +60 kW at the root with two cars at +22: group ok (44 > 30 -> 30),
    # root 30 + 60 = 90 > 25 -> everything x 25/90
    o.step(np.array([20, 20, 20], np.int8))
    pw, bp = o.power(), o.battery()["p"][0]
    np.testing.assert_allclose(pw, [15.0 * 25 / 90, 15.0 * 25 / 90], rtol=1e-12)
    assert abs(bp - 60.0 * 25 / 90) < 1e-12


def run_v2g_invariants(w, steps, seed):
    o = Oracle(w)
    st, p = w.stations, w.params
    po, go = st.port_off, st.group_off
    rng = np.random.default_rng(seed)
    pmax = np.asarray(p.p_max_kw)[st.port_type]
    eta = np.asarray(p.eta_port)[st.port_type]
    n_disch = 0
    for step in range(steps):
        s0, b0 = o.state(), o.battery()
        r, d = o.step(v2g_actions(rng, st))
        s1, b1 = o.state(), o.battery()
        inf, v = o.info(), o.info_v2g()
        pw = o.power()
        occ0 = s0["trem"] > 0
        assert np.all(pw[~occ0] == 0.0)
        assert np.all(np.abs(pw) <= pmax * (1 + 1e-12))
        n_disch += int((pw < 0).sum())
        for e in range(st.n_envs):
            sl = slice(po[e], po[e + 1])
            dE = pw[sl] * p.dt_h
            e_b = b1["p"][e] * p.dt_h
            assert abs(inf["enet"][e] - dE.sum()) < 1e-9
            assert abs(inf["egrid"][e] - (dE[dE > 0] / eta[sl][dE > 0]).sum()) < 1e-9
            assert abs(v["e_to"][e] - (dE[dE < 0] * eta[sl][dE < 0]).sum()) < 1e-9
            assert abs(v["e_b"][e] - e_b) < 1e-12
            assert abs(v["e_grid_net"][e] - (inf["egrid"][e] + v["e_to"][e] + e_b)) < 1e-9
            assert abs(v["degrad"][e] - (max(0.0, -e_b) - v["e_to"][e])) < 1e-12
            # profit reconstruction: the two cases of A.3
            en, gn, price = inf["enet"][e], v["e_grid_net"][e], inf["price"][e]
            pg = price if gn > 0 else p.sell_grid_ratio * price
            decl = inf["M"][e] - inf["admitted"][e]
            expect = (p.p_sell * en - pg * gn - p.c_fixed - p.alpha_sat * inf["csat"][e] - p.alpha_decl * decl
                      - p.alpha_con * inf["ccon"][e] - p.alpha_degrad * v["degrad"][e])
            assert abs(r[e] - expect) < 1e-9
            if d[e]:
                continue
            o_ = po[e]
            for g in range(go[e], go[e + 1]):
                n = st.group_size[g]
                assert abs(pw[o_:o_ + n].sum()) <= float(st.group_eta[g]) * float(st.group_limit_kw[g]) * (1 + 1e-9) + 1e-9
                o_ += n
            assert abs(pw[sl].sum() + b1["p"][e]) <= float(st.grid_eta[e]) * float(st.grid_limit_kw[e]) * (1 + 1e-9) + 1e-9
            stay = occ0[sl] & (s0["trem"][sl] > 1)
            gain = (s1["soc"][sl] - s0["soc"][sl]) * s0["cap"][sl]
            np.testing.assert_allclose(gain[stay], dE[stay], rtol=1e-9, atol=1e-9)
            np.testing.assert_allclose((b1["soc"][e] - b0["soc"][e]) * p.batt_cap_kwh, e_b, rtol=1e-9, atol=1e-9)
        assert np.all((s1["soc"] >= 0) & (s1["soc"] <= 1))
        assert np.all((b1["soc"] >= 0) & (b1["soc"] <= 1))
        assert np.all(s1["erem"] >= 0)
    assert n_disch > 0


def test_v2g_invariants_heterogeneous():
    w = I.heterogeneous(n_envs=16, seed=5)
    w.params = I.EnvParams(**{**w.params.__dict__, **V2G, "alpha_con": 0.05, "c_fixed": 0.01, "eta_port": (0.95, 0.9)})
    run_v2g_invariants(w, 150, seed=6)


def test_v2g_random_battery_level_uses_the_next_port_index():
    w = hand_workload(n_ports=3, lam=0.0, **V2G)
    o = Oracle(w)
    g = 0
    o.step(None)
    k = o.random_action(0, g, 3)
    h = (w.params.n_levels - 1) // 2
    preq = (k - h) / h * w.params.batt_rate_kw
    # from SoC 0.5 no cap binds in one step at these sizes
    assert abs(o.battery()["p"][0] - preq) < 1e-12


def test_v2g_observation_battery_features():
    w = hand_workload(n_ports=2, batt_rate_kw=40.0, **V2G)
    o = Oracle(w)
    o.set_battery(np.array([0.37]), np.array([-12.0]))
    ob = o.observe()
    assert ob.shape == (10 + 12,)
    assert ob[8] == 0.37 and ob[9] == -12.0 / 40.0
