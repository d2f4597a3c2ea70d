"""Pins of the oracle's Delta-current action form (A.2 "Apply Actions": the
new current is the last one plus the action, then clipped) and of the
discharge maximum I_max<- of the V2G clip, against what the paper and
arithmetic fix: arithmetic-series ramps of a held increment (cars and the
station battery, through the two-case profit), the reduction of the Delta
form to the absolute form wherever no cap binds, the clip at 0 from below
without V2G, the zero power an arriving car starts from, and linear
discharge at the port's discharge maximum."""
import numpy as np
import pytest

from oracle import Oracle

from test_oracle_pins import hand_workload, park


def test_delta_ramp_is_an_arithmetic_series():
    """Charge-only Delta form, 21 levels on a 22 kW charger: level 11 adds
    2.2 kW per step, so the power ramps t x 2.2 until the car's 20 kW rate
    holds it; SoC follows the sum 2.2 n(n+1)/2 dt / C, then grows linearly.
    Level 10 holds the power; level 0 (-22 kW) clips at 0; level 20 (+22)
    from 0 climbs back to the car's rate."""
    w = hand_workload(n_ports=1, n_levels=21, action_delta=1, alpha_sat=0.0, alpha_decl=0.0)
    o = Oracle(w)
    C, soc0, dt, d = 100.0, 0.1, w.params.dt_h, 2.2
    park(o, 0, soc=soc0, cap=C, rbar=20.0, trem=200)
    pw, soc = [], []
    for _ in range(15):
        o.step(np.array([11], np.int8))
        s = o.state()
        pw.append(s["p"][0]); soc.append(s["soc"][0])
    np.testing.assert_allclose(pw[:9], d * np.arange(1, 10), rtol=1e-12)
    np.testing.assert_allclose(pw[9:], 20.0, rtol=0, atol=0)
    np.testing.assert_allclose(soc[8], soc0 + d * 45 * dt / C, rtol=1e-12)
    np.testing.assert_allclose(soc[14], soc0 + (d * 45 + 6 * 20.0) * dt / C, rtol=1e-12)
    o.step(np.array([10], np.int8))
    assert o.state()["p"][0] == 20.0
    o.step(np.array([0], np.int8))
    s = o.state()
    assert s["p"][0] == 0.0
    soc_now = s["soc"][0]
    o.step(np.array([20], np.int8))
    s = o.state()
    assert s["p"][0] == 20.0
    np.testing.assert_allclose(s["soc"][0], soc_now + 20.0 * dt / C, rtol=1e-12)


def test_delta_reduces_to_absolute_where_no_cap_binds():
    """V2G mode: a walk of absolute levels k_t and the Delta form fed the
    increments k_t - k_(t-1) + h give the same trajectory while no cap binds
    (large cars with rates above the charger maximum, mid SoC, the battery
    inside its bulk ranges)."""
    kw = dict(n_ports=2, n_levels=21, v2g=1, alpha_sat=0.0, alpha_decl=0.0, c_fixed=0.01,
              sell_grid_ratio=0.8, alpha_degrad=0.03, batt_cap_kwh=2000.0, batt_rate_kw=60.0, batt_soc0=0.5)
    wa = hand_workload(**kw)
    wd = hand_workload(action_delta=1, **kw)
    oa, od = Oracle(wa), Oracle(wd)
    for o in (oa, od):
        for port in (0, 1):
            park(o, port, soc=0.5, cap=1000.0, rbar=200.0, trem=250, erem=500.0)
    rng = np.random.default_rng(11)
    h = 10
    k = np.full(3, h)
    for step in range(60):
        k_new = np.clip(k + rng.integers(-3, 4, 3), 0, 20)
        ra, _ = oa.step(k_new.astype(np.int8))
        rd, _ = od.step((k_new - k + h).astype(np.int8))
        k = k_new
        np.testing.assert_allclose(rd, ra, rtol=1e-11, atol=1e-12, err_msg=f"step {step}")
        sa, sd = oa.state(), od.state()
        for key in ("soc", "erem", "p"):
            np.testing.assert_allclose(sd[key], sa[key], rtol=1e-11, atol=1e-12, err_msg=f"{key} step {step}")
        ba, bd = oa.battery(), od.battery()
        np.testing.assert_allclose(bd["p"], ba["p"], rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(bd["soc"], ba["soc"], rtol=1e-11, atol=1e-12)
    assert np.any(oa.battery()["p"] != 0.0)


def test_delta_battery_ramp_through_zero():
    """No cars, V2G Delta form: the battery's level 11 adds 6 kW per step up
    to its 60 kW rate, level 9 then takes 6 kW per step down through zero
    into discharge; SoC follows the arithmetic sums and the reward switches
    from the buy price to the sell-back price with the degradation cost."""
    price, ratio, Cb, rate, ad, cf = float(np.float32(0.3)), 0.7, 5000.0, 60.0, 0.05, 0.01
    w = hand_workload(n_ports=1, price=price, n_levels=21, v2g=1, action_delta=1, alpha_sat=0.0, alpha_decl=0.0,
                      c_fixed=cf, sell_grid_ratio=ratio, alpha_degrad=ad, batt_cap_kwh=Cb, batt_rate_kw=rate,
                      batt_soc0=0.5)
    o = Oracle(w)
    dt = w.params.dt_h
    pb, rew = [], []
    for lv in [11] * 12 + [9] * 20:
        r, _ = o.step(np.array([10, lv], np.int8))
        pb.append(o.battery()["p"][0]); rew.append(r[0])
    pb, rew = np.array(pb), np.array(rew)
    expect = np.concatenate([6.0 * np.arange(1, 11), [60.0, 60.0], 60.0 - 6.0 * np.arange(1, 21)])
    np.testing.assert_allclose(pb, expect, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(o.battery()["soc"][0], 0.5 + dt / Cb * expect.sum(), rtol=1e-12)
    e_b = expect * dt
    want = np.where(e_b > 0, -price * e_b, -ratio * price * e_b - ad * np.maximum(-e_b, 0.0)) - cf
    np.testing.assert_allclose(rew, want, rtol=1e-10, atol=1e-12)


def test_delta_arriving_car_starts_from_zero():
    """A car leaving a charger that ran at 11 kW: in the Delta form the
    charger drops to 0 at the departure and the next car's first increment
    (level 11, +2.2 kW) is its power; the absolute form keeps the departed
    car's last power on view until the next step."""
    for delta in (1, 0):
        w = hand_workload(n_ports=1, n_levels=21, action_delta=delta, lam=20.0, alpha_sat=0.0, alpha_decl=0.0)
        o = Oracle(w)
        park(o, 0, soc=0.2, cap=60.0, rbar=11.0, trem=3)
        for _ in range(3):
            o.step(np.array([20], np.int8))
        s = o.state()
        assert s["trem"][0] > 0, "a new car should have parked"
        assert s["p"][0] == (0.0 if delta else 11.0)
        if delta:
            soc0 = s["soc"][0]
            o.step(np.array([11], np.int8))
            s = o.state()
            np.testing.assert_allclose(s["p"][0], 2.2, rtol=1e-12)
            np.testing.assert_allclose(s["soc"][0], soc0 + 2.2 * w.params.dt_h / s["cap"][0], rtol=1e-12)


def test_discharge_maximum_caps_only_discharge():
    """V2G with I_max<- = (7, 50) kW below the chargers' maxima: full
    discharge runs at the discharge maximum (SoC falls linearly by
    p dt / C), full charge still reaches the car's rate above it."""
    w = hand_workload(n_ports=2, port_types=[0, 1], n_levels=21, v2g=1, p_max_dis_kw=(7.0, 50.0),
                      alpha_sat=0.0, alpha_decl=0.0)
    o = Oracle(w)
    dt = w.params.dt_h
    park(o, 0, soc=0.9, cap=50.0, rbar=20.0, trem=250, erem=5.0)
    park(o, 1, soc=0.9, cap=500.0, rbar=120.0, trem=250, erem=5.0)
    n = 10
    for _ in range(n):
        o.step(np.array([0, 0, 10], np.int8))
    s = o.state()
    np.testing.assert_allclose(s["p"], [-7.0, -50.0], rtol=1e-12)
    np.testing.assert_allclose(s["soc"], [0.9 - n * 7.0 * dt / 50.0, 0.9 - n * 50.0 * dt / 500.0], rtol=1e-12)
    park(o, 1, soc=0.3, cap=500.0, rbar=120.0, trem=250, erem=300.0)
    o.step(np.array([10, 20, 10], np.int8))
    assert o.state()["p"][1] == 120.0


@pytest.mark.parametrize("v2g", [0, 1])
def test_delta_request_capped_at_charger_maximum(v2g):
    """Delta form on a 22 kW charger with a car able to take 50 kW: level
    20 adds 22 kW per step, so the request climbs 22, 44, 66 ...; the
    charger maximum holds the power at 22 kW (only the Delta form can
    request more than the maximum), in the charge-only and the V2G clip;
    level 0 then takes 22 kW per step off, down to 0 (charge-only) or
    through 0 to the discharge maximum (V2G)."""
    w = hand_workload(n_ports=1, n_levels=21, action_delta=1, v2g=v2g, alpha_sat=0.0, alpha_decl=0.0)
    o = Oracle(w)
    park(o, 0, soc=0.5, cap=80.0, rbar=50.0, trem=100)
    for _ in range(3):                                  # V2G: the battery holds its level (10 = idle)
        o.step(np.array([20] if not v2g else [20, 10], np.int8))
        assert o.state()["p"][0] == 22.0
    for want in (0.0, 0.0) if not v2g else (0.0, -22.0, -22.0):
        o.step(np.array([0] if not v2g else [0, 10], np.int8))
        assert o.state()["p"][0] == want
