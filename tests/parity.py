"""Helpers shared by the GPU parity tests: run the CUDA library and the CPU
oracle on the same seeded inputs and compare what they produce.

Tolerances (all stated here, used by every parity test):

* events are compared exactly: remaining stay of every charger (which
  encodes occupancy, arrivals, FCFS placement and departures), done flags,
  step of day, day, global step, admitted and rejected car counters;
* one step from a shared FP32 state (``STEP_RTOL`` = 1e-5): SoC, remaining
  demand, applied power relative to their own value (floor 1e-3 of the field's
  scale), the reward relative to the sum of the magnitudes of its terms (so
  cancellation between profit and penalties does not inflate it);
* trajectories run independently on both sides (``TRAJ_RTOL`` = 1e-4): the
  FP32 state is a running sum (SoC and remaining demand change by one
  rounded increment per step for up to 255 steps), so its error is bounded
  relative to the quantity it accumulates, not to its current value: SoC
  against 1, remaining demand and capacity against the car's capacity, power
  against the charger's maximum, and a step's reward against the largest
  profit the station could make in one step;
* episode returns (``RETURN_RTOL`` = 1e-4) relative to max(|return|, 1 EUR);
* a step's reward along independent trajectories (``traj_reward_scale``):
  TRAJ_RTOL relative to the sum of its terms' magnitudes, plus what the
  drift of the FP32 state can change.  The charger power is a minimum of
  terms of which three depend on the state: the taper r_bar (1 - SoC) /
  (1 - tau) (V2G: SoC r_bar / (1 - tau) when discharging), the SoC cap
  (1 - SoC) C / dt and the demand cap e_rem / dt.  A SoC that differs by
  dS moves them by at most S dS, S = max(r_bar / (1 - tau), C / dt), and
  e_rem by de moves the demand cap by de / dt; node rescaling only
  redistributes or scales such differences down.  Near SoC = 1 this is not
  small against the step's own energy: FP32 resolves SoC to 6e-8, while
  1 - SoC of a car deep in the taper is 1e-4 or less, so a tail car's
  power carries a relative error of a few percent (an FP32-stored-state
  model of the oracle shows the same).  The allowance per station is
  sum_i dt (p_sell + |p_buy| / eta_min + alpha_sat + alpha_con / eta_node)
  dP_i + alpha_sat de_i over the occupied chargers whose power can depend
  on SoC or e_rem (in or near the taper or a cap; V2G: all occupied), with
  dP_i = S_i dS_i + de_i / dt (+ the drift of the last applied power in the
  increment form), where dS_i and de_i are the state differences measured
  at the start and at the end of the launch (the larger) plus
  ``DRIFT_PER_STEP`` per step of the launch for cars that came and went
  inside it (each step rounds SoC once in the addition and once in the
  increment; the taper's feedback on SoC is contracting, factor |1 -
  r_bar dt / ((1 - tau) C)| <= 1).  Chargers in the bulk phase, away from
  every cap, get no allowance.
"""
from __future__ import annotations

import numpy as np

STEP_RTOL = 1e-5
TRAJ_RTOL = 1e-4
RETURN_RTOL = 1e-4


def reward_scale(info, params):
    """Sum of magnitudes of the reward's terms, per env (oracle record)."""
    decl = (info["M"] - info["admitted"]).astype(np.float64)
    return (abs(params.p_sell * info["enet"]) + abs(info["price"] * info["egrid"]) + abs(params.c_fixed)
            + abs(params.alpha_sat * info["csat"]) + abs(params.alpha_decl * decl)
            + abs(params.alpha_con * info["ccon"]) + 1e-6)


def assert_events_equal(gs: dict, os_: dict, where: str = ""):
    np.testing.assert_array_equal(gs["trem"].astype(np.int32), os_["trem"], err_msg=f"trem {where}")
    for k in ("tod", "day", "gstep", "ncar", "key0", "key1"):
        np.testing.assert_array_equal(gs[k].astype(np.int64), os_[k].astype(np.int64), err_msg=f"{k} {where}")


def assert_floats_close(gs: dict, os_: dict, rtol: float, where: str = "", cap_hi: float = 100.0):
    """One-step comparison: each field relative to its own value, with a
    floor of 1e-3 of the field's scale."""
    scales = dict(soc=1.0, erem=cap_hi, cap=cap_hi, rbar=150.0, p=150.0)
    for k, sc in scales.items():
        d = np.abs(gs[k].astype(np.float64) - os_[k])
        tol = rtol * np.maximum(np.abs(os_[k]), 1e-3 * sc)
        _report(k, where, d, tol, gs[k], os_[k])


def assert_traj_close(gs: dict, os_: dict, pmax: np.ndarray, rtol: float, where: str = ""):
    """Trajectory comparison: each field against the magnitude it accumulates
    (see module docstring).  ``pmax``: maximum power of every charger."""
    cap = np.maximum(np.abs(os_["cap"]), np.abs(gs["cap"].astype(np.float64)))
    scales = dict(soc=np.ones_like(cap), erem=np.maximum(cap, 1.0), cap=np.maximum(cap, 1.0),
                  rbar=pmax, p=pmax)
    for k, sc in scales.items():
        d = np.abs(gs[k].astype(np.float64) - os_[k])
        _report(k, where, d, rtol * sc, gs[k], os_[k])


def _report(k, where, d, tol, g, o):
    bad = d > tol
    if bad.any():
        i = int(np.argmax(d - tol))
        raise AssertionError(f"{k} {where}: {bad.sum()} mismatches, worst at {i}: gpu {g[i]!r} "
                             f"oracle {o[i]!r} (tol {tol[i]:.3g})")


DRIFT_PER_STEP = 3 * 2.0 ** -24


def state_drift(gs: dict | None, os_: dict | None, n: int | None = None, gb=None, ob=None) -> dict:
    """|GPU - oracle| per charger (soc, erem, p) and per station (battery
    SoC, V2G) for two states of the same chargers; zeros (n chargers) when
    the states are the same by construction (gs is None)."""
    if gs is None:
        z = np.zeros(n)
        return dict(soc=z, erem=z, p=z, bsoc=None)
    d = {k: np.abs(gs[k].astype(np.float64) - os_[k]) for k in ("soc", "erem", "p")}
    d["bsoc"] = None if gb is None else np.abs(gb["soc"].astype(np.float64) - ob["soc"])
    return d


def traj_reward_scale(w, info, o_before: dict, d0: dict, d1: dict, kk: int, b_before=None):
    """Reward scale of one step along independent trajectories (see the
    module docstring): reward_scale plus the drift allowance / TRAJ_RTOL, so
    that assert_reward_close(..., TRAJ_RTOL) allows TRAJ_RTOL x the terms'
    magnitudes plus the allowance.  o_before: the oracle's state before the
    step; d0, d1: state_drift at the launch's start and end; kk: steps of
    the launch; b_before: the oracle's battery before the step (V2G)."""
    st, p = w.stations, w.params
    pmax = np.asarray(p.p_max_kw, np.float64)[st.port_type]
    eta = np.asarray(p.eta_port, np.float64)[st.port_type]
    grow = kk * DRIFT_PER_STEP
    dS = np.maximum(d0["soc"], d1["soc"]) + grow
    cap = np.asarray(o_before["cap"], np.float64)
    de = np.maximum(d0["erem"], d1["erem"]) + grow * np.maximum(cap, 1.0)
    soc, erem = np.asarray(o_before["soc"], np.float64), np.asarray(o_before["erem"], np.float64)
    rbar = np.asarray(o_before["rbar"], np.float64)
    occ = np.asarray(o_before["trem"]) > 0
    if p.v2g:
        sens = occ
    else:
        sens = occ & ((soc >= p.tau - dS - 1e-6) | ((1.0 - soc) * cap / p.dt_h <= pmax * (1 + 1e-6))
                      | (erem / p.dt_h <= pmax * (1 + 1e-6)))
    S = np.maximum(rbar / (1.0 - p.tau), cap / p.dt_h)
    dP = np.where(sens, S * dS + de / p.dt_h, 0.0)
    if p.action_delta:
        dP = dP + np.where(occ, np.maximum(d0["p"], d1["p"]) + grow * pmax, 0.0)
    dP = np.minimum(dP, 2.0 * pmax)
    etas = [np.asarray(st.group_eta, np.float64), np.asarray(st.grid_eta, np.float64)]
    if getattr(st, "upper_eta", None) is not None and len(st.upper_eta):
        etas.append(np.asarray(st.upper_eta, np.float64))
    eta_node = min(float(e.min()) for e in etas if len(e))
    price = np.abs(np.asarray(info["price"], np.float64))
    starts = st.port_off[:-1]
    coef_env = p.p_sell + price / float(eta.min()) + p.alpha_sat + p.alpha_con / eta_node
    if p.v2g:
        coef_env = coef_env + price * p.sell_grid_ratio + p.alpha_degrad
    per_port = p.dt_h * dP
    allow = coef_env * np.add.reduceat(per_port, starts) + p.alpha_sat * np.add.reduceat(np.where(occ, de, 0.0), starts)
    if p.v2g and b_before is not None:
        db = (np.zeros(len(starts)) if d1.get("bsoc") is None else np.maximum(
            d1["bsoc"], 0.0 if d0.get("bsoc") is None else d0["bsoc"])) + grow
        Sb = max(p.batt_rate_kw / (1.0 - p.batt_tau), p.batt_cap_kwh / p.dt_h)
        allow = allow + coef_env * p.dt_h * np.minimum(Sb * db, 2.0 * p.batt_rate_kw)
    return reward_scale(info, p) + allow / TRAJ_RTOL


def charger_pmax(w):
    return np.asarray(w.params.p_max_kw, np.float64)[w.stations.port_type]


def assert_reward_close(r_gpu, r_orc, scale, rtol, where=""):
    d = np.abs(np.asarray(r_gpu, np.float64) - r_orc)
    bad = d > rtol * scale
    if bad.any():
        i = int(np.argmax(d / scale))
        raise AssertionError(f"reward {where}: {bad.sum()} mismatches, worst env {i}: gpu {r_gpu[i]!r} "
                             f"oracle {r_orc[i]!r} scale {scale[i]:.4g}")


def to_f32_state(s: dict) -> dict:
    """An oracle state rounded to what the GPU stores (FP32, u8 stays)."""
    out = {}
    for k, v in s.items():
        if k in ("soc", "erem", "cap", "rbar", "p", "ep_ret"):
            out[k] = v.astype(np.float32)
        elif k == "trem":
            out[k] = v.astype(np.uint8)
        else:
            out[k] = v.copy()
    return out


def widen(s32: dict) -> dict:
    """FP32 state -> the oracle's dtypes (exact widening)."""
    out = {}
    for k, v in s32.items():
        if k in ("soc", "erem", "cap", "rbar", "p", "ep_ret"):
            out[k] = v.astype(np.float64)
        elif k == "trem":
            out[k] = v.astype(np.int32)
        else:
            out[k] = v.copy()
    return out
