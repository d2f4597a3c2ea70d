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
* episode returns (``RETURN_RTOL`` = 1e-4) relative to max(|return|, 1 EUR).
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


def station_step_scale(w, info):
    """Largest one-step profit magnitude of each station: selling and buying
    all energy its chargers could deliver in one step at full power."""
    st, p = w.stations, w.params
    pmax = np.asarray(p.p_max_kw, np.float64)[st.port_type]
    e_max = np.add.reduceat(pmax, st.port_off[:-1]) * p.dt_h
    eta_min = min(p.eta_port)
    return (p.p_sell + np.abs(info["price"]) / eta_min) * e_max


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
