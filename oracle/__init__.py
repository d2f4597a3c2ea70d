"""CPU oracle of the charging-station step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``chargax_oracle.c`` (plain C, FP64,
single thread) through ctypes and shares nothing with the CUDA library: the
two only see the same arrays produced by ``paper_2507_01522_b300.inputs``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chargax_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libchargax_oracle.so")

# -ffp-contract=off and no fast-math: the Poisson decision is an exact FP32
# computation that must not be fused or reassociated.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (seconds).  Returns the library path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("ep_len", C.c_int32), ("n_levels", C.c_int32),
        ("dt_h", C.c_double), ("tau", C.c_double), ("p_sell", C.c_double), ("c_fixed", C.c_double),
        ("alpha_sat", C.c_double), ("alpha_decl", C.c_double), ("alpha_con", C.c_double),
        ("soc_target", C.c_double),
        ("p_max_kw", C.c_double * 2), ("eta_port", C.c_double * 2),
        ("cap_kwh", C.c_double * 2), ("soc0", C.c_double * 2),
        ("stay_steps", C.c_int32 * 2),
        ("rbar_kw", (C.c_double * 2) * 2),
        ("v2g", C.c_int32), ("sell_grid_ratio", C.c_double), ("alpha_degrad", C.c_double),
        ("batt_cap_kwh", C.c_double), ("batt_rate_kw", C.c_double), ("batt_tau", C.c_double),
        ("batt_soc0", C.c_double),
        ("action_delta", C.c_int32), ("p_max_dis_kw", C.c_double * 2),
        ("cs_share_256", C.c_int32), ("alpha_sat1", C.c_double), ("beta_early", C.c_double),
        ("eps_cap", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, i32, u64, i64 = C.c_void_p, C.c_int32, C.c_uint64, C.c_int64
        L.orc_create.restype = vp
        L.orc_create.argtypes = [C.POINTER(_Params), i32] + [vp] * 9 + [i32, vp, i32, vp, u64]
        L.orc_destroy.argtypes = [vp]
        L.orc_reset.argtypes = [vp, vp, i32, u64]
        L.orc_step.argtypes = [vp, vp, i64, vp, vp]
        L.orc_observe.argtypes = [vp, vp]
        L.orc_get_state.argtypes = [vp] + [vp] * 13
        L.orc_set_state.argtypes = [vp] + [vp] * 13
        L.orc_get_info.argtypes = [vp] + [vp] * 9
        L.orc_get_stats.argtypes = [vp] + [vp] * 6
        L.orc_get_power.argtypes = [vp, vp]
        L.orc_set_streams.argtypes = [vp, vp, u64]
        L.orc_philox.argtypes = [vp, vp, vp]
        L.orc_poisson.restype = i32
        L.orc_poisson.argtypes = [C.c_float, C.c_uint32]
        L.orc_taper.restype = C.c_double
        L.orc_taper.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_policy_uniforms.argtypes = [vp, i32, vp]
        L.orc_obs_env_features.restype = i32
        L.orc_obs_env_features.argtypes = [vp]
        L.orc_get_battery.argtypes = [vp, vp, vp]
        L.orc_set_battery.argtypes = [vp, vp, vp]
        L.orc_get_info_v2g.argtypes = [vp, vp, vp, vp, vp]
        L.orc_obs_port_features.restype = i32
        L.orc_obs_port_features.argtypes = [vp]
        L.orc_get_due.argtypes = [vp, vp]
        L.orc_set_due.argtypes = [vp, vp]
        L.orc_get_info_cs.argtypes = [vp, vp, vp]
        L.orc_set_tree.argtypes = [vp, vp, vp, vp, vp, vp]
        L.orc_random_action.restype = i32
        L.orc_random_action.argtypes = [vp, i32, C.c_uint32, i32]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def philox(ctr, key):
    """Philox4x32-10 of one counter (4 x u32) under one key (2 x u32)."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def poisson(lam: float, word: int) -> int:
    return int(lib().orc_poisson(C.c_float(lam), C.c_uint32(word)))


def taper(soc: float, rbar: float, tau: float) -> float:
    return float(lib().orc_taper(soc, rbar, tau))


def params_struct(p) -> _Params:
    s = _Params()
    s.ep_len = int(p.ep_len); s.n_levels = int(p.n_levels)
    s.dt_h = p.dt_h; s.tau = p.tau; s.p_sell = p.p_sell; s.c_fixed = p.c_fixed
    s.alpha_sat = p.alpha_sat; s.alpha_decl = p.alpha_decl; s.alpha_con = p.alpha_con
    s.soc_target = p.soc_target
    for k in range(2):
        s.p_max_kw[k] = p.p_max_kw[k]; s.eta_port[k] = p.eta_port[k]
        s.cap_kwh[k] = p.cap_kwh[k]; s.soc0[k] = p.soc0[k]; s.stay_steps[k] = int(p.stay_steps[k])
    for k in range(2):
        s.rbar_kw[0][k] = p.rbar_ac_kw[k]; s.rbar_kw[1][k] = p.rbar_dc_kw[k]
    s.v2g = int(p.v2g); s.sell_grid_ratio = p.sell_grid_ratio; s.alpha_degrad = p.alpha_degrad
    s.batt_cap_kwh = p.batt_cap_kwh; s.batt_rate_kw = p.batt_rate_kw; s.batt_tau = p.batt_tau
    s.batt_soc0 = p.batt_soc0
    s.action_delta = int(p.action_delta)
    pd = p.p_max_kw if p.p_max_dis_kw is None else p.p_max_dis_kw
    for k in range(2):
        s.p_max_dis_kw[k] = pd[k]
    s.cs_share_256 = int(p.cs_share_256); s.alpha_sat1 = p.alpha_sat1; s.beta_early = p.beta_early
    s.eps_cap = p.eps_cap
    return s


class Oracle:
    """A batch of envs simulated by the CPU oracle (FP64)."""

    def __init__(self, workload, seed: int | None = None, streams=None):
        w = workload
        st, exo = w.stations, w.exo
        self.params = w.params
        self.E = st.n_envs
        self.P = st.total_ports
        self.port_off = st.port_off
        self._keep = [np.ascontiguousarray(a) for a in (
            st.n_ports.astype(np.int32), st.port_type.astype(np.uint8), st.n_groups.astype(np.int32),
            st.group_size.astype(np.int32), st.group_limit_kw.astype(np.float32), st.group_eta.astype(np.float32),
            st.grid_limit_kw.astype(np.float32), st.grid_eta.astype(np.float32), st.arrival_class.astype(np.int32),
            exo.price.astype(np.float32), exo.arrival_rate.astype(np.float32))]
        k = self._keep
        self._p = params_struct(w.params)
        seed = w.seed if seed is None else seed
        self.h = lib().orc_create(C.byref(self._p), self.E, *[_ptr(a) for a in k[:9]],
                                  int(exo.price.shape[0]), _ptr(k[9]), int(exo.arrival_rate.shape[0]),
                                  _ptr(k[10]), C.c_uint64(seed))
        st = w.stations
        if st.n_upper is not None:
            self._tree = [np.ascontiguousarray(a, dtype=dt) for a, dt in (
                (st.n_upper, np.int32), (st.group_parent, np.int32), (st.upper_parent, np.int32),
                (st.upper_limit_kw, np.float32), (st.upper_eta, np.float32))]
            lib().orc_set_tree(self.h, *[_ptr(a) for a in self._tree])
        if streams is not None:
            ids = np.ascontiguousarray(streams, dtype=np.uint32)
            assert ids.shape == (self.E,)
            lib().orc_set_streams(self.h, _ptr(ids), C.c_uint64(seed))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def reset(self, env_ids=None, seed: int = 0):
        if env_ids is None:
            lib().orc_reset(self.h, None, 0, C.c_uint64(seed))
        else:
            ids = np.ascontiguousarray(env_ids, dtype=np.int32)
            lib().orc_reset(self.h, _ptr(ids), len(ids), C.c_uint64(seed))

    def step(self, actions: np.ndarray | None = None, lda: int = 1):
        """One step of every env.  ``actions``: int8 per port (batch order),
        element ``port * lda``; None draws uniform levels with Philox."""
        r = np.zeros(self.E, np.float64)
        d = np.zeros(self.E, np.uint8)
        a = None if actions is None else np.ascontiguousarray(actions, dtype=np.int8)
        lib().orc_step(self.h, _ptr(a), lda, _ptr(r), _ptr(d))
        return r, d

    @property
    def obs_env_features(self) -> int:
        return int(lib().orc_obs_env_features(self.h))

    @property
    def obs_port_features(self) -> int:
        return int(lib().orc_obs_port_features(self.h))

    def observe(self) -> np.ndarray:
        o = np.zeros(self.obs_env_features * self.E + self.obs_port_features * self.P, np.float64)
        lib().orc_observe(self.h, _ptr(o))
        return o

    def battery(self) -> dict:
        d = dict(soc=np.zeros(self.E), p=np.zeros(self.E))
        lib().orc_get_battery(self.h, _ptr(d["soc"]), _ptr(d["p"]))
        return d

    def set_battery(self, soc, p):
        a = np.ascontiguousarray(soc, dtype=np.float64)
        b = np.ascontiguousarray(p, dtype=np.float64)
        lib().orc_set_battery(self.h, _ptr(a), _ptr(b))

    def due(self) -> np.ndarray:
        """Delta t_remain of charge-sensitive cars per port (0 elsewhere)."""
        d = np.zeros(self.P, np.int32)
        lib().orc_get_due(self.h, _ptr(d))
        return d

    def set_due(self, due):
        a = np.ascontiguousarray(due, dtype=np.int32)
        lib().orc_set_due(self.h, _ptr(a))

    def info_cs(self) -> dict:
        d = dict(csat1=np.zeros(self.E), margin=np.zeros(self.E))
        lib().orc_get_info_cs(self.h, _ptr(d["csat1"]), _ptr(d["margin"]))
        return d

    def info_v2g(self) -> dict:
        d = dict(e_to=np.zeros(self.E), e_b=np.zeros(self.E), degrad=np.zeros(self.E), e_grid_net=np.zeros(self.E))
        lib().orc_get_info_v2g(self.h, *[_ptr(d[k]) for k in ("e_to", "e_b", "degrad", "e_grid_net")])
        return d

    def state(self) -> dict:
        P, E = self.P, self.E
        s = dict(soc=np.zeros(P), erem=np.zeros(P), cap=np.zeros(P), rbar=np.zeros(P), p=np.zeros(P),
                 trem=np.zeros(P, np.int32), tod=np.zeros(E, np.int32), day=np.zeros(E, np.int32),
                 gstep=np.zeros(E, np.uint32), ncar=np.zeros(E, np.uint32), key0=np.zeros(E, np.uint32),
                 key1=np.zeros(E, np.uint32),
                 ep_ret=np.zeros(E))
        lib().orc_get_state(self.h, *[_ptr(s[k]) for k in STATE_KEYS])
        return s

    def set_state(self, s: dict):
        conv = dict(soc=np.float64, erem=np.float64, cap=np.float64, rbar=np.float64, p=np.float64,
                    trem=np.int32, tod=np.int32, day=np.int32, gstep=np.uint32, ncar=np.uint32, key0=np.uint32,
                    key1=np.uint32, ep_ret=np.float64)
        arrs = [np.ascontiguousarray(s[k], dtype=conv[k]) for k in STATE_KEYS]
        lib().orc_set_state(self.h, *[_ptr(a) for a in arrs])

    def info(self) -> dict:
        E = self.E
        d = dict(M=np.zeros(E, np.int32), admitted=np.zeros(E, np.int32), departed=np.zeros(E, np.int32),
                 csat=np.zeros(E), ccon=np.zeros(E), enet=np.zeros(E), egrid=np.zeros(E), price=np.zeros(E),
                 req_sum=np.zeros(E))
        lib().orc_get_info(self.h, *[_ptr(d[k]) for k in
                                     ("M", "admitted", "departed", "csat", "ccon", "enet", "egrid", "price", "req_sum")])
        return d

    def stats(self) -> dict:
        E = self.E
        d = dict(arrived=np.zeros(E), rejected=np.zeros(E), missing=np.zeros(E), charged=np.zeros(E),
                 n_episodes=np.zeros(E, np.uint32), last_ret=np.zeros(E))
        lib().orc_get_stats(self.h, *[_ptr(d[k]) for k in
                                      ("arrived", "rejected", "missing", "charged", "n_episodes", "last_ret")])
        return d

    def power(self) -> np.ndarray:
        p = np.zeros(self.P)
        lib().orc_get_power(self.h, _ptr(p))
        return p

    def random_action(self, env: int, gstep: int, port: int) -> int:
        return int(lib().orc_random_action(self.h, env, gstep, port))

    def policy_uniforms(self, n_ports: int) -> np.ndarray:
        """[E, n_ports] uniforms of the policy's next action samples (every
        env must have n_ports chargers)."""
        u = np.zeros((self.E, n_ports))
        lib().orc_policy_uniforms(self.h, n_ports, _ptr(u))
        return u


STATE_KEYS = ("soc", "erem", "cap", "rbar", "p", "trem", "tod", "day", "gstep", "ncar", "key0", "key1", "ep_ret")
