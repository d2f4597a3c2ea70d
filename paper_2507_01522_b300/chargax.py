"""Python binding of ``libchargax_b300.so`` (the C interface in
``include/chargax_b300.h``).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  Device buffers are torch CUDA tensors (their ``data_ptr()`` is
passed), host buffers numpy arrays.  If the library has not been built the
import of this module fails; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchargax_b300.so")

CHX_OK, CHX_EINVAL, CHX_ENOMEM, CHX_ECUDA, CHX_ETIMEOUT, CHX_EFAULT = 0, -1, -2, -3, -4, -5

# every symbol the header declares (checked by the CPU tests)
EXPORTS = (
    "chx_create", "chx_destroy", "chx_last_error", "chx_n_envs", "chx_n_ports_total", "chx_port_offsets",
    "chx_obs_size", "chx_reset", "chx_step", "chx_step_n", "chx_rollout", "chx_rollout_host", "chx_rollout_host_actions",
    "chx_rollout_host_levels4", "chx_step_host",
    "chx_autotune", "chx_set_launch", "chx_observe", "chx_get_state", "chx_set_state", "chx_stats", "chx_save",
    "chx_load", "chx_check", "chx_rollout_noalloc", "chx_policy_load", "chx_policy_act", "chx_policy_rollout",
    "chx_get_battery", "chx_set_battery", "chx_get_due", "chx_set_due", "chx_selftest_wait",
    "chx_srv_start", "chx_srv_stop", "chx_srv_admit", "chx_srv_evict", "chx_srv_submit", "chx_srv_wait",
    "chx_srv_test", "chx_srv_stats", "chx_srv_simulate",
)

CHX_SRV_STEP, CHX_SRV_RESET = 0, 1
CHX_ROLLOUT_FUSED, CHX_ROLLOUT_SPLIT = 0, 1


class ChxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"chargax_b300 error {code}: {msg}")
        self.code = code


class _Params(C.Structure):
    _fields_ = [
        ("ep_len", C.c_int32), ("n_levels", C.c_int32),
        ("dt_h", C.c_float), ("tau", C.c_float), ("p_sell", C.c_float), ("c_fixed", C.c_float),
        ("alpha_sat", C.c_float), ("alpha_decl", C.c_float), ("alpha_con", C.c_float), ("soc_target", C.c_float),
        ("p_max_kw", C.c_float * 2), ("eta_port", C.c_float * 2), ("cap_kwh", C.c_float * 2),
        ("soc0", C.c_float * 2), ("stay_steps", C.c_int32 * 2), ("rbar_kw", (C.c_float * 2) * 2),
        ("v2g", C.c_int32), ("sell_grid_ratio", C.c_float), ("alpha_degrad", C.c_float),
        ("batt_cap_kwh", C.c_float), ("batt_rate_kw", C.c_float), ("batt_tau", C.c_float),
        ("batt_soc0", C.c_float),
        ("action_delta", C.c_int32), ("p_max_dis_kw", C.c_float * 2),
        ("cs_share_256", C.c_int32), ("alpha_sat1", C.c_float), ("beta_early", C.c_float), ("eps_cap", C.c_float),
    ]


class _Stations(C.Structure):
    _fields_ = [
        ("n_envs", C.c_int32), ("h_n_ports", C.c_void_p), ("h_port_type", C.c_void_p), ("h_n_groups", C.c_void_p),
        ("h_group_size", C.c_void_p), ("h_group_limit_kw", C.c_void_p), ("h_group_eta", C.c_void_p),
        ("h_grid_limit_kw", C.c_void_p), ("h_grid_eta", C.c_void_p), ("h_arrival_class", C.c_void_p),
        ("h_n_upper", C.c_void_p), ("h_group_parent", C.c_void_p), ("h_upper_parent", C.c_void_p),
        ("h_upper_limit_kw", C.c_void_p), ("h_upper_eta", C.c_void_p),
    ]


class _Exo(C.Structure):
    _fields_ = [("n_days", C.c_int32), ("h_price", C.c_void_p), ("n_arrival_classes", C.c_int32),
                ("h_arrival_rate", C.c_void_p)]


class _SrvCfg(C.Structure):
    _fields_ = [("params", _Params), ("exo", _Exo), ("class_capacity", C.c_int32 * 5),
                ("hbm_budget_bytes", C.c_double), ("max_tick_envs", C.c_int32), ("n_streams", C.c_int32),
                ("max_tick_obs_floats", C.c_int64)]


class _SrvReq(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_envs", C.c_int32), ("h_env_ids", C.c_void_p), ("h_actions", C.c_void_p),
                ("h_reward", C.c_void_p), ("h_done", C.c_void_p), ("h_obs", C.c_void_p), ("seed", C.c_uint64)]


class _SrvStats(C.Structure):
    _fields_ = [("n_ticks", C.c_int64), ("n_requests", C.c_int64), ("env_steps", C.c_int64),
                ("env_resets", C.c_int64), ("resident", C.c_int32), ("used_bytes", C.c_double),
                ("budget_bytes", C.c_double), ("device_busy_ms", C.c_double), ("elapsed_ms", C.c_double),
                ("host_submit_ms", C.c_double), ("host_scan_ms", C.c_double), ("host_pack_ms", C.c_double),
                ("host_launch_ms", C.c_double),
                ("host_complete_ms", C.c_double), ("n_scans", C.c_int64)]


class _SimCfg(C.Structure):
    _fields_ = [("n_actors", C.c_int32), ("envs_per_actor", C.c_int32), ("n_threads", C.c_int32),
                ("reset_every", C.c_int32), ("mean_think_us", C.c_double), ("warmup_s", C.c_double),
                ("duration_s", C.c_double), ("seed", C.c_uint64)]


class _SimRes(C.Structure):
    _fields_ = [("n_requests", C.c_int64), ("env_steps", C.c_int64), ("seconds", C.c_double),
                ("env_steps_per_s", C.c_double), ("p50_us", C.c_double), ("p90_us", C.c_double),
                ("p99_us", C.c_double), ("max_us", C.c_double), ("mean_us", C.c_double),
                ("mean_tick_envs", C.c_double), ("device_busy_frac", C.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2507_01522_b300.build`")
    L = C.CDLL(path)
    vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    sig = {
        "chx_create": [vp, vp, vp, u64, vp], "chx_destroy": [vp], "chx_n_envs": [vp, vp],
        "chx_n_ports_total": [vp, vp], "chx_port_offsets": [vp, vp], "chx_obs_size": [vp, vp],
        "chx_reset": [vp, vp, i32, u64, vp], "chx_step": [vp, vp, i64, vp, vp, vp],
        "chx_step_n": [vp, i32, vp, i64, vp, vp, i64, vp, vp], "chx_rollout": [vp, i32, vp, vp, vp, vp],
        "chx_rollout_host": [vp, i32, vp, vp, vp, vp], "chx_step_host": [vp, vp, vp, vp, vp, vp],
        "chx_rollout_host_actions": [vp, i32, vp, vp, vp, vp, vp], "chx_rollout_host_levels4": [vp, i32, vp, vp, vp, vp, vp],
        "chx_autotune": [vp, i32, vp, vp], "chx_set_launch": [vp, i32, i32], "chx_observe": [vp, vp, vp],
        "chx_get_state": [vp] + [vp] * 13, "chx_set_state": [vp] + [vp] * 13, "chx_stats": [vp] + [vp] * 6,
        "chx_save": [vp, vp, vp], "chx_load": [vp, vp, C.c_size_t], "chx_check": [vp, vp],
        "chx_rollout_noalloc": [vp, i32, vp, vp, vp, vp],
        "chx_policy_load": [vp, i32, vp, vp, vp, vp, vp, vp], "chx_policy_act": [vp, vp, vp, vp, vp],
        "chx_policy_rollout": [vp, i32, vp, vp, vp, vp, vp, i32, vp],
        "chx_get_battery": [vp, vp, vp], "chx_set_battery": [vp, vp, vp],
        "chx_get_due": [vp, vp], "chx_set_due": [vp, vp], "chx_selftest_wait": [vp, vp],
        "chx_srv_start": [vp, vp], "chx_srv_stop": [vp], "chx_srv_admit": [vp, vp, u64, vp],
        "chx_srv_evict": [vp, vp, i32], "chx_srv_submit": [vp, vp, vp], "chx_srv_wait": [vp, u64, i64, vp],
        "chx_srv_test": [vp, u64, vp, vp], "chx_srv_stats": [vp, vp], "chx_srv_simulate": [vp, vp, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.chx_last_error.restype = C.c_char_p
    L.chx_last_error.argtypes = []
    _lib = L
    return L


def _check(rc):
    if rc != CHX_OK:
        raise ChxError(rc, _lib.chx_last_error().decode())


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dev_ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def params_struct(p: "_inputs.EnvParams") -> _Params:
    s = _Params()
    s.ep_len = int(p.ep_len); s.n_levels = int(p.n_levels)
    s.dt_h = p.dt_h; s.tau = p.tau; s.p_sell = p.p_sell; s.c_fixed = p.c_fixed
    s.alpha_sat = p.alpha_sat; s.alpha_decl = p.alpha_decl; s.alpha_con = p.alpha_con; s.soc_target = p.soc_target
    for k in range(2):
        s.p_max_kw[k] = p.p_max_kw[k]; s.eta_port[k] = p.eta_port[k]; s.cap_kwh[k] = p.cap_kwh[k]
        s.soc0[k] = p.soc0[k]; s.stay_steps[k] = int(p.stay_steps[k])
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


STATE_FIELDS = (("soc", np.float32, "P"), ("erem", np.float32, "P"), ("cap", np.float32, "P"),
                ("rbar", np.float32, "P"), ("p", np.float32, "P"), ("trem", np.uint8, "P"),
                ("tod", np.int32, "E"), ("day", np.int32, "E"), ("gstep", np.uint32, "E"), ("ncar", np.uint32, "E"),
                ("key0", np.uint32, "E"), ("key1", np.uint32, "E"), ("ep_ret", np.float32, "E"))


class Batch:
    """A batch of stations on the current CUDA device (one chx_handle)."""

    def __init__(self, workload: "_inputs.Workload", seed: int | None = None):
        L = load_library()
        st, exo = workload.stations, workload.exo
        self.workload = workload
        self._keep = [np.ascontiguousarray(a) for a in (
            st.n_ports.astype(np.int32), st.port_type.astype(np.uint8), st.n_groups.astype(np.int32),
            st.group_size.astype(np.int32), st.group_limit_kw.astype(np.float32), st.group_eta.astype(np.float32),
            st.grid_limit_kw.astype(np.float32), st.grid_eta.astype(np.float32), st.arrival_class.astype(np.int32),
            exo.price.astype(np.float32), exo.arrival_rate.astype(np.float32))]
        k = self._keep
        s = _Stations(st.n_envs, *[_np_ptr(a) for a in k[:9]])
        if st.n_upper is not None:
            self._tree = [np.ascontiguousarray(a, dtype=dt) for a, dt in (
                (st.n_upper, np.int32), (st.group_parent, np.int32), (st.upper_parent, np.int32),
                (st.upper_limit_kw, np.float32), (st.upper_eta, np.float32))]
            (s.h_n_upper, s.h_group_parent, s.h_upper_parent, s.h_upper_limit_kw,
             s.h_upper_eta) = [_np_ptr(a) for a in self._tree]
        x = _Exo(int(exo.price.shape[0]), _np_ptr(k[9]), int(exo.arrival_rate.shape[0]), _np_ptr(k[10]))
        self._p = params_struct(workload.params)
        h = C.c_void_p()
        seed = workload.seed if seed is None else seed
        _check(L.chx_create(C.byref(s), C.byref(self._p), C.byref(x), C.c_uint64(seed), C.byref(h)))
        self.h = h
        n = C.c_int32(); P = C.c_int64(); O = C.c_int64()
        _check(L.chx_n_envs(h, C.byref(n)))
        _check(L.chx_n_ports_total(h, C.byref(P)))
        _check(L.chx_obs_size(h, C.byref(O)))
        self.E, self.P, self.obs_size = n.value, P.value, O.value
        self.port_off = np.zeros(self.E + 1, np.int64)
        _check(L.chx_port_offsets(h, _np_ptr(self.port_off)))

    def close(self):
        if getattr(self, "h", None):
            _lib.chx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- stepping -------------------------------------------------------
    def reset(self, env_ids=None, seed: int = 0, stream=None):
        n = 0 if env_ids is None else int(env_ids.numel())
        if env_ids is not None and n == 0:       # an empty list (its pointer may be NULL, which means "all")
            return
        _check(_lib.chx_reset(self.h, _dev_ptr(env_ids), n, C.c_uint64(seed), _stream_ptr(stream)))

    def step(self, actions=None, reward=None, done=None, lda: int = 1, stream=None):
        _check(_lib.chx_step(self.h, _dev_ptr(actions), lda, _dev_ptr(reward), _dev_ptr(done), _stream_ptr(stream)))

    def step_n(self, k_steps: int, actions=None, reward=None, done=None, lda: int = 0, ld_out: int = 0, obs=None,
               stream=None):
        _check(_lib.chx_step_n(self.h, k_steps, _dev_ptr(actions), lda or k_steps, _dev_ptr(reward), _dev_ptr(done),
                               ld_out or k_steps, _dev_ptr(obs), _stream_ptr(stream)))

    def rollout(self, n_steps: int, reward=None, done=None, obs=None, stream=None):
        _check(_lib.chx_rollout(self.h, n_steps, _dev_ptr(reward), _dev_ptr(done), _dev_ptr(obs), _stream_ptr(stream)))

    def rollout_noalloc(self, n_steps: int, reward=None, done=None, obs=None, stream=None):
        """chx_rollout_noalloc: the rollout for callers that cannot allocate
        device memory during the call (scratch in a static device array)."""
        _check(_lib.chx_rollout_noalloc(self.h, n_steps, _dev_ptr(reward), _dev_ptr(done), _dev_ptr(obs),
                                        _stream_ptr(stream)))

    def rollout_host(self, n_steps: int, reward=None, done=None, obs=None, stream=None):
        _check(_lib.chx_rollout_host(self.h, n_steps, _np_ptr(reward), _np_ptr(done), _np_ptr(obs),
                                     _stream_ptr(stream)))

    def rollout_host_actions(self, n_steps: int, actions, reward=None, done=None, obs=None, stream=None):
        """chx_rollout_host_actions: host levels [n_steps][n_act] int8 in, host
        rewards/done flags [n_steps][n_envs] and the final observation out."""
        _check(_lib.chx_rollout_host_actions(self.h, n_steps, _np_ptr(actions), _np_ptr(reward), _np_ptr(done),
                                             _np_ptr(obs), _stream_ptr(stream)))

    def rollout_host_levels4(self, n_steps: int, levels4, reward=None, done=None, obs=None, stream=None):
        """chx_rollout_host_levels4: host levels packed two per byte
        ([n_steps][ceil(n_act / 2)] uint8, see pack_levels4) in, outputs as
        rollout_host_actions."""
        _check(_lib.chx_rollout_host_levels4(self.h, n_steps, _np_ptr(levels4), _np_ptr(reward), _np_ptr(done),
                                             _np_ptr(obs), _stream_ptr(stream)))

    def step_host(self, actions=None, reward=None, done=None, obs=None, stream=None):
        _check(_lib.chx_step_host(self.h, _np_ptr(actions), _np_ptr(reward), _np_ptr(done), _np_ptr(obs),
                                  _stream_ptr(stream)))

    def observe(self, obs, stream=None):
        _check(_lib.chx_observe(self.h, _dev_ptr(obs), _stream_ptr(stream)))

    def autotune(self, n_steps: int):
        k = C.c_int32(); w = C.c_int32()
        _check(_lib.chx_autotune(self.h, n_steps, C.byref(k), C.byref(w)))
        return k.value, w.value

    def set_launch(self, steps_per_launch: int = 0, warps_per_block: int = 0):
        _check(_lib.chx_set_launch(self.h, steps_per_launch, warps_per_block))

    def check(self, stream=None):
        _check(_lib.chx_check(self.h, _stream_ptr(stream)))

    def selftest_wait(self):
        """chx_selftest_wait: (gave_up, cycles waited / 2^20)."""
        res = np.zeros(2, np.int32)
        _check(_lib.chx_selftest_wait(self.h, _np_ptr(res)))
        return bool(res[0]), int(res[1])

    # ---- state ----------------------------------------------------------
    def get_state(self) -> dict:
        out = {name: np.zeros(self.P if kind == "P" else self.E, dt) for name, dt, kind in STATE_FIELDS}
        _check(_lib.chx_get_state(self.h, *[_np_ptr(out[n]) for n, _, _ in STATE_FIELDS]))
        return out

    def set_state(self, s: dict):
        arrs = [None if s.get(n) is None else np.ascontiguousarray(s[n], dtype=dt) for n, dt, _ in STATE_FIELDS]
        _check(_lib.chx_set_state(self.h, *[_np_ptr(a) for a in arrs]))

    def battery(self) -> dict:
        d = dict(soc=np.zeros(self.E, np.float32), p=np.zeros(self.E, np.float32))
        _check(_lib.chx_get_battery(self.h, _np_ptr(d["soc"]), _np_ptr(d["p"])))
        return d

    def set_battery(self, soc=None, p=None):
        a = None if soc is None else np.ascontiguousarray(soc, dtype=np.float32)
        b = None if p is None else np.ascontiguousarray(p, dtype=np.float32)
        _check(_lib.chx_set_battery(self.h, _np_ptr(a), _np_ptr(b)))

    def due(self) -> np.ndarray:
        """Delta t_remain of charge-sensitive cars per charger (batch order)."""
        d = np.zeros(self.P, np.int16)
        _check(_lib.chx_get_due(self.h, _np_ptr(d)))
        return d

    def set_due(self, due):
        a = np.ascontiguousarray(due, dtype=np.int16)
        _check(_lib.chx_set_due(self.h, _np_ptr(a)))

    @property
    def n_actions(self) -> int:
        """Actions per step: one per charger, plus one battery level per
        station in V2G mode."""
        return self.P + (self.E if self.workload.params.v2g else 0)

    def stats(self) -> dict:
        E = self.E
        d = dict(arrived=np.zeros(E, np.uint32), rejected=np.zeros(E, np.uint32), missing=np.zeros(E, np.float32),
                 charged=np.zeros(E, np.float32), n_episodes=np.zeros(E, np.uint32), last_ret=np.zeros(E, np.float32))
        _check(_lib.chx_stats(self.h, *[_np_ptr(d[k]) for k in
                                        ("arrived", "rejected", "missing", "charged", "n_episodes", "last_ret")]))
        return d

    def save(self) -> bytes:
        n = C.c_size_t()
        _check(_lib.chx_save(self.h, None, C.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        _check(_lib.chx_save(self.h, _np_ptr(buf), C.byref(n)))
        return buf.tobytes()

    def load(self, blob: bytes):
        buf = np.frombuffer(blob, np.uint8).copy()
        _check(_lib.chx_load(self.h, _np_ptr(buf), len(blob)))

    # ---- on-device policy -----------------------------------------------
    def policy_load(self, w1, b1, w2, b2, w3, b3):
        """chx_policy_load.  Weights are float arrays whose values are BF16
        numbers (their top 16 bits are passed); shapes [H][D], [H][H],
        [N * n_levels][H]; biases float32."""
        def bits(w):
            w = np.ascontiguousarray(w, dtype=np.float32)
            u = w.view(np.uint32)
            if np.any(u & 0xFFFF):
                raise ValueError("policy weights must be BF16 values")
            return np.ascontiguousarray((u >> 16).astype(np.uint16))
        ws = [bits(w1), bits(w2), bits(w3)]
        bs = [np.ascontiguousarray(b, dtype=np.float32) for b in (b1, b2, b3)]
        self._policy_keep = ws + bs
        _check(_lib.chx_policy_load(self.h, int(np.shape(w1)[0]), _np_ptr(ws[0]), _np_ptr(bs[0]), _np_ptr(ws[1]),
                                    _np_ptr(bs[1]), _np_ptr(ws[2]), _np_ptr(bs[2])))

    def policy_act(self, obs, actions, logits=None, stream=None):
        _check(_lib.chx_policy_act(self.h, _dev_ptr(obs), _dev_ptr(actions), _dev_ptr(logits), _stream_ptr(stream)))

    def policy_rollout(self, n_steps: int, obs, actions, reward=None, done=None, logits=None, form=None,
                       stream=None):
        """chx_policy_rollout; form CHX_ROLLOUT_FUSED (default) or CHX_ROLLOUT_SPLIT."""
        form = CHX_ROLLOUT_FUSED if form is None else form
        _check(_lib.chx_policy_rollout(self.h, n_steps, _dev_ptr(obs), _dev_ptr(actions), _dev_ptr(reward),
                                       _dev_ptr(done), _dev_ptr(logits), form, _stream_ptr(stream)))


def pack_levels4(levels: np.ndarray) -> np.ndarray:
    """[n_steps][n_act] levels 0..15 -> [n_steps][ceil(n_act / 2)] uint8, two
    per byte (even slot in the low nibble), the layout of
    chx_rollout_host_levels4."""
    lv = np.asarray(levels).astype(np.uint8)
    n_steps, n_act = lv.shape
    if n_act % 2:
        lv = np.concatenate([lv, np.zeros((n_steps, 1), np.uint8)], axis=1)
    return np.ascontiguousarray(lv[:, 0::2] | (lv[:, 1::2] << 4))


def _stations_struct(st, keep):
    arrs = [np.ascontiguousarray(a) for a in (
        st.n_ports.astype(np.int32), st.port_type.astype(np.uint8), st.n_groups.astype(np.int32),
        st.group_size.astype(np.int32), st.group_limit_kw.astype(np.float32), st.group_eta.astype(np.float32),
        st.grid_limit_kw.astype(np.float32), st.grid_eta.astype(np.float32), st.arrival_class.astype(np.int32))]
    keep.extend(arrs)
    return _Stations(st.n_envs, *[_np_ptr(a) for a in arrs])


class Server:
    """The serving loop (chx_srv_*): a pool of device-resident stations stepped
    by requests with continuous batching.  Host numpy buffers throughout."""

    def __init__(self, params, exo, class_capacity, hbm_budget_bytes=150e9, max_tick_envs=65536, n_streams=2,
                 max_tick_obs_floats=0):
        L = load_library()
        self._keep = [np.ascontiguousarray(exo.price, dtype=np.float32),
                      np.ascontiguousarray(exo.arrival_rate, dtype=np.float32)]
        cfg = _SrvCfg()
        cfg.params = params_struct(params)
        cfg.exo = _Exo(int(exo.price.shape[0]), _np_ptr(self._keep[0]), int(exo.arrival_rate.shape[0]),
                       _np_ptr(self._keep[1]))
        for c in range(5):
            cfg.class_capacity[c] = int(class_capacity[c])
        cfg.hbm_budget_bytes = float(hbm_budget_bytes)
        cfg.max_tick_envs = int(max_tick_envs)
        cfg.n_streams = int(n_streams)
        cfg.max_tick_obs_floats = int(max_tick_obs_floats)
        self._cfg = cfg
        h = C.c_void_p()
        _check(L.chx_srv_start(C.byref(cfg), C.byref(h)))
        self.h = h
        self.params = params
        self._inflight = {}

    def stop(self):
        if getattr(self, "h", None):
            _lib.chx_srv_stop(self.h)
            self.h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass

    def admit(self, stations, seed: int = 0) -> np.ndarray:
        keep = []
        s = _stations_struct(stations, keep)
        ids = np.zeros(stations.n_envs, np.int32)
        _check(_lib.chx_srv_admit(self.h, C.byref(s), C.c_uint64(seed), _np_ptr(ids)))
        return ids

    def evict(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        _check(_lib.chx_srv_evict(self.h, _np_ptr(ids), len(ids)))

    def submit(self, env_ids, kind=CHX_SRV_STEP, actions=None, reward=None, done=None, obs=None, seed: int = 0):
        """Queue a request; the output arrays are kept alive here until the
        ticket is seen complete by wait() or test()."""
        ids = np.ascontiguousarray(env_ids, dtype=np.int32)
        acts = None if actions is None else np.ascontiguousarray(actions, dtype=np.int8)
        r = _SrvReq(kind, len(ids), _np_ptr(ids), _np_ptr(acts), _np_ptr(reward), _np_ptr(done), _np_ptr(obs),
                    C.c_uint64(seed))
        t = C.c_uint64()
        _check(_lib.chx_srv_submit(self.h, C.byref(r), C.byref(t)))
        self._inflight[t.value] = (ids, acts, reward, done, obs)
        return t.value

    def wait(self, ticket: int, timeout_us: int = 30_000_000) -> int:
        lat = C.c_int64()
        rc = _lib.chx_srv_wait(self.h, C.c_uint64(ticket), timeout_us, C.byref(lat))
        if rc != CHX_ETIMEOUT:
            self._inflight.pop(ticket, None)
        _check(rc)
        return lat.value

    def test(self, ticket: int):
        d = C.c_int32()
        lat = C.c_int64()
        rc = _lib.chx_srv_test(self.h, C.c_uint64(ticket), C.byref(d), C.byref(lat))
        if d.value:
            self._inflight.pop(ticket, None)
        _check(rc)
        return bool(d.value), lat.value

    def stats(self) -> dict:
        st = _SrvStats()
        _check(_lib.chx_srv_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in _SrvStats._fields_}

    def simulate(self, station_ids, n_actors, envs_per_actor, mean_think_us, duration_s, warmup_s=0.5,
                 n_threads=8, reset_every=0, seed=0) -> dict:
        ids = np.ascontiguousarray(station_ids, dtype=np.int32)
        assert len(ids) >= n_actors * envs_per_actor
        c = _SimCfg(n_actors, envs_per_actor, n_threads, reset_every, mean_think_us, warmup_s, duration_s, seed)
        r = _SimRes()
        _check(_lib.chx_srv_simulate(self.h, C.byref(c), _np_ptr(ids), C.byref(r)))
        return {k: getattr(r, k) for k, _ in _SimRes._fields_}
