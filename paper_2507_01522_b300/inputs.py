"""Seeded synthetic workloads for the charging-station step.

This module builds the *inputs* of the simulator and nothing else: station
layouts (the architecture tree of the EV Station Layout section, restricted to
root -> groups -> ports), the exogenous time series (buy-price bank and
per-step mean arrival counts, the exogenous state space of Appendix A.1) and
the environment parameters.  It contains none of the step's arithmetic: no
clipping, charging, Poisson sampling, Philox or reward.  Both the CUDA library
and the CPU oracle consume exactly these arrays, so the two sides never share
method code.

The paper's real datasets (price profiles, car and user distributions,
arrival frequencies; Table "data-overview") are not available; the generators
below stand in with fixed synthetic distributions:

* arrivals: mean ``lambda(t) = (N/16) * 0.5 * (1 + sin(2 pi t / T))`` cars per
  step, t = step of day from midnight, N = number of ports of the station;
* prices: ``0.1 + 0.05 sin(2 pi t / T) + Normal(0, 0.01)`` EUR/kWh per step, one
  row per synthetic day (365 days);
* car/user profiles are *parameters* of uniform distributions (capacity,
  arrival SoC, stay, maximum rate per charger type) that the step samples
  itself with its counter-based generator.

All arrays are numpy, C-contiguous, in the dtypes the C interfaces expect.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

AC, DC = 0, 1
STEPS_PER_DAY = 288          # 24 h of 5-minute steps (Table "ppo-config")


@dataclasses.dataclass
class EnvParams:
    """Scalar environment parameters (Table "ppo-config" plus the readings
    that fill gaps in the paper; every field is plain data)."""
    ep_len: int = STEPS_PER_DAY
    n_levels: int = 11            # discretisation 10 -> levels 0,10%,..,100%
    dt_h: float = 5.0 / 60.0
    tau: float = 0.8
    p_sell: float = 0.75
    c_fixed: float = 0.0
    alpha_sat: float = 0.1
    alpha_decl: float = 0.5
    alpha_con: float = 0.0
    soc_target: float = 1.0
    p_max_kw: tuple = (22.0, 150.0)      # per charger type (AC, DC)
    eta_port: tuple = (0.95, 0.95)
    cap_kwh: tuple = (40.0, 100.0)       # uniform range
    soc0: tuple = (0.1, 0.5)             # uniform range
    stay_steps: tuple = (12, 96)         # inclusive integer range (1 h .. 8 h)
    rbar_ac_kw: tuple = (7.0, 22.0)
    rbar_dc_kw: tuple = (50.0, 150.0)
    # vehicle-to-grid mode (signed levels, station battery); off by default
    v2g: int = 0
    sell_grid_ratio: float = 0.8         # feed-in price = ratio x buy price
    alpha_degrad: float = 0.02           # EUR per discharged kWh
    batt_cap_kwh: float = 200.0
    batt_rate_kw: float = 60.0
    batt_tau: float = 0.8
    batt_soc0: float = 0.5
    # discharge maximum per charger type (I_max<-); None = the charging maximum
    p_max_dis_kw: tuple | None = None
    # action form: 0 = absolute levels, 1 = increments of the last applied
    # power (Delta-current form of A.2 "Apply Actions"; n_levels odd)
    action_delta: int = 0
    # charge-sensitive users (u = 1): share in 256ths, weight of c_Sat,1 per
    # step overdue, beta (weight of steps early), "demand met" threshold as a
    # fraction of the car's capacity
    cs_share_256: int = 0
    alpha_sat1: float = 0.05
    beta_early: float = 0.5
    eps_cap: float = 1e-3


@dataclasses.dataclass
class Stations:
    """Flat (CSR) description of a batch of stations.

    Ports of station e are ``port_off[e] .. port_off[e+1]-1``; its groups are
    contiguous port ranges listed in order (``group_size`` sums to the port
    count), each group node with a power limit (kW) and efficiency.

    Deeper trees (optional): ``n_upper[e]`` nodes above station e's groups,
    listed per station; ``group_parent`` [G] and ``upper_parent`` [U] index
    the station's own upper nodes, -1 = the root; every node's chargers must
    form one contiguous range (chargers in depth-first order).
    """
    n_ports: np.ndarray          # int32 [E]
    port_type: np.ndarray        # uint8 [P]
    n_groups: np.ndarray         # int32 [E]
    group_size: np.ndarray       # int32 [G]
    group_limit_kw: np.ndarray   # float32 [G]
    group_eta: np.ndarray        # float32 [G]
    grid_limit_kw: np.ndarray    # float32 [E]
    grid_eta: np.ndarray         # float32 [E]
    arrival_class: np.ndarray    # int32 [E]
    n_upper: Optional[np.ndarray] = None          # int32 [E]
    group_parent: Optional[np.ndarray] = None     # int32 [G]
    upper_parent: Optional[np.ndarray] = None     # int32 [U]
    upper_limit_kw: Optional[np.ndarray] = None   # float32 [U]
    upper_eta: Optional[np.ndarray] = None        # float32 [U]

    @property
    def n_envs(self) -> int:
        return int(self.n_ports.shape[0])

    @property
    def port_off(self) -> np.ndarray:
        off = np.zeros(self.n_envs + 1, dtype=np.int64)
        np.cumsum(self.n_ports, out=off[1:])
        return off

    @property
    def group_off(self) -> np.ndarray:
        off = np.zeros(self.n_envs + 1, dtype=np.int64)
        np.cumsum(self.n_groups, out=off[1:])
        return off

    @property
    def upper_off(self) -> np.ndarray:
        off = np.zeros(self.n_envs + 1, dtype=np.int64)
        if self.n_upper is not None:
            np.cumsum(self.n_upper, out=off[1:])
        return off

    @property
    def total_ports(self) -> int:
        return int(self.n_ports.sum())

    def subset(self, env_ids) -> "Stations":
        """Stations ``env_ids`` (in that order) as a new batch."""
        env_ids = np.asarray(env_ids, dtype=np.int64)
        po, go = self.port_off, self.group_off
        pt = np.concatenate([self.port_type[po[e]:po[e + 1]] for e in env_ids]) if len(env_ids) else np.zeros(0, np.uint8)
        gsl = [slice(go[e], go[e + 1]) for e in env_ids]
        cat = lambda a, dt: (np.concatenate([a[s] for s in gsl]) if len(env_ids) else np.zeros(0, dt))
        tree = {}
        if self.n_upper is not None:
            uo = self.upper_off
            usl = [slice(uo[e], uo[e + 1]) for e in env_ids]
            ucat = lambda a, dt: (np.concatenate([a[s] for s in usl]) if len(env_ids) else np.zeros(0, dt))
            tree = dict(n_upper=self.n_upper[env_ids].copy(), group_parent=cat(self.group_parent, np.int32),
                        upper_parent=ucat(self.upper_parent, np.int32),
                        upper_limit_kw=ucat(self.upper_limit_kw, np.float32), upper_eta=ucat(self.upper_eta, np.float32))
        return Stations(
            n_ports=self.n_ports[env_ids].copy(), port_type=pt.astype(np.uint8),
            n_groups=self.n_groups[env_ids].copy(), group_size=cat(self.group_size, np.int32),
            group_limit_kw=cat(self.group_limit_kw, np.float32), group_eta=cat(self.group_eta, np.float32),
            grid_limit_kw=self.grid_limit_kw[env_ids].copy(), grid_eta=self.grid_eta[env_ids].copy(),
            arrival_class=self.arrival_class[env_ids].copy(), **tree)


@dataclasses.dataclass
class Exo:
    """Exogenous tables: buy-price bank [D][T] and mean arrivals [C][T]."""
    price: np.ndarray            # float32 [D, T]
    arrival_rate: np.ndarray     # float32 [C, T]


@dataclasses.dataclass
class Workload:
    name: str
    params: EnvParams
    stations: Stations
    exo: Exo
    seed: int = 0


# ----------------------------------------------------------------------------
# exogenous series
# ----------------------------------------------------------------------------

def price_bank(n_days: int = 365, ep_len: int = STEPS_PER_DAY, seed: int = 0) -> np.ndarray:
    """Synthetic day-ahead buy prices: 0.1 + 0.05 sin(2 pi t/T) + N(0, 0.01)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x50]))
    t = np.arange(ep_len, dtype=np.float64)
    base = 0.1 + 0.05 * np.sin(2.0 * math.pi * t / ep_len)
    noise = rng.normal(0.0, 0.01, size=(n_days, ep_len))
    return np.ascontiguousarray((base[None, :] + noise).astype(np.float32))


def arrival_rates(port_counts, ep_len: int = STEPS_PER_DAY, base: float = 0.5) -> np.ndarray:
    """Mean cars per step for each listed station size N:
    (N/16) * base * (1 + sin(2 pi t / T)).  Row c belongs to ``port_counts[c]``."""
    t = np.arange(ep_len, dtype=np.float64)
    shape = base * (1.0 + np.sin(2.0 * math.pi * t / ep_len))
    rows = [(float(n) / 16.0) * shape for n in port_counts]
    return np.ascontiguousarray(np.asarray(rows, dtype=np.float64).astype(np.float32).reshape(len(rows), ep_len))


# ----------------------------------------------------------------------------
# station layouts
# ----------------------------------------------------------------------------

def _build(per_env: List[dict], class_of_n: Dict[int, int]) -> Stations:
    n_ports = np.array([d["n"] for d in per_env], dtype=np.int32)
    port_type = np.concatenate([np.asarray(d["types"], dtype=np.uint8) for d in per_env])
    n_groups = np.array([len(d["groups"]) for d in per_env], dtype=np.int32)
    group_size = np.concatenate([np.asarray(d["groups"], dtype=np.int32) for d in per_env])
    group_limit = np.concatenate([np.asarray(d["glim"], dtype=np.float32) for d in per_env])
    group_eta = np.concatenate([np.asarray(d.get("geta", [1.0] * len(d["groups"])), dtype=np.float32) for d in per_env])
    grid_limit = np.array([d["grid"] for d in per_env], dtype=np.float32)
    grid_eta = np.array([d.get("grid_eta", 1.0) for d in per_env], dtype=np.float32)
    arrival_class = np.array([class_of_n[d["n"]] for d in per_env], dtype=np.int32)
    return Stations(n_ports, port_type, n_groups, group_size, group_limit, group_eta,
                    grid_limit, grid_eta, arrival_class)


def uniform_stations(n_envs: int, n_ports: int, groups: List[int], group_limit_kw: float,
                     grid_limit_kw: float, port_type: int = AC) -> Stations:
    d = dict(n=n_ports, types=[port_type] * n_ports, groups=list(groups),
             glim=[group_limit_kw] * len(groups), grid=grid_limit_kw)
    return _build([d] * n_envs, {n_ports: 0})


def mixed_stations(rng: np.random.Generator, sizes: np.ndarray, p_max_kw, p_dc: float = 0.25,
                   grid_kw_per_port: float = 9.0, group_frac: float = 0.5,
                   class_sizes: Optional[List[int]] = None, group_lo: int = 4, group_hi: int = 16) -> Stations:
    """Heterogeneous stations: per port DC with probability ``p_dc`` else AC;
    sequential groups of U{group_lo..group_hi} ports (the last one takes what
    is left; a remainder below ``group_lo`` joins the previous group), each
    limited to ``group_frac`` of its ports' summed maximum power; grid limit
    ``grid_kw_per_port`` x N.  Vectorised over stations."""
    sizes = np.asarray(sizes, dtype=np.int64)
    E = len(sizes)
    if class_sizes is None:
        class_sizes = sorted(set(int(n) for n in sizes))
    class_of_n = np.full(max(class_sizes) + 1, -1, np.int64)
    class_of_n[np.asarray(class_sizes)] = np.arange(len(class_sizes))
    port_type = (rng.random(int(sizes.sum())) < p_dc).astype(np.uint8)
    # candidate group sizes, their running sums, and the groups that fit
    kmax = int(sizes.max()) // group_lo + 2
    draws = rng.integers(group_lo, group_hi + 1, size=(E, kmax))
    csum = np.cumsum(draws, axis=1)
    full = csum < sizes[:, None]                       # groups completed before the end
    k = full.sum(axis=1)                               # number of full groups
    last = sizes - np.where(k > 0, csum[np.arange(E), np.maximum(k - 1, 0)], 0)
    merge = (last < group_lo) & (k > 0)
    n_groups = np.where(merge, k, k + 1)
    cols = np.arange(kmax)[None, :]
    g = np.where(cols < k[:, None], draws, 0)
    g[np.arange(E), np.where(merge, k - 1, k)] += last   # the remainder: own group or merged
    group_size = g[cols < n_groups[:, None]].astype(np.int32)
    # group limits: fraction of the summed charger maxima of each group
    pmax = np.asarray(p_max_kw, np.float64)[port_type]
    g_start = np.concatenate([[0], np.cumsum(group_size)[:-1]])
    glim = group_frac * np.add.reduceat(pmax, g_start) if len(g_start) else np.zeros(0)
    return Stations(
        n_ports=sizes.astype(np.int32), port_type=port_type, n_groups=n_groups.astype(np.int32),
        group_size=group_size, group_limit_kw=glim.astype(np.float32),
        group_eta=np.ones(len(group_size), np.float32),
        grid_limit_kw=(grid_kw_per_port * sizes).astype(np.float32), grid_eta=np.ones(E, np.float32),
        arrival_class=class_of_n[sizes].astype(np.int32))


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def small_uniform(n_envs: int = 16, seed: int = 0) -> Workload:
    """16 stations x 16 AC chargers of 22 kW, one group, 150 kW grid."""
    p = EnvParams(p_max_kw=(22.0, 150.0))
    st = uniform_stations(n_envs, 16, [16], 150.0, 150.0)
    exo = Exo(price_bank(seed=seed), arrival_rates([16]))
    return Workload("uniform-16x16", p, st, exo, seed)


def fixed_station(n_envs: int = 4096, seed: int = 0) -> Workload:
    """4096 stations x 16 chargers in 2 groups of 8 (80 kW each), 22 kW ports,
    150 kW grid."""
    p = EnvParams(p_max_kw=(22.0, 150.0))
    st = uniform_stations(n_envs, 16, [8, 8], 80.0, 150.0)
    exo = Exo(price_bank(seed=seed), arrival_rates([16]))
    return Workload(f"fixed-{n_envs}x16", p, st, exo, seed)


def heterogeneous(n_envs: int = 65536, seed: int = 0, classes=(8, 16, 32, 64)) -> Workload:
    """Mixed batch: 25 % each of 8/16/32/64-charger stations, randomly
    interleaved; 11 kW AC / 150 kW DC ports (DC with p = 0.25); grid 9 kW per
    charger; groups of 4..16 at half their summed port maximum."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x53]))
    per = n_envs // len(classes)
    sizes = np.concatenate([np.full(per + (1 if i < n_envs % len(classes) else 0), c, np.int32)
                            for i, c in enumerate(classes)])
    rng.shuffle(sizes)
    p = EnvParams(p_max_kw=(11.0, 150.0))
    st = mixed_stations(rng, sizes, p.p_max_kw, class_sizes=list(classes))
    exo = Exo(price_bank(seed=seed), arrival_rates(list(classes)))
    return Workload(f"hetero-{n_envs}-8/16/32/64", p, st, exo, seed)


def tree_stations(rng: np.random.Generator, n_envs: int, p_max_kw=(22.0, 150.0), eta: float = 0.98) -> Stations:
    """Stations with the deeper architecture of Fig. charge-tree c: the root
    (grid) feeds one splitter per charger type, each type splitter feeds
    1..3 sub-splitters, each sub-splitter 1..3 groups of 2..6 chargers; a
    third of the stations skip the sub-splitters of the DC branch (its
    groups hang from the type splitter: a tree of uneven depth).  Limits
    take 0.75 / 0.6 / 0.5 / 0.4 of the summed charger maxima at the group /
    sub-splitter / type splitter / grid; node efficiencies ``eta``."""
    pm = np.asarray(p_max_kw, np.float64)
    n_ports, port_type, n_groups, group_size, glim, geta = [], [], [], [], [], []
    n_upper, group_parent, upper_parent, ulim, ueta, grid = [], [], [], [], [], []
    for e in range(n_envs):
        nodes = []                                        # (parent, limit) of this station's upper nodes
        n, ng, total = 0, 0, 0.0
        shallow_dc = rng.random() < 1 / 3
        for ty in (AC, DC):
            t_idx = len(nodes)
            nodes.append([-1, 0.0])
            t_sum = 0.0
            subs = [None] if (ty == DC and shallow_dc) else [len(nodes) + i for i in range(int(rng.integers(1, 4)))]
            for sidx in subs:
                if sidx is not None:
                    nodes.append([t_idx, 0.0])
                s_sum = 0.0
                for _ in range(int(rng.integers(1, 4))):
                    k = int(rng.integers(2, 7))
                    port_type.extend([ty] * k)
                    group_size.append(k)
                    glim.append(0.75 * k * pm[ty])
                    geta.append(eta)
                    group_parent.append(t_idx if sidx is None else sidx)
                    s_sum += k * pm[ty]
                    n += k
                    ng += 1
                if sidx is not None:
                    nodes[sidx][1] = 0.6 * s_sum
                t_sum += s_sum
            nodes[t_idx][1] = 0.5 * t_sum
            total += t_sum
        n_ports.append(n)
        n_groups.append(ng)
        n_upper.append(len(nodes))
        for par, lim in nodes:
            upper_parent.append(par)
            ulim.append(lim)
            ueta.append(eta)
        grid.append(0.4 * total)
    return Stations(
        n_ports=np.array(n_ports, np.int32), port_type=np.array(port_type, np.uint8),
        n_groups=np.array(n_groups, np.int32), group_size=np.array(group_size, np.int32),
        group_limit_kw=np.array(glim, np.float32), group_eta=np.array(geta, np.float32),
        grid_limit_kw=np.array(grid, np.float32), grid_eta=np.full(n_envs, eta, np.float32),
        arrival_class=np.zeros(n_envs, np.int32), n_upper=np.array(n_upper, np.int32),
        group_parent=np.array(group_parent, np.int32), upper_parent=np.array(upper_parent, np.int32),
        upper_limit_kw=np.array(ulim, np.float32), upper_eta=np.array(ueta, np.float32))


def tree_workload(n_envs: int = 256, seed: int = 0) -> Workload:
    """Stations of ``tree_stations`` (3..63 chargers), arrivals of a
    32-charger station."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x7E]))
    p = EnvParams(p_max_kw=(22.0, 150.0))
    st = tree_stations(rng, n_envs, p.p_max_kw)
    exo = Exo(price_bank(seed=seed), arrival_rates([32]))
    return Workload(f"tree-{n_envs}", p, st, exo, seed)


def v2g_variant(w: Workload, n_levels: int = 21, batt_cap_kwh: float = 150.0, batt_rate_kw: float = 60.0) -> Workload:
    """The same stations in vehicle-to-grid mode: 21 signed levels (-100 %
    .. +100 % in 10 % steps), a 150 kWh / 60 kW station battery starting
    half full, feed-in at 0.8 x the buy price, 0.02 EUR per discharged kWh."""
    p = EnvParams(**{**w.params.__dict__, "v2g": 1, "n_levels": n_levels, "batt_cap_kwh": batt_cap_kwh,
                     "batt_rate_kw": batt_rate_kw})
    return Workload(w.name + "-v2g", p, w.stations, w.exo, w.seed)


def rollout_stations(n_envs: int = 16384, seed: int = 0) -> Workload:
    """16384 stations x 32 AC chargers (22 kW) in groups of 8 at 80 kW, grid
    9 kW x 32."""
    p = EnvParams(p_max_kw=(22.0, 150.0))
    st = uniform_stations(n_envs, 32, [8, 8, 8, 8], 80.0, 9.0 * 32)
    exo = Exo(price_bank(seed=seed), arrival_rates([32]))
    return Workload(f"rollout-{n_envs}x32", p, st, exo, seed)


def log_uniform_sizes(rng: np.random.Generator, n_envs: int, lo: int = 8, hi: int = 128) -> np.ndarray:
    x = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_envs))
    return np.clip(np.rint(x), lo, hi).astype(np.int32)


def serving_pool(n_envs: int, seed: int = 0) -> Workload:
    """Stations for the serving loop: N = round(exp(U(ln 8, ln 128))) chargers,
    groups and limits as in the heterogeneous batch."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x55]))
    sizes = log_uniform_sizes(rng, n_envs)
    p = EnvParams(p_max_kw=(11.0, 150.0))
    classes = list(range(8, 129))
    st = mixed_stations(rng, sizes, p.p_max_kw, class_sizes=classes)
    exo = Exo(price_bank(seed=seed), arrival_rates(classes))
    return Workload(f"serve-{n_envs}-logU(8,128)", p, st, exo, seed)


def random_actions(rng: np.random.Generator, n_ports_total: int, n_levels: int = 11, steps: Optional[int] = None) -> np.ndarray:
    """Uniform action levels 0..n_levels-1 as int8, shape [P] or [P, steps]."""
    shape = (n_ports_total,) if steps is None else (n_ports_total, steps)
    return rng.integers(0, n_levels, size=shape, dtype=np.int64).astype(np.int8)


# ----------------------------------------------------------------------------
# policy weights (the agent's actor network, random initialisation)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class PolicyWeights:
    """A 3-layer actor obs [D] -> H -> H -> N * L logits.  Float32 arrays
    whose values are BF16 numbers (low 16 bits of each float zero)."""
    w1: np.ndarray               # [H, D]
    b1: np.ndarray               # [H]
    w2: np.ndarray               # [H, H]
    b2: np.ndarray               # [H]
    w3: np.ndarray               # [N * L, H]; row c * L + j = level j of charger c
    b3: np.ndarray               # [N * L]


def _orthogonal(rng: np.random.Generator, rows: int, cols: int, gain: float) -> np.ndarray:
    a = rng.standard_normal((max(rows, cols), min(rows, cols)))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))
    q = q if rows >= cols else q.T
    return gain * q[:rows, :cols]


def _bf16_values(x: np.ndarray) -> np.ndarray:
    """float32 copy with the low 16 bits cleared, i.e. exact BF16 values."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    return u.view(np.float32)


def policy_weights(obs_dim: int, n_ports: int, n_levels: int = 11, hidden: int = 256, seed: int = 0,
                   head_gain: float = 0.01, bias_scale: float = 0.0) -> PolicyWeights:
    """Random initialisation as PPO actors are commonly initialised:
    orthogonal matrices, gain sqrt(2) for the hidden layers and `head_gain`
    for the logits layer, zero biases; `bias_scale` > 0 draws biases from
    U(-bias_scale, bias_scale) instead (tests use it to exercise the bias
    path and to make the distributions far from uniform)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x9011C7]))
    n_out = n_ports * n_levels
    mats = [_orthogonal(rng, hidden, obs_dim, math.sqrt(2.0)), _orthogonal(rng, hidden, hidden, math.sqrt(2.0)),
            _orthogonal(rng, n_out, hidden, head_gain)]
    biases = [rng.uniform(-bias_scale, bias_scale, n) if bias_scale > 0 else np.zeros(n) for n in (hidden, hidden, n_out)]
    w1, w2, w3 = (_bf16_values(m) for m in mats)
    b1, b2, b3 = (np.asarray(b, np.float32) for b in biases)
    return PolicyWeights(w1, b1, w2, b2, w3, b3)
