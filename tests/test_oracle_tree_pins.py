"""Pins of the oracle's deeper architecture trees (Fig. charge-tree c; Eq.
ArchConst for every subtree, proportional rescale bottom-up) against what
the paper and arithmetic fix: a hand-computed three-level station whose
result depends on processing children before parents, the constraint
penalty on requested power, a chain of nodes acting as the smallest of
their limits, node efficiencies, the reduction to the two-level tree when
the upper nodes never bind, and every node's constraint holding along
random trajectories."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2507_01522_b300 import inputs as I

from test_oracle_pins import park


def tree_station(groups, group_limit, group_parent, upper_parent, upper_limit, upper_eta=None, group_eta=None,
                 grid_limit=1e9, types=None, **pkw):
    """One station: groups of the given sizes (AC chargers unless types),
    upper nodes with parents (-1 = root)."""
    n = int(sum(groups))
    st = I.Stations(
        n_ports=np.array([n], np.int32), port_type=np.array(types or [I.AC] * n, np.uint8),
        n_groups=np.array([len(groups)], np.int32), group_size=np.array(groups, np.int32),
        group_limit_kw=np.array(group_limit, np.float32),
        group_eta=np.array(group_eta or [1.0] * len(groups), np.float32),
        grid_limit_kw=np.array([grid_limit], np.float32), grid_eta=np.ones(1, np.float32),
        arrival_class=np.zeros(1, np.int32), n_upper=np.array([len(upper_parent)], np.int32),
        group_parent=np.array(group_parent, np.int32), upper_parent=np.array(upper_parent, np.int32),
        upper_limit_kw=np.array(upper_limit, np.float32),
        upper_eta=np.array(upper_eta or [1.0] * len(upper_parent), np.float32))
    exo = I.Exo(np.full((1, 288), 0.2, np.float32), np.zeros((1, 288), np.float32))
    return I.Workload("tree-hand", I.EnvParams(**pkw), st, exo, 0)


def fill(o, n, rbar=50.0):
    for q in range(n):
        park(o, q, soc=0.2, cap=80.0, rbar=rbar, trem=100)


def test_children_before_parents():
    """Node A (30 kW) holds group g1 (20 kW, 2 chargers) and group g2 (100
    kW, 2 chargers); every charger asks 22 kW.  g1 scales to 20/44 (10 kW
    each), then A sees 20 + 44 = 64 and scales all by 30/64: 4.6875 and
    10.3125 kW.  (Parents first would give 30/88 to all, then g1 would not
    bind: 7.5 kW each.)  The penalty takes the largest requested excess:
    A's 88 - 30 = 58."""
    out = {}
    for a in (0.0, 1.0):
        w = tree_station([2, 2], [20.0, 100.0], [0, 0], [-1], [30.0], alpha_con=a, alpha_sat=0.0, alpha_decl=0.0)
        o = Oracle(w)
        fill(o, 4)
        r, _ = o.step(np.full(4, 10, np.int8))
        out[a] = (r[0], o.state()["p"].copy())
    np.testing.assert_allclose(out[0.0][1], [4.6875, 4.6875, 10.3125, 10.3125], rtol=1e-12)
    np.testing.assert_allclose(out[0.0][0] - out[1.0][0], 58.0, rtol=1e-12)


def test_uneven_depth_and_sibling_charger_group():
    """Node U (30 kW) holds group g (20 kW, 2 chargers) under it and a
    sibling group g' (100 kW, 1 charger) directly under U; a third group
    hangs from the root.  Child first: g gives 10 + 10, U scales 20 + 22 by
    30/42; the root's own group is untouched."""
    w = tree_station([2, 1, 1], [20.0, 100.0, 100.0], [0, 0, -1], [-1], [30.0])
    o = Oracle(w)
    fill(o, 4)
    o.step(np.full(4, 10, np.int8))
    np.testing.assert_allclose(o.state()["p"], [10 * 30 / 42, 10 * 30 / 42, 22 * 30 / 42, 22.0], rtol=1e-12)


@pytest.mark.parametrize("limits", [(40.0, 25.0, 60.0), (15.0, 90.0, 50.0), (100.0, 100.0, 33.0)])
def test_chain_acts_as_smallest_limit(limits):
    """root -> U1 -> U2 -> one group of 4 chargers asking 22 kW each: the
    proportional rescales compose to the smallest limit (or the demand)."""
    l1, l2, lg = limits
    w = tree_station([4], [lg], [1], [-1, 0], [l1, l2])
    o = Oracle(w)
    fill(o, 4)
    o.step(np.full(4, 10, np.int8))
    p = o.state()["p"]
    np.testing.assert_allclose(p.sum(), min(l1, l2, lg, 88.0), rtol=1e-12)
    np.testing.assert_allclose(p, p[0], rtol=1e-12)


def test_upper_node_efficiency():
    """An upper node with efficiency 0.8 and limit 50 kW passes at most
    0.8 x 50 = 40 kW to its chargers."""
    w = tree_station([2, 2], [100.0, 100.0], [0, 0], [-1], [50.0], upper_eta=[0.8])
    o = Oracle(w)
    fill(o, 4)
    o.step(np.full(4, 10, np.int8))
    np.testing.assert_allclose(o.state()["p"].sum(), float(np.float32(0.8)) * 50.0, rtol=1e-12)


def test_reduces_to_two_levels_when_upper_nodes_never_bind():
    """Upper nodes with limits far above any flow: rewards and state equal
    the same stations without them (every term on)."""
    w = I.tree_workload(24, seed=3)
    p = w.params
    p.alpha_con, p.alpha_sat, p.alpha_decl, p.ep_len = 0.05, 0.2, 0.3, 60
    w.exo = I.Exo(I.price_bank(n_days=3, ep_len=60, seed=3), I.arrival_rates([32], ep_len=60, base=1.5))
    st = w.stations
    st_hi = I.Stations(**{**st.__dict__, "upper_limit_kw": np.full_like(st.upper_limit_kw, 1e9)})
    st_none = I.Stations(**{**st.__dict__, "n_upper": None, "group_parent": None, "upper_parent": None,
                            "upper_limit_kw": None, "upper_eta": None})
    o1 = Oracle(I.Workload(w.name, p, st_hi, w.exo, 0))
    o0 = Oracle(I.Workload(w.name, p, st_none, w.exo, 0))
    rng = np.random.default_rng(5)
    for step in range(80):
        a = rng.integers(0, 11, st.total_ports).astype(np.int8)
        r0, _ = o0.step(a)
        r1, _ = o1.step(a)
        np.testing.assert_array_equal(r0, r1, err_msg=f"step {step}")
    for k, v in o0.state().items():
        np.testing.assert_array_equal(v, o1.state()[k], err_msg=k)


def test_every_node_constraint_holds_along_trajectories():
    """Random levels on the Fig. c stations: after every step each group,
    upper node and grid connection carries at most eta x I (proportional
    rescale keeps each node within its limit), and some nodes bind."""
    w = I.tree_workload(48, seed=1)
    st = w.stations
    o = Oracle(w)
    po, go, uo = st.port_off, st.group_off, st.upper_off
    rng = np.random.default_rng(2)
    bound = 0
    for step in range(120):
        o.step(rng.integers(0, 11, st.total_ports).astype(np.int8))
        pw = o.state()["p"]
        for e in range(st.n_envs):
            gsz = st.group_size[go[e]:go[e + 1]]
            gstart = po[e] + np.concatenate([[0], np.cumsum(gsz)[:-1]])
            gsum = np.array([pw[s:s + k].sum() for s, k in zip(gstart, gsz)])
            gcap = st.group_eta[go[e]:go[e + 1]].astype(np.float64) * st.group_limit_kw[go[e]:go[e + 1]]
            assert np.all(gsum <= gcap * (1 + 1e-9))
            gpar = st.group_parent[go[e]:go[e + 1]]
            upar = st.upper_parent[uo[e]:uo[e + 1]]
            for u in range(st.n_upper[e]):
                under = []
                for g in range(len(gsz)):
                    a = gpar[g]
                    while a >= 0 and a != u:
                        a = upar[a]
                    under.append(a == u)
                s = gsum[np.array(under, bool)].sum()
                cap = float(st.upper_eta[uo[e] + u]) * float(st.upper_limit_kw[uo[e] + u])
                assert s <= cap * (1 + 1e-9)
                bound += s >= cap * (1 - 1e-9)
            assert pw[po[e]:po[e + 1]].sum() <= float(st.grid_eta[e]) * float(st.grid_limit_kw[e]) * (1 + 1e-9)
    assert bound > 100


def test_upper_levels_deepest_first():
    """U1 (30 kW) holds U2 (20 kW) over group g (2 chargers) and a group g'
    (1 charger) directly: U2 first gives g 10 + 10, then U1 scales 20 + 22 by
    30/42.  (U1 first would cut all to 30/66 and leave U2 unbound: 10 kW
    each.)"""
    w = tree_station([2, 1], [100.0, 100.0], [1, 0], [-1, 0], [30.0, 20.0])
    o = Oracle(w)
    fill(o, 3)
    o.step(np.full(3, 10, np.int8))
    np.testing.assert_allclose(o.state()["p"], [10 * 30 / 42, 10 * 30 / 42, 22 * 30 / 42], rtol=1e-12)


def test_penalty_divides_by_node_efficiency():
    """c_con = max over nodes of (1/eta_H) x requested sum - I_H (Eq.
    ArchConst as a soft constraint): a group with eta 0.8 and limit 20 kW
    under two 22 kW requests gives 44/0.8 - 20 = 35; an upper node with eta
    0.5 and limit 60 kW over four such requests gives 88/0.5 - 60 = 116."""
    f32 = lambda x: float(np.float32(x))
    out = {}
    for case, kw in (("group", dict(groups=[2], group_limit=[20.0], group_parent=[-1], upper_parent=[], upper_limit=[],
                                     group_eta=[0.8])),
                     ("upper", dict(groups=[2, 2], group_limit=[1e6, 1e6], group_parent=[0, 0], upper_parent=[-1],
                                     upper_limit=[60.0], upper_eta=[0.5]))):
        r = {}
        for a in (0.0, 1.0):
            w = tree_station(alpha_con=a, alpha_sat=0.0, alpha_decl=0.0, **kw)
            o = Oracle(w)
            fill(o, int(sum(kw["groups"])))
            rr, _ = o.step(np.full(int(sum(kw["groups"])), 10, np.int8))
            r[a] = rr[0]
        out[case] = r[0.0] - r[1.0]
    np.testing.assert_allclose(out["group"], 44.0 / f32(0.8) - 20.0, rtol=1e-9)
    np.testing.assert_allclose(out["upper"], 88.0 / f32(0.5) - 60.0, rtol=1e-9)
