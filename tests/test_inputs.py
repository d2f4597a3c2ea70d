"""The seeded input generators (no GPU): the Fig. c tree stations obey the
library's tree rules, subsets keep every station's description, and the
variants change only what they name."""
import numpy as np

from paper_2507_01522_b300 import inputs as I


def upper_depths(parent):
    depth = []
    for u in range(len(parent)):
        d, a = 0, u
        while a >= 0 and d <= 3:
            a = parent[a]
            d += 1
        assert a < 0, "chain longer than three levels, or a cycle"
        depth.append(d)
    return depth


def test_tree_stations_obey_the_tree_rules():
    """Parents in range, at most three levels above the groups, every upper
    node with groups below it and those groups consecutive; group sizes
    cover the chargers; limits positive; uneven depth occurs."""
    st = I.tree_stations(np.random.default_rng(0), 400)
    po, go, uo = st.port_off, st.group_off, st.upper_off
    uneven = 0
    for e in range(st.n_envs):
        G, U = int(st.n_groups[e]), int(st.n_upper[e])
        assert st.group_size[go[e]:go[e + 1]].sum() == st.n_ports[e]
        gp, up = st.group_parent[go[e]:go[e + 1]], st.upper_parent[uo[e]:uo[e + 1]]
        assert np.all((gp >= -1) & (gp < U)) and np.all((up >= -1) & (up < U))
        depth = upper_depths(up)
        for u in range(U):
            below = [k for k in range(G) if _under(gp[k], u, up)]
            assert below and below == list(range(below[0], below[-1] + 1))
        group_depth = [1 + (depth[a] if a >= 0 else 0) for a in gp]
        uneven += len(set(group_depth)) > 1
        assert np.all(st.upper_limit_kw[uo[e]:uo[e + 1]] > 0) and np.all(st.group_limit_kw[go[e]:go[e + 1]] > 0)
        assert 1 <= st.n_ports[e] <= 128 and G <= 32 and U <= 32
    assert uneven > 50


def _under(a, u, up):
    while a >= 0 and a != u:
        a = up[a]
    return a == u


def test_subset_keeps_each_station():
    w = I.tree_workload(64, seed=2)
    st = w.stations
    ids = np.array([5, 0, 63, 17])
    sub = st.subset(ids)
    for j, e in enumerate(ids):
        for name, off_full, off_sub in (("group_size", st.group_off, sub.group_off),
                                        ("group_parent", st.group_off, sub.group_off),
                                        ("upper_parent", st.upper_off, sub.upper_off),
                                        ("upper_limit_kw", st.upper_off, sub.upper_off)):
            a = getattr(st, name)[off_full[e]:off_full[e + 1]]
            b = getattr(sub, name)[off_sub[j]:off_sub[j + 1]]
            np.testing.assert_array_equal(a, b, err_msg=name)
        np.testing.assert_array_equal(st.port_type[st.port_off[e]:st.port_off[e + 1]],
                                      sub.port_type[sub.port_off[j]:sub.port_off[j + 1]])
    assert sub.n_ports.tolist() == st.n_ports[ids].tolist()


def test_v2g_variant_changes_only_the_mode():
    w = I.heterogeneous(n_envs=16)
    v = I.v2g_variant(w)
    assert v.params.v2g == 1 and v.params.n_levels == 21 and w.params.v2g == 0
    assert v.stations is w.stations and v.exo is w.exo
    same = {k: x for k, x in w.params.__dict__.items() if k not in ("v2g", "n_levels", "batt_cap_kwh", "batt_rate_kw")}
    assert all(getattr(v.params, k) == x for k, x in same.items())
