"""Randomised configurations against the oracle: seeded draws of station
layouts (1..128 chargers, group partitions of 4..32, limits from tight to
loose, node and root efficiencies below 1, AC/DC mixes), of the car and
reward parameters (taper threshold, charging target, efficiencies, prices,
penalty weights, stays, episode length) and of the forms (absolute or
increment levels, charge-only or V2G with a station battery, with or without
charge-sensitive users); plain and fused kernels, each over more than one
episode.  Events exact, floats within the tolerances of tests/parity.py."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2507_01522_b300 import inputs as I

from test_gpu_cs import compare_cs
from test_gpu_v2g import compare_traj

pytestmark = pytest.mark.gpu

FORMS = ["absolute", "delta", "v2g", "v2g_delta", "cs", "cs_v2g"]


def random_workload(seed):
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xC0F]))
    form = FORMS[seed % len(FORMS)]
    E = int(rng.integers(40, 110))
    sizes = np.clip(np.rint(np.exp(rng.uniform(0.0, np.log(128.0), E))), 1, 128).astype(np.int32)
    sizes[: 3] = (1, 128, 64)                         # the extremes every time
    ep_len = int(rng.integers(18, 50))
    lo = int(rng.integers(1, 8))
    hi = int(rng.integers(lo, min(3 * ep_len, 120)))
    v2g = form.startswith("v2g") or form == "cs_v2g"
    delta = form.endswith("delta")
    n_levels = int(rng.choice([5, 11, 21])) if (v2g or delta) else int(rng.integers(2, 16))
    pmax = (float(rng.uniform(3.0, 22.0)), float(rng.uniform(40.0, 350.0)))
    cap_lo = float(rng.uniform(10.0, 60.0))
    soc_lo = float(rng.uniform(0.0, 0.6))
    p = I.EnvParams(
        ep_len=ep_len, n_levels=n_levels, tau=float(rng.uniform(0.4, 0.95)), p_sell=float(rng.uniform(0.2, 1.0)),
        c_fixed=float(rng.uniform(0.0, 0.05)), alpha_sat=float(rng.uniform(0.0, 0.3)),
        alpha_decl=float(rng.uniform(0.0, 1.0)), alpha_con=float(rng.uniform(0.0, 0.1)),
        soc_target=float(rng.uniform(0.6, 1.0)), p_max_kw=pmax,
        eta_port=(float(rng.uniform(0.8, 1.0)), float(rng.uniform(0.8, 1.0))),
        cap_kwh=(cap_lo, cap_lo + float(rng.uniform(0.0, 80.0))),
        soc0=(soc_lo, min(1.0, soc_lo + float(rng.uniform(0.0, 0.4)))), stay_steps=(lo, hi),
        rbar_ac_kw=(float(rng.uniform(1.0, 10.0)), float(rng.uniform(10.0, 30.0))),
        rbar_dc_kw=(float(rng.uniform(20.0, 100.0)), float(rng.uniform(100.0, 400.0))),
        v2g=int(v2g), action_delta=int(delta),
        sell_grid_ratio=float(rng.uniform(0.3, 1.0)), alpha_degrad=float(rng.uniform(0.0, 0.05)),
        batt_cap_kwh=float(rng.uniform(50.0, 300.0)), batt_rate_kw=float(rng.uniform(10.0, 120.0)),
        batt_tau=float(rng.uniform(0.5, 0.95)), batt_soc0=float(rng.uniform(0.0, 1.0)),
        p_max_dis_kw=(pmax[0] * float(rng.uniform(0.3, 1.0)), pmax[1] * float(rng.uniform(0.3, 1.0))),
        cs_share_256=int(rng.integers(32, 224)) if form.startswith("cs") else 0,
        alpha_sat1=float(rng.uniform(0.0, 0.1)), beta_early=float(rng.uniform(0.0, 1.0)))
    classes = sorted(set(int(n) for n in sizes))
    group_lo = int(rng.integers(4, 9))
    st = I.mixed_stations(rng, sizes, p.p_max_kw, p_dc=float(rng.uniform(0.0, 1.0)),
                          grid_kw_per_port=float(rng.uniform(3.0, 30.0)), group_frac=float(rng.uniform(0.2, 1.5)),
                          class_sizes=classes, group_lo=group_lo, group_hi=int(rng.integers(group_lo, 33)))
    st.group_eta[:] = rng.uniform(0.8, 1.0, st.group_eta.shape).astype(np.float32)
    st.grid_eta[:] = rng.uniform(0.8, 1.0, st.grid_eta.shape).astype(np.float32)
    exo = I.Exo(I.price_bank(n_days=int(rng.integers(2, 12)), ep_len=ep_len, seed=seed),
                I.arrival_rates(classes, ep_len=ep_len, base=float(rng.uniform(0.3, 3.0))))
    return I.Workload(f"random-{seed}-{form}", p, st, exo, seed), form


@pytest.mark.parametrize("seed", range(30))
@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_random_configuration(cuda_lib, seed, mode):
    import torch
    from paper_2507_01522_b300.chargax import Batch
    w, form = random_workload(seed)
    b, o = Batch(w, seed=seed), Oracle(w, seed=seed)
    steps = w.params.ep_len + 11                       # past an episode end
    k = 1 if mode == "plain" else int(np.random.default_rng(seed).integers(5, 40))
    if form.startswith("cs"):
        compare_cs(w, b, o, torch, steps, mode=mode, k=k)
    else:
        n_done = compare_traj(w, b, o, torch, steps, mode=mode, k=k)
        assert n_done == b.E                          # every station finished one episode
    assert b.stats()["arrived"].sum() > 0
