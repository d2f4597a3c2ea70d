// handle.cu -- the C interface (include/chargax_b300.h): batch creation and
// layout, launches, CUDA-graph rollouts, autotuning, state access.
#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/chargax_b300.h"
#include "chx_device.cuh"
#include "chx_handle.h"
#include "chx_kernels.h"

using namespace chx;

namespace chx {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(CHX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace chx

#define CUDA_TRY(expr)                                          \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return chx::cuda_fail(_e, #expr); \
    } while (0)

namespace {

template <class T>
int dalloc(Buffers& bufs, T** p, size_t n)
{
    void* q = nullptr;
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return fail(CHX_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    e = cudaMemset(q, 0, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    bufs.push_back(q);
    *p = static_cast<T*>(q);
    return CHX_OK;
}

}  // namespace

namespace chx {

int class_of_ports(int n)
{
    int c = 0;
    while ((8 << c) < n) ++c;
    return c;
}

int validate_params(const chx_env_params* p, const chx_exo* x)
{
    if (!p || !x) return fail(CHX_EINVAL, "null configuration pointer");
    if (p->ep_len < 1 || p->ep_len > (1 << 20)) return fail(CHX_EINVAL, "ep_len out of range");
    if (p->n_levels < 2 || p->n_levels > 255) return fail(CHX_EINVAL, "n_levels must be in 2..255");
    if (!(p->dt_h > 0.f) || !std::isfinite(p->dt_h)) return fail(CHX_EINVAL, "dt_h must be > 0");
    if (!(p->tau > 0.f && p->tau < 1.f)) return fail(CHX_EINVAL, "tau must be in (0,1)");
    if (p->stay_steps[0] < 1 || p->stay_steps[1] > CHX_MAX_STAY || p->stay_steps[0] > p->stay_steps[1])
        return fail(CHX_EINVAL, "stay_steps must satisfy 1 <= lo <= hi <= 255");
    if (!(p->cap_kwh[0] > 0.f) || p->cap_kwh[1] < p->cap_kwh[0]) return fail(CHX_EINVAL, "cap_kwh range invalid");
    if (p->soc0[0] < 0.f || p->soc0[1] > 1.f || p->soc0[1] < p->soc0[0]) return fail(CHX_EINVAL, "soc0 range invalid");
    for (int t = 0; t < 2; ++t) {
        if (!(p->p_max_kw[t] > 0.f)) return fail(CHX_EINVAL, "p_max_kw must be > 0");
        if (!(p->eta_port[t] > 0.f && p->eta_port[t] <= 1.f)) return fail(CHX_EINVAL, "eta_port must be in (0,1]");
        if (p->rbar_kw[t][0] < 0.f || p->rbar_kw[t][1] < p->rbar_kw[t][0]) return fail(CHX_EINVAL, "rbar range invalid");
    }
    if (p->v2g != 0 && p->v2g != 1) return fail(CHX_EINVAL, "v2g must be 0 or 1");
    if (p->v2g) {
        if (p->n_levels < 3 || (p->n_levels & 1) == 0)
            return fail(CHX_EINVAL, "V2G mode needs an odd n_levels >= 3 (levels symmetric around idle)");
        if (!(p->batt_cap_kwh > 0.f) || !std::isfinite(p->batt_cap_kwh)) return fail(CHX_EINVAL, "batt_cap_kwh must be > 0");
        if (!(p->batt_rate_kw >= 0.f) || !std::isfinite(p->batt_rate_kw)) return fail(CHX_EINVAL, "batt_rate_kw must be >= 0");
        if (!(p->batt_tau > 0.f && p->batt_tau < 1.f)) return fail(CHX_EINVAL, "batt_tau must be in (0,1)");
        if (!(p->batt_soc0 >= 0.f && p->batt_soc0 <= 1.f)) return fail(CHX_EINVAL, "batt_soc0 must be in [0,1]");
        if (!(p->sell_grid_ratio >= 0.f) || !std::isfinite(p->sell_grid_ratio))
            return fail(CHX_EINVAL, "sell_grid_ratio must be >= 0");
        if (!std::isfinite(p->alpha_degrad)) return fail(CHX_EINVAL, "alpha_degrad must be finite");
        for (int t = 0; t < 2; ++t)
            if (!(p->p_max_dis_kw[t] > 0.f) || !std::isfinite(p->p_max_dis_kw[t]))
                return fail(CHX_EINVAL, "p_max_dis_kw must be > 0");
    }
    if (p->cs_share_256 < 0 || p->cs_share_256 > 256) return fail(CHX_EINVAL, "cs_share_256 must be in 0..256");
    if (p->cs_share_256 > 0) {
        if (p->stay_steps[1] > 254)
            return fail(CHX_EINVAL, "with charge-sensitive users stays must be <= 254 steps (255 marks such a car)");
        if (!(p->eps_cap >= 0.f && p->eps_cap < 1.f)) return fail(CHX_EINVAL, "eps_cap must be in [0,1)");
        if (!std::isfinite(p->alpha_sat1) || !std::isfinite(p->beta_early))
            return fail(CHX_EINVAL, "alpha_sat1 and beta_early must be finite");
    }
    if (p->action_delta != 0 && p->action_delta != 1) return fail(CHX_EINVAL, "action_delta must be 0 or 1");
    if (p->action_delta && (p->n_levels < 3 || (p->n_levels & 1) == 0))
        return fail(CHX_EINVAL, "the Delta action form needs an odd n_levels >= 3 (increments symmetric around 0)");
    if (x->n_days < 1 || !x->h_price) return fail(CHX_EINVAL, "price bank missing");
    if (x->n_arrival_classes < 1 || !x->h_arrival_rate) return fail(CHX_EINVAL, "arrival table missing");
    const size_t nl = (size_t)x->n_arrival_classes * (size_t)p->ep_len;
    for (size_t i = 0; i < nl; ++i) {
        const float l = x->h_arrival_rate[i];
        if (!(l >= 0.f && l <= 64.f)) return fail(CHX_EINVAL, "arrival rates must be in [0, 64]");
    }
    return CHX_OK;
}

static_assert(kMaxUpperDepth == CHX_MAX_UPPER_DEPTH, "tree depth limits differ");

// Depth below the root of every upper node of one station (a child of the
// root has depth 1); -1 if some chain does not reach the root within
// CHX_MAX_UPPER_DEPTH steps (too deep, or a cycle).
int upper_depths(const int32_t* parent, int n_up, std::vector<int>& depth)
{
    depth.assign(n_up, 0);
    int dmax = 0;
    for (int u = 0; u < n_up; ++u) {
        int d = 0, a = u;
        while (a >= 0 && d <= CHX_MAX_UPPER_DEPTH) {
            a = parent[a];
            ++d;
        }
        if (a >= 0 || d > CHX_MAX_UPPER_DEPTH) return -1;
        depth[u] = d;
        dmax = std::max(dmax, d);
    }
    return dmax;
}

int validate_tree(const chx_stations* st)
{
    if (!st->h_group_parent || !st->h_upper_parent || !st->h_upper_limit_kw)
        return fail(CHX_EINVAL, "deeper tree: missing group_parent, upper_parent or upper_limit_kw");
    long long go = 0, uo = 0;
    std::vector<int> depth;
    for (int e = 0; e < st->n_envs; ++e) {
        const int G = st->h_n_groups[e], U = st->h_n_upper[e];
        const std::string where = "station " + std::to_string(e) + ": ";
        if (U < 0 || U > CHX_MAX_GROUPS) return fail(CHX_EINVAL, where + "n_upper out of 0..32");
        for (int k = 0; k < G; ++k) {
            const int a = st->h_group_parent[go + k];
            if (a < -1 || a >= U) return fail(CHX_EINVAL, where + "group parent out of range");
        }
        for (int u = 0; u < U; ++u) {
            const int a = st->h_upper_parent[uo + u];
            if (a < -1 || a >= U) return fail(CHX_EINVAL, where + "upper parent out of range");
            if (!(st->h_upper_limit_kw[uo + u] > 0.f)) return fail(CHX_EINVAL, where + "upper limit must be > 0");
            if (st->h_upper_eta && !(st->h_upper_eta[uo + u] > 0.f && st->h_upper_eta[uo + u] <= 1.f))
                return fail(CHX_EINVAL, where + "upper eta must be in (0,1]");
        }
        if (upper_depths(st->h_upper_parent + uo, U, depth) < 0)
            return fail(CHX_EINVAL, where + "upper nodes deeper than CHX_MAX_UPPER_DEPTH levels, or a cycle");
        // every node's groups: non-empty and consecutive
        for (int u = 0; u < U; ++u) {
            int lo = G, hi = -1, cnt = 0;
            for (int k = 0; k < G; ++k) {
                int a = st->h_group_parent[go + k];
                while (a >= 0 && a != u) a = st->h_upper_parent[uo + a];
                if (a == u) {
                    lo = std::min(lo, k);
                    hi = std::max(hi, k);
                    ++cnt;
                }
            }
            if (cnt == 0) return fail(CHX_EINVAL, where + "an upper node has no group below it");
            if (hi - lo + 1 != cnt) return fail(CHX_EINVAL, where + "the groups below an upper node are not consecutive");
        }
        go += G;
        uo += U;
    }
    return CHX_OK;
}

int validate_stations(const chx_stations* st, const chx_exo* x, long long max_envs)
{
    if (!st || !x) return fail(CHX_EINVAL, "null configuration pointer");
    if (st->n_envs < 1 || st->n_envs > max_envs) return fail(CHX_EINVAL, "n_envs out of range");
    if (!st->h_n_ports || !st->h_port_type || !st->h_n_groups || !st->h_group_size || !st->h_group_limit_kw ||
        !st->h_grid_limit_kw || !st->h_arrival_class)
        return fail(CHX_EINVAL, "missing station array");
    long long go = 0, po = 0;
    for (int e = 0; e < st->n_envs; ++e) {
        const int n = st->h_n_ports[e], G = st->h_n_groups[e];
        if (n < 1 || n > CHX_MAX_PORTS) return fail(CHX_EINVAL, "station " + std::to_string(e) + ": n_ports out of 1..128");
        if (G < 1 || G > std::min(n, CHX_MAX_GROUPS))
            return fail(CHX_EINVAL, "station " + std::to_string(e) + ": n_groups out of 1..min(n_ports,32)");
        long long sum = 0;
        for (int k = 0; k < G; ++k) {
            const int gs = st->h_group_size[go + k];
            if (gs < 1) return fail(CHX_EINVAL, "station " + std::to_string(e) + ": empty group");
            sum += gs;
            const float L = st->h_group_limit_kw[go + k];
            if (!(L > 0.f)) return fail(CHX_EINVAL, "station " + std::to_string(e) + ": group limit must be > 0");
            if (st->h_group_eta) {
                const float eta = st->h_group_eta[go + k];
                if (!(eta > 0.f && eta <= 1.f)) return fail(CHX_EINVAL, "group eta must be in (0,1]");
            }
        }
        if (sum != n) return fail(CHX_EINVAL, "station " + std::to_string(e) + ": group sizes do not cover the chargers");
        if (!(st->h_grid_limit_kw[e] > 0.f)) return fail(CHX_EINVAL, "grid limit must be > 0");
        if (st->h_grid_eta && !(st->h_grid_eta[e] > 0.f && st->h_grid_eta[e] <= 1.f))
            return fail(CHX_EINVAL, "grid eta must be in (0,1]");
        if (st->h_arrival_class[e] < 0 || st->h_arrival_class[e] >= x->n_arrival_classes)
            return fail(CHX_EINVAL, "arrival_class out of range");
        for (int q = 0; q < n; ++q)
            if (st->h_port_type[po + q] > 1) return fail(CHX_EINVAL, "port_type must be 0 or 1");
        go += G;
        po += n;
    }
    if (po >= (1LL << 31)) return fail(CHX_EINVAL, "more than 2^31 - 1 chargers in one batch");
    if (st->h_n_upper) return validate_tree(st);
    return CHX_OK;
}

int validate(const chx_stations* st, const chx_env_params* p, const chx_exo* x)
{
    int rc = validate_params(p, x);
    if (rc) return rc;
    return validate_stations(st, x, 1LL << 26);
}

void build_poisson_cdf(const float* lam, size_t n_rows_steps, std::vector<float>& F)
{
    F.assign(n_rows_steps * kCdfLen, 0.f);
    for (size_t i = 0; i < n_rows_steps; ++i) {
        float* f = F.data() + i * kCdfLen;
        const float l = lam[i];
        float pk = (float)std::exp(-(double)l);
        float cdf = pk;
        f[0] = cdf;
        for (int k = 1; k < kPoissonMax; ++k) {
            const float num = pk * l;           // separate statements: no contraction
            pk = num / (float)k;
            cdf = cdf + pk;
            f[k] = cdf;
        }
        f[kPoissonMax] = INFINITY;
    }
}

DevParams make_params(const chx_env_params& q, int n_days)
{
    DevParams p{};
    p.ep_len = q.ep_len;
    p.n_levels = q.n_levels;
    p.n_days = n_days;
    p.dt = q.dt_h;
    p.inv_dt = (float)(1.0 / (double)q.dt_h);
    p.tau = q.tau;
    p.inv_1m_tau = (float)(1.0 / (1.0 - (double)q.tau));
    p.p_sell = q.p_sell;
    p.c_fixed = q.c_fixed;
    p.a_sat = q.alpha_sat;
    p.a_decl = q.alpha_decl;
    p.a_con = q.alpha_con;
    p.soc_target = q.soc_target;
    p.pmax0 = q.p_max_kw[0];
    p.pmax1 = q.p_max_kw[1];
    p.v2g = q.v2g ? 1 : 0;
    p.delta = q.action_delta ? 1 : 0;
    p.half = (p.v2g || p.delta) ? (q.n_levels - 1) / 2 : 0;
    const double per_level = p.half ? (double)p.half : (double)(q.n_levels - 1);
    p.pdis0 = p.v2g ? q.p_max_dis_kw[0] : q.p_max_kw[0];
    p.pdis1 = p.v2g ? q.p_max_dis_kw[1] : q.p_max_kw[1];
    p.lvl0 = (float)((double)q.p_max_kw[0] / per_level);
    p.lvl1 = (float)((double)q.p_max_kw[1] / per_level);
    p.eta0 = q.eta_port[0];
    p.eta1 = q.eta_port[1];
    if (p.v2g) {
        p.batt_cap = q.batt_cap_kwh;
        p.inv_batt_cap = (float)(1.0 / (double)q.batt_cap_kwh);
        p.batt_rate = q.batt_rate_kw;
        p.batt_lvl = (float)((double)q.batt_rate_kw / (double)p.half);
        p.batt_tau = q.batt_tau;
        p.batt_inv_1m_tau = (float)(1.0 / (1.0 - (double)q.batt_tau));
        p.batt_soc0 = q.batt_soc0;
        p.sell_grid_ratio = q.sell_grid_ratio;
        p.a_degrad = q.alpha_degrad;
        p.obs_inv_batt_rate = q.batt_rate_kw > 0.f ? (float)(1.0 / (double)q.batt_rate_kw) : 0.f;
    }
    p.obs_env = p.v2g ? 10 : 8;
    p.cs_share = q.cs_share_256;
    p.a_sat1 = q.alpha_sat1;
    p.beta = q.beta_early;
    p.eps = q.eps_cap;
    p.obs_port = q.cs_share_256 > 0 ? 7 : 6;
    p.inv_eta0 = (float)(1.0 / (double)q.eta_port[0]);
    p.inv_eta1 = (float)(1.0 / (double)q.eta_port[1]);
    p.cap_lo = q.cap_kwh[0];
    p.cap_span = q.cap_kwh[1] - q.cap_kwh[0];
    p.soc_lo = q.soc0[0];
    p.soc_span = q.soc0[1] - q.soc0[0];
    p.stay_lo = q.stay_steps[0];
    p.stay_span = (uint32_t)(q.stay_steps[1] - q.stay_steps[0] + 1);
    p.rb_lo0 = q.rbar_kw[0][0];
    p.rb_span0 = q.rbar_kw[0][1] - q.rbar_kw[0][0];
    p.rb_lo1 = q.rbar_kw[1][0];
    p.rb_span1 = q.rbar_kw[1][1] - q.rbar_kw[1][0];
    p.inv_pmax0 = 1.0f / q.p_max_kw[0];      // FP32 division: the value the kernels computed before
    p.inv_pmax1 = 1.0f / q.p_max_kw[1];
    p.obs_inv_stay = (float)(1.0 / (double)q.stay_steps[1]);
    p.obs_inv_cap = (float)(1.0 / (double)q.cap_kwh[1]);
    p.obs_inv_days = (float)(1.0 / (double)n_days);
    p.obs_inv_len = (float)(1.0 / (double)q.ep_len);
    return p;
}

}  // namespace chx

// ===========================================================================
// lifetime
// ===========================================================================

extern "C" const char* chx_last_error(void) { return chx::g_last_error.c_str(); }

namespace chx {

int build_handle(const chx_stations* st, const chx_env_params* prm, const chx_exo* exo, uint64_t seed,
                 int min_pad_envs_per_class, chx_handle** out)
{
    int rc = validate(st, prm, exo);
    if (rc) return rc;
    auto* h = new chx_handle();
    h->params = *prm;
    h->E = st->n_envs;
    h->n_days = exo->n_days;
    h->n_arrival_classes = exo->n_arrival_classes;
    CUDA_TRY(cudaGetDevice(&h->device));
    CUDA_TRY(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device));

    // ---- classes and slot layout
    const int E = h->E;
    std::vector<int> cls(E);
    h->user_port_off.assign(E + 1, 0);
    std::vector<long long> group_off(E + 1, 0);
    for (int e = 0; e < E; ++e) {
        cls[e] = class_of_ports(st->h_n_ports[e]);
        h->user_port_off[e + 1] = h->user_port_off[e] + st->h_n_ports[e];
        group_off[e + 1] = group_off[e] + st->h_n_groups[e];
    }
    h->P = h->user_port_off[E];
    int count[kNumClasses] = {0, 0, 0, 0, 0};
    for (int e = 0; e < E; ++e) count[cls[e]]++;
    int env_base = 0;
    long long port_base = 0;
    for (int c = 0; c < kNumClasses; ++c) {
        const int C = 8 << c;
        const int epw = tile_epw(c);
        int padded = (count[c] + epw - 1) / epw * epw;
        if (padded < min_pad_envs_per_class && count[c] > 0) padded = min_pad_envs_per_class;
        h->cls_n_env[c] = padded;
        h->cls_n_real[c] = count[c];
        h->cls_env_base[c] = env_base;
        h->cls_port_base[c] = port_base;
        env_base += padded;
        port_base += (long long)padded * C;
    }
    h->n_slots = env_base;
    h->n_port_slots = port_base;
    h->user_to_slot.assign(E, -1);
    h->slot_user.assign(h->n_slots, -1);
    {
        int fill[kNumClasses] = {0, 0, 0, 0, 0};
        for (int e = 0; e < E; ++e) {
            const int c = cls[e];
            const int s = h->cls_env_base[c] + fill[c]++;
            h->user_to_slot[e] = s;
            h->slot_user[s] = e;
        }
    }

    // ---- host images of the static arrays
    const long long PS = h->n_port_slots;
    const int NS = h->n_slots;
    std::vector<uint32_t> meta(PS, 0);
    std::vector<float> gcap(PS, 0.f), ginv(PS, 0.f);
    std::vector<int32_t> s_uid(NS, -1), s_uoff(NS, 0), s_n(NS, 0), s_arr(NS, 0);
    std::vector<float> s_gcap(NS, 0.f), s_ginv(NS, 0.f);
    h->slot_port_base.assign(NS, 0);
    for (int s = 0; s < NS; ++s) {
        int c = 0;
        for (int i = 1; i < kNumClasses; ++i)
            if (s >= h->cls_env_base[i]) c = i;
        h->slot_port_base[s] = h->cls_port_base[c] + (long long)(s - h->cls_env_base[c]) * (8 << c);
    }
    for (int e = 0; e < E; ++e) {
        const int s = h->user_to_slot[e];
        const long long pb = h->slot_port_base[s];
        const int n = st->h_n_ports[e];
        s_uid[s] = e;
        s_uoff[s] = (int32_t)h->user_port_off[e];
        s_n[s] = n;
        s_arr[s] = st->h_arrival_class[e];
        const double eta0 = st->h_grid_eta ? st->h_grid_eta[e] : 1.0;
        s_gcap[s] = (float)(eta0 * (double)st->h_grid_limit_kw[e]);
        s_ginv[s] = (float)(1.0 / eta0);
        int q = 0;
        for (int k = 0; k < st->h_n_groups[e]; ++k) {
            const long long gi = group_off[e] + k;
            const int gs = st->h_group_size[gi];
            const double eta = st->h_group_eta ? st->h_group_eta[gi] : 1.0;
            const float cap = (float)(eta * (double)st->h_group_limit_kw[gi]);
            const float inv = (float)(1.0 / eta);
            for (int r = 0; r < gs; ++r, ++q) {
                uint32_t m = kMetaValid | (uint32_t)k << kMetaGroupShift;
                if (st->h_port_type[h->user_port_off[e] + q]) m |= kMetaDC;
                if (r == 0) m |= kMetaHead;
                if (r == gs - 1) m |= kMetaTail;
                meta[pb + q] = m;
                gcap[pb + q] = cap;
                ginv[pb + q] = inv;
            }
        }
    }

    // ---- deeper trees: per level (deepest first) a partition of each
    // station's chargers into its upper nodes at that depth and
    // pass-through runs (branches that are shallower); per charger and level
    // head / tail / slot bits and the node's eta * I and 1 / eta
    int tree_levels = 0;
    std::vector<uint32_t> meta2;
    std::vector<float> ucap, uinv;
    if (st->h_n_upper) {
        std::vector<int> depth;
        long long uo = 0;
        std::vector<long long> upper_off(E + 1, 0);
        for (int e = 0; e < E; ++e) {
            upper_off[e + 1] = upper_off[e] + st->h_n_upper[e];
            tree_levels = std::max(tree_levels, upper_depths(st->h_upper_parent + upper_off[e], st->h_n_upper[e], depth));
        }
        meta2.assign(PS, 0u);
        ucap.assign((size_t)tree_levels * PS, 0.f);
        uinv.assign((size_t)tree_levels * PS, 0.f);
        for (int e = 0; e < E; ++e) {
            const int G = st->h_n_groups[e], U = st->h_n_upper[e];
            uo = upper_off[e];
            upper_depths(st->h_upper_parent + uo, U, depth);
            const long long pb = h->slot_port_base[h->user_to_slot[e]];
            for (int j = 0; j < tree_levels; ++j) {
                const int lev = tree_levels - j;          // depth of the nodes of level j
                int q = 0, slot = -1, prev = -2;
                for (int k = 0; k < G; ++k) {
                    int a = st->h_group_parent[group_off[e] + k];
                    while (a >= 0 && depth[a] > lev) a = st->h_upper_parent[uo + a];
                    const int anc = (a >= 0 && depth[a] == lev) ? a : -1;   // -1: pass-through
                    if (anc != prev || (anc < 0 && prev >= 0)) ++slot;
                    const int gs = st->h_group_size[group_off[e] + k];
                    double eta = 1.0, lim = 0.0;
                    if (anc >= 0) {
                        eta = st->h_upper_eta ? st->h_upper_eta[uo + anc] : 1.0;
                        lim = st->h_upper_limit_kw[uo + anc];
                    }
                    for (int r = 0; r < gs; ++r, ++q) {
                        const long long i = pb + q;
                        uint32_t bits = (uint32_t)slot << 2;
                        if (anc != prev && r == 0) bits |= 1u;   // head
                        meta2[i] |= bits << (8 * j);
                        ucap[(size_t)j * PS + i] = anc >= 0 ? (float)(eta * lim) : FLT_MAX;
                        uinv[(size_t)j * PS + i] = (float)(1.0 / eta);
                    }
                    prev = anc;
                }
                // tails: the last charger of each segment
                for (int r = 0; r < q; ++r) {
                    const long long i = pb + r;
                    const bool last = r == q - 1 || ((meta2[i + 1] >> (8 * j)) & 1u);
                    if (last) meta2[i] |= 2u << (8 * j);
                }
            }
        }
    }

    // ---- device arrays
    DevBatch& b = h->b;
    Buffers& B = h->bufs;
#define ALLOC(ptr, n) \
    if ((rc = dalloc(B, &(ptr), (n)))) { chx_destroy(h); return rc; }
    ALLOC(b.soc, PS) ALLOC(b.erem, PS) ALLOC(b.cap, PS) ALLOC(b.rbar, PS) ALLOC(b.pw, PS)
    ALLOC(b.trem, PS) ALLOC(b.meta, PS) ALLOC(b.gcap, PS) ALLOC(b.ginv_eta, PS)
    ALLOC(b.user_id, NS) ALLOC(b.user_port_off, NS) ALLOC(b.n_ports, NS) ALLOC(b.arrival_class, NS)
    ALLOC(b.grid_cap, NS) ALLOC(b.grid_inv_eta, NS) ALLOC(b.tod, NS) ALLOC(b.day, NS) ALLOC(b.gstep, NS) ALLOC(b.ncar, NS)
    ALLOC(b.key0, NS) ALLOC(b.key1, NS) ALLOC(b.ep_ret, NS) ALLOC(b.last_ret, NS) ALLOC(b.n_episodes, NS)
    ALLOC(b.bsoc, NS) ALLOC(b.bp, NS) ALLOC(b.due, PS)
    if (tree_levels > 0) {
        ALLOC(b.meta2, PS) ALLOC(b.ucap, (size_t)tree_levels * PS) ALLOC(b.uinv, (size_t)tree_levels * PS)
    }
    ALLOC(b.st_arrived, NS) ALLOC(b.st_rejected, NS) ALLOC(b.st_missing, NS) ALLOC(b.st_charged, NS)
    ALLOC(h->d_user_to_slot, E) ALLOC(h->d_counter, 64) ALLOC(b.err, 1)
    const size_t nprice = (size_t)exo->n_days * prm->ep_len, nlam = (size_t)exo->n_arrival_classes * prm->ep_len;
    float *price = nullptr, *cdf = nullptr;
    ALLOC(price, nprice) ALLOC(cdf, nlam * kCdfLen)
#undef ALLOC
    b.price = price;
    b.cdf = cdf;
    std::vector<float> F;
    build_poisson_cdf(exo->h_arrival_rate, nlam, F);
    CUDA_TRY(cudaMemcpy(price, exo->h_price, nprice * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(cdf, F.data(), F.size() * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b.meta, meta.data(), PS * sizeof(uint32_t), cudaMemcpyHostToDevice));
    if (tree_levels > 0) {
        CUDA_TRY(cudaMemcpy(b.meta2, meta2.data(), PS * sizeof(uint32_t), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(b.ucap, ucap.data(), ucap.size() * sizeof(float), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(b.uinv, uinv.data(), uinv.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    CUDA_TRY(cudaMemcpy(b.gcap, gcap.data(), PS * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b.ginv_eta, ginv.data(), PS * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b.user_id, s_uid.data(), NS * sizeof(int32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b.user_port_off, s_uoff.data(), NS * sizeof(int32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b.n_ports, s_n.data(), NS * sizeof(int32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b.arrival_class, s_arr.data(), NS * sizeof(int32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b.grid_cap, s_gcap.data(), NS * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b.grid_inv_eta, s_ginv.data(), NS * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(h->d_user_to_slot, h->user_to_slot.data(), E * sizeof(int32_t), cudaMemcpyHostToDevice));
    for (int c = 0; c < kNumClasses; ++c) {
        b.cls_n_env[c] = h->cls_n_env[c];
        b.cls_env_base[c] = h->cls_env_base[c];
        b.cls_port_base[c] = h->cls_port_base[c];
    }
    b.n_slots = NS;
    b.port_slots = PS;
    h->dp = make_params(*prm, exo->n_days);
    h->dp.tree_levels = tree_levels;

    // fused schedule: largest class first
    h->sched.n_sched = 0;
    int tb = 0;
    for (int c = kNumClasses - 1; c >= 0; --c) {
        if (h->cls_n_env[c] == 0) continue;
        const int epw = tile_epw(c);
        h->sched.sched_cls[h->sched.n_sched] = c;
        h->sched.sched_tile_base[h->sched.n_sched] = tb;
        h->sched.n_sched++;
        tb += h->cls_n_env[c] / epw;
    }
    h->sched.sched_tile_base[h->sched.n_sched] = tb;
    h->sched.total_tiles = tb;
    h->sched.counter = h->d_counter;
    h->sched.ld_out = 1;
    h->sched.ld_step = 1;
    h->warps_per_block = 8;
    h->steps_per_launch = 32;
    CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&h->side.aux, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&h->side.fork, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&h->side.join, cudaEventDisableTiming));
    for (auto& ev : h->chunk_done) CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CUDA_TRY(cudaStreamCreateWithFlags(&h->in_stream, cudaStreamNonBlocking));
    for (int c = 0; c < kActChunks; ++c) {
        CUDA_TRY(cudaEventCreateWithFlags(&h->act_in[c], cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&h->act_done[c], cudaEventDisableTiming));
    }

    launch_reset(b, h->dp, h->d_user_to_slot, nullptr, E, E, seed, 0);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaDeviceSynchronize());
    *out = h;
    return CHX_OK;
}

void free_graph(chx_handle* h)
{
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->graph_exec = nullptr;
    h->graph = nullptr;
    h->graph_key = GraphKey{};
}

}  // namespace chx

extern "C" int chx_create(const chx_stations* st, const chx_env_params* params, const chx_exo* exo, uint64_t seed,
                          chx_handle** out)
{
    if (!out) return fail(CHX_EINVAL, "out is null");
    *out = nullptr;
    return build_handle(st, params, exo, seed, 0, out);
}

extern "C" int chx_destroy(chx_handle* h)
{
    if (!h) return CHX_OK;
    free_graph(h);
    free_policy(h);
    for (void* p : h->bufs) cudaFree(p);
    for (void* p : h->staging) cudaFree(p);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->side.aux) cudaStreamDestroy(h->side.aux);
    if (h->side.fork) cudaEventDestroy(h->side.fork);
    if (h->side.join) cudaEventDestroy(h->side.join);
    for (auto ev : h->chunk_done)
        if (ev) cudaEventDestroy(ev);
    if (h->in_stream) cudaStreamDestroy(h->in_stream);
    for (int c = 0; c < chx::kActChunks; ++c) {
        if (h->act_in[c]) cudaEventDestroy(h->act_in[c]);
        if (h->act_done[c]) cudaEventDestroy(h->act_done[c]);
    }
    delete h;
    return CHX_OK;
}

extern "C" int chx_n_envs(const chx_handle* h, int32_t* out)
{
    if (!h || !out) return fail(CHX_EINVAL, "null argument");
    *out = h->E;
    return CHX_OK;
}

extern "C" int chx_n_ports_total(const chx_handle* h, int64_t* out)
{
    if (!h || !out) return fail(CHX_EINVAL, "null argument");
    *out = h->P;
    return CHX_OK;
}

extern "C" int chx_port_offsets(const chx_handle* h, int64_t* h_offsets)
{
    if (!h || !h_offsets) return fail(CHX_EINVAL, "null argument");
    for (int e = 0; e <= h->E; ++e) h_offsets[e] = h->user_port_off[e];
    return CHX_OK;
}

extern "C" int chx_obs_size(const chx_handle* h, int64_t* out)
{
    if (!h || !out) return fail(CHX_EINVAL, "null argument");
    *out = (long long)h->dp.obs_env * h->E + (long long)h->dp.obs_port * h->P;
    return CHX_OK;
}

// ===========================================================================
// reset / step / observe
// ===========================================================================

extern "C" int chx_reset(chx_handle* h, const int32_t* d_env_ids, int32_t n, uint64_t seed, void* stream)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    if (n < 0) return fail(CHX_EINVAL, "n < 0");
    const int count = d_env_ids ? n : h->E;
    launch_reset(h->b, h->dp, h->d_user_to_slot, d_env_ids, count, h->E, seed, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    return CHX_OK;
}

extern "C" int chx_step(chx_handle* h, const int8_t* d_actions, int64_t lda, float* d_reward, uint8_t* d_done,
                        void* stream)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    if (d_actions && lda < 1) return fail(CHX_EINVAL, "lda must be >= 1");
    launch_step_plain(h->b, h->dp, d_actions, lda, d_reward, d_done, nullptr, 0, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    return CHX_OK;
}

namespace chx {

int enqueue_fused(chx_handle* h, int k_steps, const int8_t* actions, long long lda, float* reward, uint8_t* done,
                  long long ld_out, float* obs, int warps, cudaStream_t st, long long ld_step, long long lda_step,
                  int act_bits)
{
    FusedIO io = h->sched;
    io.k_steps = k_steps;
    io.actions = actions;
    io.lda = lda;
    io.lda_step = lda_step;
    io.act_bits = act_bits;
    io.reward = reward;
    io.done = done;
    io.ld_out = ld_out;
    io.ld_step = ld_step;
    io.obs = obs;
    const int threads = warps * 32;
    if (!fused_block_size_ok(threads)) return fail(CHX_ECUDA, "fused kernel cannot be resident with this block size");
    CUDA_TRY(cudaMemsetAsync(h->d_counter, 0, kFusedCounters * sizeof(int), st));
    launch_step_fused(h->b, h->dp, io, threads, h->sm_count, st, &h->side);
    CUDA_TRY(cudaGetLastError());
    return CHX_OK;
}

}  // namespace chx

extern "C" int chx_step_n(chx_handle* h, int32_t k_steps, const int8_t* d_actions, int64_t lda, float* d_reward,
                          uint8_t* d_done, int64_t ld_out, float* d_obs, void* stream)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    if (k_steps < 1) return fail(CHX_EINVAL, "k_steps must be >= 1");
    if (d_actions && lda < k_steps) return fail(CHX_EINVAL, "lda must be >= k_steps");
    if ((d_reward || d_done) && ld_out < k_steps) return fail(CHX_EINVAL, "ld_out must be >= k_steps");
    return enqueue_fused(h, k_steps, d_actions, lda, d_reward, d_done, ld_out, d_obs, h->warps_per_block,
                         (cudaStream_t)stream);
}

extern "C" int chx_observe(chx_handle* h, float* d_obs, void* stream)
{
    if (!h || !d_obs) return fail(CHX_EINVAL, "null argument");
    launch_observe(h->b, h->dp, d_obs, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    return CHX_OK;
}

// ===========================================================================
// rollout (CUDA graph) and autotuning
// ===========================================================================

namespace chx {

int build_rollout_graph(chx_handle* h, int n_steps, float* reward, uint8_t* done, float* obs)
{
    free_graph(h);
    cudaStream_t cs = h->cap_stream;
    CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = CHX_OK;
    const int K = h->steps_per_launch;
    for (int k0 = 0; k0 < n_steps && rc == CHX_OK; k0 += K) {
        const int k = std::min(K, n_steps - k0);
        const bool last = k0 + k >= n_steps;
        rc = enqueue_fused(h, k, nullptr, 0, reward ? reward + k0 : nullptr, done ? done + k0 : nullptr, n_steps,
                           last ? obs : nullptr, h->warps_per_block, cs);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    h->graph = g;
    e = cudaGraphInstantiate(&h->graph_exec, g, 0);
    if (e != cudaSuccess) {
        free_graph(h);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    h->graph_key = GraphKey{n_steps, reward, done, obs, h->steps_per_launch, h->warps_per_block, true};
    return CHX_OK;
}

int rollout(chx_handle* h, int n_steps, float* reward, uint8_t* done, float* obs, cudaStream_t st)
{
    const GraphKey want{n_steps, reward, done, obs, h->steps_per_launch, h->warps_per_block, true};
    if (!(h->graph_key == want)) {
        int rc = build_rollout_graph(h, n_steps, reward, done, obs);
        if (rc) return rc;
    }
    CUDA_TRY(cudaGraphLaunch(h->graph_exec, st));
    return CHX_OK;
}

void* staging(chx_handle* h, int slot, size_t bytes)
{
    if (h->staging_bytes[slot] < bytes) {
        if (h->staging[slot]) cudaFree(h->staging[slot]);
        h->staging[slot] = nullptr;
        h->staging_bytes[slot] = 0;
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        h->staging[slot] = p;
        h->staging_bytes[slot] = bytes;
    }
    return h->staging[slot];
}

}  // namespace chx

extern "C" int chx_rollout(chx_handle* h, int32_t n_steps, float* d_reward, uint8_t* d_done, float* d_obs,
                           void* stream)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    if (n_steps < 1) return fail(CHX_EINVAL, "n_steps must be >= 1");
    return rollout(h, n_steps, d_reward, d_done, d_obs, (cudaStream_t)stream);
}

namespace chx {

// Launch sizes of a host-buffer rollout: shrinking 5:4:2:1 shares, so each
// chunk's copy out hides behind the next chunk's compute and only the last,
// smallest chunk (and the final observation) is copied after the last launch.
int host_chunks(int n_steps, int* sizes)
{
    static_assert(kHostChunks == 4, "the shares below are for four chunks");
    if (n_steps < kHostChunks) {
        for (int c = 0; c < n_steps; ++c) sizes[c] = 1;
        return n_steps;
    }
    sizes[1] = std::max(1, n_steps * 4 / 12);
    sizes[2] = std::max(1, n_steps * 2 / 12);
    sizes[3] = std::max(1, n_steps / 12);
    sizes[0] = n_steps - sizes[1] - sizes[2] - sizes[3];
    return kHostChunks;
}

}  // namespace chx

// Host-call rollout: the steps run in up to kHostChunks fused launches on the
// caller's stream, outputs step-major in device staging; after each launch an
// event lets the copy stream bring that chunk's rows (contiguous) to the host
// while the next chunk computes; the observation follows the last chunk.
extern "C" int chx_rollout_host(chx_handle* h, int32_t n_steps, float* h_reward, uint8_t* h_done, float* h_obs,
                                void* stream)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    if (n_steps < 1) return fail(CHX_EINVAL, "n_steps must be >= 1");
    const size_t E = (size_t)h->E, ne = E * (size_t)n_steps;
    const size_t nobs = (size_t)h->dp.obs_env * E + (size_t)h->dp.obs_port * (size_t)h->P;
    float* dr = h_reward ? (float*)staging(h, 0, ne * sizeof(float)) : nullptr;
    uint8_t* dd = h_done ? (uint8_t*)staging(h, 1, ne) : nullptr;
    float* dob = h_obs ? (float*)staging(h, 2, nobs * sizeof(float)) : nullptr;
    if ((h_reward && !dr) || (h_done && !dd) || (h_obs && !dob)) return fail(CHX_ENOMEM, "staging allocation failed");
    cudaStream_t st = (cudaStream_t)stream, cs = h->copy_stream;
    int sizes[kHostChunks];
    const int n_chunks = host_chunks(n_steps, sizes);
    for (int c = 0, k0 = 0; c < n_chunks; k0 += sizes[c], ++c) {
        const int k = sizes[c];
        const bool last = c == n_chunks - 1;
        const size_t off = (size_t)k0 * E, n = (size_t)k * E;
        int rc = enqueue_fused(h, k, nullptr, 0, dr ? dr + off : nullptr, dd ? dd + off : nullptr, 1,
                               last ? dob : nullptr, h->warps_per_block, st, (long long)E);
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(h->chunk_done[c], st));
        CUDA_TRY(cudaStreamWaitEvent(cs, h->chunk_done[c], 0));
        if (h_reward) CUDA_TRY(cudaMemcpyAsync(h_reward + off, dr + off, n * sizeof(float), cudaMemcpyDeviceToHost, cs));
        if (h_done) CUDA_TRY(cudaMemcpyAsync(h_done + off, dd + off, n, cudaMemcpyDeviceToHost, cs));
        if (last && h_obs) CUDA_TRY(cudaMemcpyAsync(h_obs, dob, nobs * sizeof(float), cudaMemcpyDeviceToHost, cs));
    }
    CUDA_TRY(cudaStreamSynchronize(cs));
    CUDA_TRY(cudaStreamSynchronize(st));
    return CHX_OK;
}

// Host-actions rollout: the given levels of every step come from the host.
// The steps run in up to kActChunks fused launches on the caller's stream,
// of near-equal size but for a short last one.  The input stream copies chunk c's levels (contiguous,
// step-major) to device staging while chunk c - 1 computes; the copy stream
// brings chunk c's rewards and done flags back while chunk c + 1 computes;
// the observation follows the last chunk.
namespace {
// Step ranges of a host-levels rollout: chunk c runs steps start[c] ..
// start[c + 1] - 1, each launch starting when its levels have arrived.
// With int8 levels the copy in is the slowest stream (a step's levels take
// about twice as long to copy as to step), so what follows the last copy in
// (the last launch, its outputs' copy out, the final observation's copy) is
// on the critical path: consecutive chunks shrink by `shrink`, each launch
// still ending before the next chunk's levels arrive, and the last is short.
// Packed 4-bit levels copy about as fast as the kernel steps: there equal
// chunks (shrink 1) keep the first launch's wait short, which measured
// better than shrinking ones.
int act_chunks(int n_steps, double shrink, int* start)
{
    const int n = n_steps < kActChunks ? n_steps : kActChunks;
    double wc[kActChunks], tot = 0.0, w = 1.0;
    for (int c = 0; c < n; ++c) {
        wc[c] = w;
        tot += w;
        w *= shrink;
    }
    double acc = 0.0;
    start[0] = 0;
    for (int c = 1; c < n; ++c) {
        acc += wc[c - 1];
        int x = (int)std::lround((double)n_steps * acc / tot);
        x = std::max(x, start[c - 1] + 1);       // every chunk at least one step
        x = std::min(x, n_steps - (n - c));      // and room for the ones after it
        start[c] = x;
    }
    start[n] = n_steps;
    return n;
}

// The host-actions rollout: n_steps of given levels from pinned host memory
// (bits 8: one int8 per action slot; 4: two per byte, rows of whole bytes per
// step), copied in kActChunks pieces on the input stream; each launch waits
// only for its own piece, and its outputs go back while the next computes.
int rollout_host_levels(chx_handle* h, int32_t n_steps, const void* h_levels, int bits, float* h_reward,
                        uint8_t* h_done, float* h_obs, void* stream)
{
    const size_t E = (size_t)h->E, ne = E * (size_t)n_steps;
    const size_t nact = (size_t)h->P + (h->dp.v2g ? E : 0);
    const size_t row = bits == 4 ? (nact + 1) / 2 : nact;   // bytes of one step's levels
    const size_t nobs = (size_t)h->dp.obs_env * E + (size_t)h->dp.obs_port * (size_t)h->P;
    char* da = (char*)staging(h, 6, row * (size_t)n_steps);
    float* dr = h_reward ? (float*)staging(h, 0, ne * sizeof(float)) : nullptr;
    uint8_t* dd = h_done ? (uint8_t*)staging(h, 1, ne) : nullptr;
    float* dob = h_obs ? (float*)staging(h, 2, nobs * sizeof(float)) : nullptr;
    if (!da || (h_reward && !dr) || (h_done && !dd) || (h_obs && !dob))
        return fail(CHX_ENOMEM, "staging allocation failed");
    cudaStream_t st = (cudaStream_t)stream, cs = h->copy_stream, is = h->in_stream;
    int start[kActChunks + 1];
    const int n_chunks = act_chunks(n_steps, bits == 8 ? kActShrink8 : 1.0, start);
    const char* hl = static_cast<const char*>(h_levels);
    // the staging of the previous call may still be read by its last launch
    CUDA_TRY(cudaEventRecord(h->act_done[0], st));
    CUDA_TRY(cudaStreamWaitEvent(is, h->act_done[0], 0));
    for (int c = 0; c < n_chunks; ++c) {
        const int k0 = start[c], k1 = start[c + 1];
        CUDA_TRY(cudaMemcpyAsync(da + (size_t)k0 * row, hl + (size_t)k0 * row, (size_t)(k1 - k0) * row,
                                 cudaMemcpyHostToDevice, is));
        CUDA_TRY(cudaEventRecord(h->act_in[c], is));
    }
    for (int c = 0; c < n_chunks; ++c) {
        const int k0 = start[c], k1 = start[c + 1];
        const bool last = c == n_chunks - 1;
        const size_t off = (size_t)k0 * E, n = (size_t)(k1 - k0) * E;
        CUDA_TRY(cudaStreamWaitEvent(st, h->act_in[c], 0));
        // index of slot q at step k: q + k * (row in level units)
        int rc = enqueue_fused(h, k1 - k0, reinterpret_cast<const int8_t*>(da + (size_t)k0 * row), 1,
                               dr ? dr + off : nullptr, dd ? dd + off : nullptr, 1, last ? dob : nullptr,
                               h->warps_per_block, st, (long long)E, (long long)(bits == 4 ? 2 * row : row), bits);
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(h->act_done[c], st));
        CUDA_TRY(cudaStreamWaitEvent(cs, h->act_done[c], 0));
        if (h_reward) CUDA_TRY(cudaMemcpyAsync(h_reward + off, dr + off, n * sizeof(float), cudaMemcpyDeviceToHost, cs));
        if (h_done) CUDA_TRY(cudaMemcpyAsync(h_done + off, dd + off, n, cudaMemcpyDeviceToHost, cs));
        if (last && h_obs) CUDA_TRY(cudaMemcpyAsync(h_obs, dob, nobs * sizeof(float), cudaMemcpyDeviceToHost, cs));
    }
    CUDA_TRY(cudaStreamSynchronize(cs));
    CUDA_TRY(cudaStreamSynchronize(st));
    return CHX_OK;
}
}  // namespace

extern "C" int chx_rollout_host_actions(chx_handle* h, int32_t n_steps, const int8_t* h_actions, float* h_reward,
                                        uint8_t* h_done, float* h_obs, void* stream)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    if (!h_actions) return fail(CHX_EINVAL, "h_actions is null (use chx_rollout_host for Philox actions)");
    if (n_steps < 1) return fail(CHX_EINVAL, "n_steps must be >= 1");
    return rollout_host_levels(h, n_steps, h_actions, 8, h_reward, h_done, h_obs, stream);
}

extern "C" int chx_rollout_host_levels4(chx_handle* h, int32_t n_steps, const uint8_t* h_levels4, float* h_reward,
                                        uint8_t* h_done, float* h_obs, void* stream)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    if (!h_levels4) return fail(CHX_EINVAL, "h_levels4 is null (use chx_rollout_host for Philox actions)");
    if (n_steps < 1) return fail(CHX_EINVAL, "n_steps must be >= 1");
    if (h->params.n_levels > 16) return fail(CHX_EINVAL, "4-bit levels need n_levels <= 16");
    return rollout_host_levels(h, n_steps, h_levels4, 4, h_reward, h_done, h_obs, stream);
}

extern "C" int chx_step_host(chx_handle* h, const int8_t* h_actions, float* h_reward, uint8_t* h_done, float* h_obs,
                             void* stream)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nobs = (size_t)h->dp.obs_env * (size_t)h->E + (size_t)h->dp.obs_port * (size_t)h->P;
    const size_t nact = (size_t)h->P + (h->dp.v2g ? (size_t)h->E : 0);
    int8_t* da = h_actions ? (int8_t*)staging(h, 3, nact) : nullptr;
    float* dr = h_reward ? (float*)staging(h, 4, (size_t)h->E * sizeof(float)) : nullptr;
    uint8_t* dd = h_done ? (uint8_t*)staging(h, 5, (size_t)h->E) : nullptr;
    float* dob = h_obs ? (float*)staging(h, 2, nobs * sizeof(float)) : nullptr;
    if ((h_actions && !da) || (h_reward && !dr) || (h_done && !dd) || (h_obs && !dob))
        return fail(CHX_ENOMEM, "staging allocation failed");
    if (h_actions) CUDA_TRY(cudaMemcpyAsync(da, h_actions, nact, cudaMemcpyHostToDevice, st));
    launch_step_plain(h->b, h->dp, da, 1, dr, dd, nullptr, 0, st);
    CUDA_TRY(cudaGetLastError());
    if (h_obs) {
        launch_observe(h->b, h->dp, dob, st);
        CUDA_TRY(cudaGetLastError());
    }
    if (h_reward) CUDA_TRY(cudaMemcpyAsync(h_reward, dr, (size_t)h->E * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (h_done) CUDA_TRY(cudaMemcpyAsync(h_done, dd, (size_t)h->E, cudaMemcpyDeviceToHost, st));
    if (h_obs) CUDA_TRY(cudaMemcpyAsync(h_obs, dob, nobs * sizeof(float), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return CHX_OK;
}

extern "C" int chx_set_launch(chx_handle* h, int32_t steps_per_launch, int32_t warps_per_block)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    if (steps_per_launch < 0 || warps_per_block < 0 || warps_per_block > 8)
        return fail(CHX_EINVAL, "launch shape out of range");
    if (steps_per_launch) h->steps_per_launch = steps_per_launch;
    if (warps_per_block) h->warps_per_block = warps_per_block;
    free_graph(h);
    return CHX_OK;
}

namespace chx {

// device-side snapshot of every mutable array, for the autotuner
struct Snapshot {
    std::vector<std::pair<void*, size_t>> items;
    std::vector<void*> copies;
};

int snapshot_take(chx_handle* h, Snapshot& s)
{
    const DevBatch& b = h->b;
    const size_t PS = h->n_port_slots, NS = h->n_slots;
    s.items = {{b.soc, PS * 4}, {b.erem, PS * 4}, {b.cap, PS * 4}, {b.rbar, PS * 4}, {b.pw, PS * 4},
               {b.trem, PS}, {b.tod, NS * 4}, {b.day, NS * 4}, {b.gstep, NS * 4}, {b.ncar, NS * 4}, {b.key0, NS * 4},
               {b.key1, NS * 4}, {b.ep_ret, NS * 4}, {b.last_ret, NS * 4}, {b.n_episodes, NS * 4},
               {b.st_arrived, NS * 4}, {b.st_rejected, NS * 4}, {b.st_missing, NS * 4}, {b.st_charged, NS * 4},
               {b.bsoc, NS * 4}, {b.bp, NS * 4}, {b.due, PS * 2}};
    for (auto& it : s.items) {
        void* c = nullptr;
        if (cudaMalloc(&c, it.second) != cudaSuccess) return fail(CHX_ENOMEM, "snapshot allocation failed");
        s.copies.push_back(c);
        CUDA_TRY(cudaMemcpy(c, it.first, it.second, cudaMemcpyDeviceToDevice));
    }
    return CHX_OK;
}

int snapshot_restore(Snapshot& s)
{
    for (size_t i = 0; i < s.copies.size(); ++i)
        CUDA_TRY(cudaMemcpy(s.items[i].first, s.copies[i], s.items[i].second, cudaMemcpyDeviceToDevice));
    for (void* c : s.copies) cudaFree(c);
    s.copies.clear();
    return CHX_OK;
}

}  // namespace chx

extern "C" int chx_autotune(chx_handle* h, int32_t n_steps, int32_t* h_steps_per_launch, int32_t* h_warps_per_block)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    if (n_steps < 1) return fail(CHX_EINVAL, "n_steps must be >= 1");
    Snapshot snap;
    int rc = snapshot_take(h, snap);
    if (rc) return rc;
    const size_t ne = (size_t)h->E * (size_t)n_steps;
    float* dr = nullptr;
    uint8_t* dd = nullptr;
    if (cudaMalloc(&dr, ne * sizeof(float)) != cudaSuccess || cudaMalloc(&dd, ne) != cudaSuccess) {
        cudaFree(dr);
        snapshot_restore(snap);
        return fail(CHX_ENOMEM, "autotune output allocation failed");
    }
    cudaStream_t st = h->cap_stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int ks[] = {8, 16, 32, 72, 144, 288};
    const int ws[] = {2, 4, 8};
    float best = 1e30f;
    int best_k = h->steps_per_launch, best_w = h->warps_per_block;
    const int old_k = h->steps_per_launch, old_w = h->warps_per_block;
    for (int w : ws) {
        if (!fused_block_size_ok(w * 32)) continue;
        for (int k : ks) {
            if (k > n_steps && k != ks[0]) continue;
            h->steps_per_launch = k;
            h->warps_per_block = w;
            rc = rollout(h, n_steps, dr, dd, nullptr, st);   // capture + warm-up
            if (rc) break;
            float ms_best = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, st);
                rollout(h, n_steps, dr, dd, nullptr, st);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms_best = std::min(ms_best, ms);
            }
            if (ms_best < best) {
                best = ms_best;
                best_k = k;
                best_w = w;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(dr);
    cudaFree(dd);
    free_graph(h);
    int rc2 = snapshot_restore(snap);
    if (rc) {
        h->steps_per_launch = old_k;
        h->warps_per_block = old_w;
        return rc;
    }
    if (rc2) return rc2;
    h->steps_per_launch = best_k;
    h->warps_per_block = best_w;
    h->tuned_ms = best;
    if (h_steps_per_launch) *h_steps_per_launch = best_k;
    if (h_warps_per_block) *h_warps_per_block = best_w;
    return CHX_OK;
}

// ===========================================================================
// state, statistics, checkpoints
// ===========================================================================

namespace {

template <class T>
int fetch(std::vector<T>& v, const T* d, size_t n)
{
    v.resize(n);
    CUDA_TRY(cudaMemcpy(v.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost));
    return CHX_OK;
}
template <class T>
int push(T* d, const std::vector<T>& v)
{
    CUDA_TRY(cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return CHX_OK;
}

// per-charger field: slot array <-> batch-order array
template <class T>
int get_port_field(chx_handle* h, T* out, const T* d)
{
    if (!out) return CHX_OK;
    std::vector<T> v;
    int rc = fetch(v, d, (size_t)h->n_port_slots);
    if (rc) return rc;
    for (int e = 0; e < h->E; ++e) {
        const long long pb = h->slot_port_base[h->user_to_slot[e]];
        const long long n = h->user_port_off[e + 1] - h->user_port_off[e];
        std::memcpy(out + h->user_port_off[e], v.data() + pb, n * sizeof(T));
    }
    return CHX_OK;
}
template <class T>
int set_port_field(chx_handle* h, const T* in, T* d)
{
    if (!in) return CHX_OK;
    std::vector<T> v;
    int rc = fetch(v, d, (size_t)h->n_port_slots);
    if (rc) return rc;
    for (int e = 0; e < h->E; ++e) {
        const long long pb = h->slot_port_base[h->user_to_slot[e]];
        const long long n = h->user_port_off[e + 1] - h->user_port_off[e];
        std::memcpy(v.data() + pb, in + h->user_port_off[e], n * sizeof(T));
    }
    return push(d, v);
}
template <class T>
int get_env_field(chx_handle* h, T* out, const T* d)
{
    if (!out) return CHX_OK;
    std::vector<T> v;
    int rc = fetch(v, d, (size_t)h->n_slots);
    if (rc) return rc;
    for (int e = 0; e < h->E; ++e) out[e] = v[h->user_to_slot[e]];
    return CHX_OK;
}
template <class T>
int set_env_field(chx_handle* h, const T* in, T* d)
{
    if (!in) return CHX_OK;
    std::vector<T> v;
    int rc = fetch(v, d, (size_t)h->n_slots);
    if (rc) return rc;
    for (int e = 0; e < h->E; ++e) v[h->user_to_slot[e]] = in[e];
    return push(d, v);
}

}  // namespace

#define RC(x)                  \
    do {                       \
        int _r = (x);          \
        if (_r) return _r;     \
    } while (0)

extern "C" int chx_get_state(chx_handle* h, float* h_soc, float* h_erem, float* h_cap, float* h_rbar, float* h_p,
                             uint8_t* h_trem, int32_t* h_tod, int32_t* h_day, uint32_t* h_gstep, uint32_t* h_ncar,
                             uint32_t* h_key0,
                             uint32_t* h_key1, float* h_ep_ret)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    CUDA_TRY(cudaDeviceSynchronize());
    const DevBatch& b = h->b;
    RC(get_port_field(h, h_soc, b.soc));
    RC(get_port_field(h, h_erem, b.erem));
    RC(get_port_field(h, h_cap, b.cap));
    RC(get_port_field(h, h_rbar, b.rbar));
    RC(get_port_field(h, h_p, b.pw));
    RC(get_port_field(h, h_trem, (const uint8_t*)b.trem));
    RC(get_env_field(h, h_tod, (const int32_t*)b.tod));
    RC(get_env_field(h, h_day, (const int32_t*)b.day));
    RC(get_env_field(h, h_gstep, (const uint32_t*)b.gstep));
    RC(get_env_field(h, h_ncar, (const uint32_t*)b.ncar));
    RC(get_env_field(h, h_key0, (const uint32_t*)b.key0));
    RC(get_env_field(h, h_key1, (const uint32_t*)b.key1));
    RC(get_env_field(h, h_ep_ret, (const float*)b.ep_ret));
    return CHX_OK;
}

extern "C" int chx_set_state(chx_handle* h, const float* h_soc, const float* h_erem, const float* h_cap,
                             const float* h_rbar, const float* h_p, const uint8_t* h_trem, const int32_t* h_tod,
                             const int32_t* h_day, const uint32_t* h_gstep, const uint32_t* h_ncar,
                             const uint32_t* h_key0,
                             const uint32_t* h_key1, const float* h_ep_ret)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    if (h_tod)
        for (int e = 0; e < h->E; ++e)
            if (h_tod[e] < 0 || h_tod[e] >= h->params.ep_len) return fail(CHX_EINVAL, "step of day out of range");
    if (h_day)
        for (int e = 0; e < h->E; ++e)
            if (h_day[e] < 0 || h_day[e] >= h->n_days) return fail(CHX_EINVAL, "day out of range");
    CUDA_TRY(cudaDeviceSynchronize());
    DevBatch& b = h->b;
    RC(set_port_field(h, h_soc, b.soc));
    RC(set_port_field(h, h_erem, b.erem));
    RC(set_port_field(h, h_cap, b.cap));
    RC(set_port_field(h, h_rbar, b.rbar));
    RC(set_port_field(h, h_p, b.pw));
    RC(set_port_field(h, h_trem, b.trem));
    RC(set_env_field(h, h_tod, b.tod));
    RC(set_env_field(h, h_day, b.day));
    RC(set_env_field(h, h_gstep, b.gstep));
    RC(set_env_field(h, h_ncar, b.ncar));
    RC(set_env_field(h, h_key0, b.key0));
    RC(set_env_field(h, h_key1, b.key1));
    RC(set_env_field(h, h_ep_ret, b.ep_ret));
    return CHX_OK;
}

extern "C" int chx_stats(chx_handle* h, uint32_t* h_arrived, uint32_t* h_rejected, float* h_missing_kwh,
                         float* h_charged_kwh, uint32_t* h_episodes, float* h_last_return)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    CUDA_TRY(cudaDeviceSynchronize());
    const DevBatch& b = h->b;
    RC(get_env_field(h, h_arrived, (const uint32_t*)b.st_arrived));
    RC(get_env_field(h, h_rejected, (const uint32_t*)b.st_rejected));
    RC(get_env_field(h, h_missing_kwh, (const float*)b.st_missing));
    RC(get_env_field(h, h_charged_kwh, (const float*)b.st_charged));
    RC(get_env_field(h, h_episodes, (const uint32_t*)b.n_episodes));
    RC(get_env_field(h, h_last_return, (const float*)b.last_ret));
    return CHX_OK;
}

extern "C" int chx_get_battery(chx_handle* h, float* h_soc, float* h_p)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    CUDA_TRY(cudaDeviceSynchronize());
    RC(get_env_field(h, h_soc, (const float*)h->b.bsoc));
    RC(get_env_field(h, h_p, (const float*)h->b.bp));
    return CHX_OK;
}

extern "C" int chx_set_battery(chx_handle* h, const float* h_soc, const float* h_p)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    if (h_soc)
        for (int e = 0; e < h->E; ++e)
            if (!(h_soc[e] >= 0.f && h_soc[e] <= 1.f)) return fail(CHX_EINVAL, "battery SoC out of [0,1]");
    CUDA_TRY(cudaDeviceSynchronize());
    RC(set_env_field(h, h_soc, h->b.bsoc));
    RC(set_env_field(h, h_p, h->b.bp));
    return CHX_OK;
}

extern "C" int chx_get_due(chx_handle* h, int16_t* h_due)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    CUDA_TRY(cudaDeviceSynchronize());
    RC(get_port_field(h, h_due, (const int16_t*)h->b.due));
    return CHX_OK;
}

extern "C" int chx_set_due(chx_handle* h, const int16_t* h_due)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    CUDA_TRY(cudaDeviceSynchronize());
    RC(set_port_field(h, h_due, h->b.due));
    return CHX_OK;
}

namespace {
constexpr uint64_t kCkptMagic = 0x43484158434B5034ull;   // "CHAXCKP4"
struct CkptHeader {
    uint64_t magic;
    int64_t n_envs, n_ports;
};
size_t ckpt_size(const chx_handle* h)
{
    return sizeof(CkptHeader) + (size_t)h->P * (5 * 4 + 1) + (size_t)h->E * (7 * 4 + 6 * 4 + 2 * 4) + (size_t)h->P * 2;
}
}  // namespace

extern "C" int chx_save(chx_handle* h, void* h_buf, size_t* size)
{
    if (!h || !size) return fail(CHX_EINVAL, "null argument");
    const size_t need = ckpt_size(h);
    if (!h_buf) {
        *size = need;
        return CHX_OK;
    }
    if (*size < need) return fail(CHX_EINVAL, "checkpoint buffer too small");
    const size_t P = h->P, E = h->E;
    char* w = static_cast<char*>(h_buf);
    CkptHeader hd{kCkptMagic, (int64_t)E, (int64_t)P};
    std::memcpy(w, &hd, sizeof hd);
    w += sizeof hd;
    float* f = reinterpret_cast<float*>(w);
    float *soc = f, *erem = f + P, *cap = f + 2 * P, *rbar = f + 3 * P, *pw = f + 4 * P;
    uint8_t* trem = reinterpret_cast<uint8_t*>(f + 5 * P);
    char* env = reinterpret_cast<char*>(trem + P);
    int32_t* tod = reinterpret_cast<int32_t*>(env);
    int32_t* day = tod + E;
    uint32_t* gstep = reinterpret_cast<uint32_t*>(day + E);
    uint32_t* ncar = gstep + E;
    uint32_t *key0 = ncar + E, *key1 = key0 + E;
    float* ret = reinterpret_cast<float*>(key1 + E);
    uint32_t* arrived = reinterpret_cast<uint32_t*>(ret + E);
    uint32_t* rejected = arrived + E;
    float* missing = reinterpret_cast<float*>(rejected + E);
    float* charged = missing + E;
    uint32_t* episodes = reinterpret_cast<uint32_t*>(charged + E);
    float* last = reinterpret_cast<float*>(episodes + E);
    float *bsoc = last + E, *bpw = bsoc + E;
    int16_t* due = reinterpret_cast<int16_t*>(bpw + E);
    RC(chx_get_state(h, soc, erem, cap, rbar, pw, trem, tod, day, gstep, ncar, key0, key1, ret));
    RC(chx_stats(h, arrived, rejected, missing, charged, episodes, last));
    RC(chx_get_battery(h, bsoc, bpw));
    RC(chx_get_due(h, due));
    *size = need;
    return CHX_OK;
}

extern "C" int chx_load(chx_handle* h, const void* h_buf, size_t size)
{
    if (!h || !h_buf) return fail(CHX_EINVAL, "null argument");
    if (size < ckpt_size(h)) return fail(CHX_EINVAL, "checkpoint too small");
    CkptHeader hd;
    std::memcpy(&hd, h_buf, sizeof hd);
    if (hd.magic != kCkptMagic || hd.n_envs != h->E || hd.n_ports != h->P)
        return fail(CHX_EINVAL, "checkpoint does not match this batch");
    const size_t P = h->P, E = h->E;
    const char* r = static_cast<const char*>(h_buf) + sizeof hd;
    const float* f = reinterpret_cast<const float*>(r);
    const uint8_t* trem = reinterpret_cast<const uint8_t*>(f + 5 * P);
    const char* env = reinterpret_cast<const char*>(trem + P);
    const int32_t* tod = reinterpret_cast<const int32_t*>(env);
    const int32_t* day = tod + E;
    const uint32_t* gstep = reinterpret_cast<const uint32_t*>(day + E);
    const uint32_t* ncar = gstep + E;
    const uint32_t *key0 = ncar + E, *key1 = key0 + E;
    const float* ret = reinterpret_cast<const float*>(key1 + E);
    const uint32_t* arrived = reinterpret_cast<const uint32_t*>(ret + E);
    const uint32_t* rejected = arrived + E;
    const float* missing = reinterpret_cast<const float*>(rejected + E);
    const float* charged = missing + E;
    const uint32_t* episodes = reinterpret_cast<const uint32_t*>(charged + E);
    const float* last = reinterpret_cast<const float*>(episodes + E);
    const float *bsoc = last + E, *bpw = bsoc + E;
    const int16_t* due = reinterpret_cast<const int16_t*>(bpw + E);
    RC(chx_set_state(h, f, f + P, f + 2 * P, f + 3 * P, f + 4 * P, trem, tod, day, gstep, ncar, key0, key1, ret));
    RC(set_env_field(h, bsoc, h->b.bsoc));
    RC(set_env_field(h, bpw, h->b.bp));
    RC(set_port_field(h, due, h->b.due));
    DevBatch& b = h->b;
    RC(set_env_field(h, arrived, b.st_arrived));
    RC(set_env_field(h, rejected, b.st_rejected));
    RC(set_env_field(h, missing, b.st_missing));
    RC(set_env_field(h, charged, b.st_charged));
    RC(set_env_field(h, episodes, b.n_episodes));
    RC(set_env_field(h, last, b.last_ret));
    return CHX_OK;
}

extern "C" int chx_check(chx_handle* h, void* stream)
{
    if (!h) return fail(CHX_EINVAL, "null handle");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t err = 0;
    CUDA_TRY(cudaMemcpy(&err, h->b.err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) {
        CUDA_TRY(cudaMemset(h->b.err, 0, sizeof(uint32_t)));
        if (err & kErrPolicyWait) return fail(CHX_ETIMEOUT, "a tensor-core wait of the policy kernel ran out of time");
        if (err & kErrEnvId) return fail(CHX_EFAULT, "a reset listed an env id outside 0..n_envs-1 (skipped)");
        return fail(CHX_EFAULT, "a kernel saw an action level outside 0..n_levels-1 (clamped)");
    }
    return CHX_OK;
}
