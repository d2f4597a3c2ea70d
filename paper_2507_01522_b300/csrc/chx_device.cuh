// chx_device.cuh -- device-side layout and arithmetic shared by the kernels
// of the charging-station step (sm_103a).
//
// State layout in HBM ("slot space").  Stations are bucketed by size class
// C in {8,16,32,64,128} (smallest power of two >= their charger count); a
// class stores its stations back to back, each padded to C charger slots,
// and its station count is padded to a multiple of 32/C for C < 32 so that
// a warp always owns whole stations.  Per-charger arrays are SoA float/u8,
// so a warp's 32*PPL consecutive chargers are one contiguous, aligned span
// (PPL = C/32 chargers per lane for C >= 64, loaded as float2/float4).
// Padding chargers and padding stations carry valid = 0 / user id -1.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace chx {

constexpr int kWarp = 32;
constexpr int kNumClasses = 5;             // 8, 16, 32, 64, 128
constexpr int kPoissonMax = 127;
constexpr int kCdfLen = 128;               // CDF entries per (row, step): F_0..F_126, then +inf
constexpr uint32_t kPurposeArrival = 0u, kPurposeCar = 1u, kPurposeAction = 2u, kPurposeDay = 3u;
constexpr uint32_t kPurposePolicy = 4u;   // policy sample: (env, step, charger / 4, 4), word charger % 4

// per-charger static bits
constexpr uint32_t kMetaDC = 1u, kMetaValid = 2u, kMetaHead = 4u, kMetaTail = 8u;
constexpr int kMetaGroupShift = 4;         // 5 bits: group slot within the warp tile (0..31)

// Warp tile shape of size class c (C = 8 << c chargers): chargers per lane,
// lanes per station and stations per warp.  Small stations take 2 chargers
// per lane so that a warp carries more of them and per-station work is
// shared by more chargers.
__host__ __device__ constexpr int tile_ppl(int c) { return c >= 4 ? 4 : 2; }
__host__ __device__ constexpr int tile_lpe(int c) { return (8 << c) / tile_ppl(c); }
__host__ __device__ constexpr int tile_epw(int c) { return 32 / tile_lpe(c); }

constexpr int kTremCS = 255;               // trem of a charger holding a charge-sensitive car
constexpr int kMaxUpperDepth = 3;          // levels of tree nodes above the groups

// device error bits
constexpr uint32_t kErrActionRange = 1u;
constexpr uint32_t kErrPolicyWait = 2u;     // a tensor-core wait of the policy kernel timed out
constexpr uint32_t kErrEnvId = 4u;          // a reset listed an env id outside 0..n_envs-1 (skipped)

struct DevParams {
    int ep_len, n_levels, n_days;
    float dt, inv_dt, tau, inv_1m_tau, p_sell, c_fixed, a_sat, a_decl, a_con, soc_target;
    float pmax0, pmax1, lvl0, lvl1;        // maximum power and power per level, per type
    float inv_eta0, inv_eta1;              // 1 / charger efficiency, per type
    float cap_lo, cap_span, soc_lo, soc_span;
    int stay_lo;
    uint32_t stay_span;
    float rb_lo0, rb_span0, rb_lo1, rb_span1;
    float obs_inv_stay, obs_inv_cap, obs_inv_days, obs_inv_len;
    float inv_pmax0, inv_pmax1;            // 1 / maximum power (FP32, correctly rounded), per type
    // vehicle-to-grid mode (signed levels, station battery)
    int v2g, half;                         // level k requests (k - half) * lvl: half = (n_levels - 1) / 2 in
                                           // V2G mode or the Delta form, else 0
    int delta;                             // Delta-current form: requests add to the last applied power
    float pdis0, pdis1;                    // discharge maximum I_max<- per type (V2G)
    // charge-sensitive users: u = 1 iff (first profile word & 0xFF) < cs_share
    int cs_share;                          // 0 = none (the mode is off)
    float a_sat1, beta, eps;               // weight of c_Sat,1, early-leave weight, "demand met" share of capacity
    int obs_port;                          // per-charger observation features: 6, or 7 with u
    int tree_levels;                       // levels of tree nodes above the groups (0 = none)
    float eta0, eta1;                      // charger efficiency per type (discharge losses)
    float batt_cap, inv_batt_cap, batt_rate, batt_lvl, batt_tau, batt_inv_1m_tau, batt_soc0;
    float sell_grid_ratio, a_degrad, obs_inv_batt_rate;
    int obs_env;                           // station features of an observation: 8, or 10 in V2G mode
};

struct DevBatch {
    // per charger slot
    float *soc, *erem, *cap, *rbar, *pw;
    uint8_t* trem;                         // remaining stay in steps, 0 = empty, kTremCS = charge-sensitive car
    int16_t* due;                          // Delta t_remain of a charge-sensitive car (cs_share > 0 only)
    // deeper trees (tree_levels > 0 only): level j (deepest first) of charger
    // i has head (bit 0), tail (bit 1) and node slot (bits 2-6) in byte j of
    // meta2[i]; its node's eta * I and 1 / eta at ucap / uinv[j * port_slots + i]
    uint32_t* meta2;
    float *ucap, *uinv;
    long long port_slots;
    uint32_t* meta;                        // kMeta* bits | group slot << 4
    float *gcap, *ginv_eta;                // eta_H * I_H of the charger's group, 1/eta_H
    // per station slot
    int32_t *user_id, *user_port_off, *n_ports, *arrival_class;
    float *grid_cap, *grid_inv_eta;        // eta_0 * I_0 of the root, 1/eta_0
    int32_t *tod, *day;
    uint32_t *gstep, *key0, *key1;
    uint32_t* ncar;                        // cars admitted since the last reset
    float *ep_ret, *last_ret;
    float *bsoc, *bp;                      // station battery (V2G mode): SoC, last applied power
    uint32_t* n_episodes;
    uint32_t *st_arrived, *st_rejected;
    float *st_missing, *st_charged;
    // exogenous tables
    const float* price;                    // [days][T] buy price
    const float* cdf;                      // [rows][T][kCdfLen] Poisson CDF of the arrival count
    // classes (index 0..4 = size 8..128)
    int cls_n_env[kNumClasses];            // padded station count
    int cls_env_base[kNumClasses];
    long long cls_port_base[kNumClasses];
    int n_slots;
    uint32_t* err;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): 10 rounds; each round
// multiplies counter words 0 and 2 by the Philox constants, crosses the high
// halves into the other words with the round key, and the key advances by the
// Weyl constants.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo_a = 0xD2511F53u * x.x, hi_a = __umulhi(0xD2511F53u, x.x);
        const uint32_t lo_b = 0xCD9E8D57u * x.z, hi_b = __umulhi(0xCD9E8D57u, x.z);
        x = make_uint4(hi_b ^ x.y ^ k0, lo_b, hi_a ^ x.w ^ k1, lo_a);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return x;
}

__device__ __forceinline__ uint32_t range_of(uint32_t w, uint32_t n) { return __umulhi(w, n); }
// uniform [0,1) from the top 24 bits, exact in FP32
__device__ __forceinline__ float unit_of(uint32_t w) { return __uint2float_rn(w >> 8) * 0x1p-24f; }

__device__ __forceinline__ uint32_t word_of(uint4 v, uint32_t i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// level of a random action from the 8-step Philox block of a charger
__device__ __forceinline__ int random_level(uint4 words, uint32_t g, int n_levels)
{
    const uint32_t w = word_of(words, (g >> 1) & 3u);
    const uint32_t half = (g & 1u) ? (w >> 16) : (w & 0xFFFFu);
    return (int)((half * (uint32_t)n_levels) >> 16);
}

// ---------------------------------------------------------------------------
// Poisson count by inverse transform: the smallest k with u < F_k, at most
// 127.  The count is an integer chosen by floating point, so F is defined by
// one exact sequence of correctly rounded FP32 operations (exp(-lambda) in
// double rounded once, p_k = (p_{k-1} * lambda) / k, F_k = F_{k-1} + p_k),
// evaluated on the host into a table per (arrival row, step of day) whose
// entry 127 is +inf; the kernel compares u against it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int poisson_count(const float* __restrict__ F, uint32_t w)
{
    const float u = __fmul_rn(__uint2float_rn(w >> 8), 0x1p-24f);
    int k = 0;
    while (u >= __ldg(F + k)) ++k;
    return k;
}

// taper r_hat(SoC): r_bar in the bulk stage, linear to 0 at SoC = 1 above tau
__device__ __forceinline__ float taper(float soc, float rbar, const DevParams& p)
{
    return soc <= p.tau ? rbar : (1.0f - soc) * rbar * p.inv_1m_tau;
}

// requested power of action level k (A.2 "Apply Actions", discretised):
// (k - half) * step, half = 0 for absolute charge-only levels; in the
// Delta-current form the increment adds to the last applied power
__device__ __forceinline__ float request(int level, float step, float last, const DevParams& p)
{
    const float a = (float)(level - p.half) * step;
    return p.delta ? last + a : a;
}

// the same with the form fixed at compile time (SIGNED: V2G or Delta form)
template <bool SIGNED, bool DELTA>
__device__ __forceinline__ float request_t(int level, float step, float last, const DevParams& p)
{
    const float a = (float)(SIGNED ? level - p.half : level) * step;
    return DELTA ? last + a : a;
}

// per-charger clip of Appendix A.2 "Apply Actions" (power form): requested
// power, car rate r_hat, charger maximum, SoC <= 1 and demand >= 0 caps,
// and 0 from below
__device__ __forceinline__ float clip_power(float preq, bool dc, float soc, float erem, float cap, float rbar,
                                            const DevParams& p)
{
    const float pmax = dc ? p.pmax1 : p.pmax0;
    const float rhat = taper(soc, rbar, p);
    const float soc_cap = (1.0f - soc) * cap * p.inv_dt;
    const float dem_cap = erem * p.inv_dt;
    float P = fminf(fminf(preq, rhat), fminf(fminf(pmax, soc_cap), dem_cap));
    return fmaxf(P, 0.0f);
}

// V2G clip (A.2 "Apply Actions", both branches) of a signed request:
// charging as clip_power, discharging limited by the request, the car's
// discharging rate (the charging curve flipped at SoC = 0.5: r_hat(1 - SoC)),
// the charger's discharge maximum I_max<- and SoC >= 0
__device__ __forceinline__ float clip_power_v2g(float preq, bool dc, float soc, float erem, float cap, float rbar,
                                                const DevParams& p)
{
    if (preq >= 0.f) {
        const float pmax = dc ? p.pmax1 : p.pmax0;
        const float rhat = taper(soc, rbar, p);
        const float soc_cap = (1.0f - soc) * cap * p.inv_dt;
        const float dem_cap = erem * p.inv_dt;
        return fmaxf(fminf(fminf(preq, rhat), fminf(fminf(pmax, soc_cap), dem_cap)), 0.0f);
    }
    // r_hat(1 - SoC) written without forming 1 - (1 - SoC) (cancellation in FP32)
    const float rdis = 1.0f - soc <= p.tau ? rbar : soc * rbar * p.inv_1m_tau;
    const float soc_cap = soc * cap * p.inv_dt;
    return -fmaxf(fminf(fminf(-preq, rdis), fminf(dc ? p.pdis1 : p.pdis0, soc_cap)), 0.0f);
}

// the station battery's power (V2G): the same two branches with its own
// rate curve and SoC in [0, 1]; it never leaves, so no demand cap
__device__ __forceinline__ float clip_battery(float preq, float bsoc, const DevParams& p)
{
    if (preq >= 0.f) {
        const float rhat = bsoc <= p.batt_tau ? p.batt_rate : (1.0f - bsoc) * p.batt_rate * p.batt_inv_1m_tau;
        return fmaxf(fminf(fminf(preq, rhat), (1.0f - bsoc) * p.batt_cap * p.inv_dt), 0.0f);
    }
    const float rdis = 1.0f - bsoc <= p.batt_tau ? p.batt_rate : bsoc * p.batt_rate * p.batt_inv_1m_tau;
    return -fmaxf(fminf(fminf(-preq, rdis), bsoc * p.batt_cap * p.inv_dt), 0.0f);
}

struct Car { float cap, soc, erem, rbar; int stay; bool cs; };

// Philox words of the station's n-th car since its last reset
__device__ __forceinline__ uint4 car_words(uint32_t uid, uint32_t n, uint32_t k0, uint32_t k1)
{
    return philox4x32_10(make_uint4(uid, n, 0u, kPurposeCar), k0, k1);
}

// the part of a car and user profile that does not depend on the charger
// the car parks at (capacity, SoC, demand, stay, user preference)
__device__ __forceinline__ Car car_core(uint4 w, const DevParams& p)
{
    Car c;
    c.cap = p.cap_lo + p.cap_span * unit_of(w.x);
    c.soc = p.soc_lo + p.soc_span * unit_of(w.y);
    c.stay = p.stay_lo + (int)range_of(w.z, p.stay_span);
    c.rbar = 0.f;
    c.erem = fmaxf(p.soc_target - c.soc, 0.0f) * c.cap;
    c.cs = (int)(w.x & 0xFFu) < p.cs_share;   // user preference: the low byte the capacity leaves unused
    return c;
}

// the car's maximum rate from its fourth profile word, at a charger of type dc
__device__ __forceinline__ float car_rbar(uint32_t w3, bool dc, const DevParams& p)
{
    return dc ? p.rb_lo1 + p.rb_span1 * unit_of(w3) : p.rb_lo0 + p.rb_span0 * unit_of(w3);
}

// car and user profile from its Philox words, at a charger of type dc
__device__ __forceinline__ Car car_from_words(uint4 w, bool dc, const DevParams& p)
{
    Car c = car_core(w, p);
    c.rbar = car_rbar(w.w, dc, p);
    return c;
}

__device__ __forceinline__ int draw_day(uint32_t uid, uint32_t c1, uint32_t c2, uint32_t k0, uint32_t k1, int n_days)
{
    const uint4 w = philox4x32_10(make_uint4(uid, c1, c2, kPurposeDay), k0, k1);
    return (int)range_of(w.x, (uint32_t)n_days);
}

// Philox words of a station's arrival draws: one call serves steps 4j..4j+3
__device__ __forceinline__ uint4 arrival_words(uint32_t uid, uint32_t g, uint32_t k0, uint32_t k1)
{
    return philox4x32_10(make_uint4(uid, g >> 2, 0u, kPurposeArrival), k0, k1);
}

// arrival count of step g from its Philox word
__device__ __forceinline__ int arrival_count(const DevBatch& b, const DevParams& p, uint32_t word, int t, int cls_row)
{
    const size_t row = ((size_t)cls_row * (size_t)p.ep_len + (size_t)t) * kCdfLen;
    return poisson_count(b.cdf + row, word);
}

__device__ __forceinline__ int arrivals(const DevBatch& b, const DevParams& p, uint32_t uid, uint32_t g, int t, int cls_row,
                                        uint32_t k0, uint32_t k1)
{
    return arrival_count(b, p, word_of(arrival_words(uid, g, k0, k1), g & 3u), t, cls_row);
}

// observation features of a station (p.obs_env floats: 8, + battery SoC and
// power / rate in V2G mode) and of one charger (6 floats)
__device__ __forceinline__ void obs_env_at(float* o, int t, int day, int occ, int n, float bsoc, float bpw,
                                           float price, const DevParams& p)
{
    float s, c;
    sincospif(2.0f * (float)t * p.obs_inv_len, &s, &c);
    o[0] = s;
    o[1] = c;
    o[2] = price;
    o[3] = p.p_sell;
    o[4] = (float)occ / (float)n;
    o[5] = (float)day * p.obs_inv_days;
    o[6] = (float)t * p.obs_inv_len;
    o[7] = (day % 7) < 5 ? 1.0f : 0.0f;
    if (p.v2g) {
        o[8] = bsoc;
        o[9] = bpw * p.obs_inv_batt_rate;
    }
}
// the same with the price of (day, t) read from the batch's price table
__device__ __forceinline__ void obs_env(float* o, int t, int day, int occ, int n, float bsoc, float bpw,
                                        const DevBatch& b, const DevParams& p)
{
    obs_env_at(o, t, day, occ, n, bsoc, bpw, __ldg(b.price + (size_t)day * (size_t)p.ep_len + (size_t)t), p);
}

// per-charger features (p.obs_port of them): occupied, SoC, stay / max stay
// (a charge-sensitive car's Delta t_remain), r_hat / P_max, last power /
// P_max, remaining demand / max capacity, and with charge-sensitive users u
// (CS = false: a caller that never runs with charge-sensitive users)
// feature x (0..5, as obs_port orders them) of a charger without a
// charge-sensitive user
__device__ __forceinline__ float obs_port_feature(int x, int trem, float soc, float erem, float rbar, float pw, bool dc,
                                                  const DevParams& p)
{
    const float inv_pmax = dc ? p.inv_pmax1 : p.inv_pmax0;
    const bool on = trem > 0;
    switch (x) {
        case 0: return on ? 1.0f : 0.0f;
        case 1: return soc;
        case 2: return (float)trem * p.obs_inv_stay;
        case 3: return on ? taper(soc, rbar, p) * inv_pmax : 0.0f;
        case 4: return pw * inv_pmax;
        default: return erem * p.obs_inv_cap;
    }
}

template <bool CS = true>
__device__ __forceinline__ void obs_port(float* o, int trem, int due, float soc, float erem, float rbar, float pw,
                                         bool dc, const DevParams& p)
{
    const float inv_pmax = dc ? p.inv_pmax1 : p.inv_pmax0;
    const bool on = trem > 0, cs = CS && trem == kTremCS && p.cs_share > 0;
    o[0] = on ? 1.0f : 0.0f;
    o[1] = soc;
    o[2] = (float)(cs ? due : trem) * p.obs_inv_stay;
    o[3] = on ? taper(soc, rbar, p) * inv_pmax : 0.0f;
    o[4] = pw * inv_pmax;
    o[5] = erem * p.obs_inv_cap;
    if (CS && p.obs_port == 7) o[6] = cs ? 1.0f : 0.0f;
}

// class of a station slot (classes are consecutive in slot space)
__device__ __forceinline__ int class_of_slot(const DevBatch& b, int s)
{
    int c = 0;
#pragma unroll
    for (int i = 1; i < kNumClasses; ++i)
        if (s >= b.cls_env_base[i]) c = i;
    return c;
}

// Start a new episode at station slot s with Philox key `seed` (the serving
// pool's reset, where a station's id is its slot; same start as chx_reset):
// the block's threads clear its chargers, thread 0 its station fields.
__device__ __forceinline__ void reset_one_slot(const DevBatch& b, const DevParams& p, int s, unsigned long long seed)
{
    const int c = class_of_slot(b, s);
    const int C = 8 << c;
    const long long pb = b.cls_port_base[c] + (long long)(s - b.cls_env_base[c]) * C;
    for (int q = threadIdx.x; q < C; q += blockDim.x) {
        const long long i = pb + q;
        b.soc[i] = 0.f; b.erem[i] = 0.f; b.cap[i] = 0.f; b.rbar[i] = 0.f; b.pw[i] = 0.f; b.trem[i] = 0;
        if (p.cs_share) b.due[i] = 0;      // the array exists only with charge-sensitive users
    }
    if (threadIdx.x == 0) {
        const uint32_t lo = (uint32_t)seed, hi = (uint32_t)(seed >> 32);
        b.key0[s] = lo;
        b.key1[s] = hi;
        b.gstep[s] = 0u;
        b.ncar[s] = 0u;
        b.tod[s] = 0;
        b.ep_ret[s] = 0.f;
        if (p.v2g) {  // the battery arrays exist only in V2G mode
            b.bsoc[s] = p.batt_soc0;
            b.bp[s] = 0.f;
        }
        b.day[s] = draw_day((uint32_t)s, 0u, 1u, lo, hi, p.n_days);
    }
}


}  // namespace chx
