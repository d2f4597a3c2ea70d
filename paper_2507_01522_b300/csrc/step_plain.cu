// step_plain.cu -- the plain form of the step: one thread per station, one
// launch per step, all state read from and written back to memory.
//
// It is the baseline the fused kernel is measured against and a second,
// structurally different CUDA implementation of the same transition
// (sequential per-station sums instead of warp reductions).
#include "chx_device.cuh"
#include "chx_kernels.h"

namespace chx {

// Four consecutive chargers of a station slot (slots start on a multiple of
// 8 chargers, so every chunk is 16-byte aligned for floats and words).
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
constexpr int kMaxPorts = 128;             // chargers per station slot at most
constexpr int kPlainThreads = 128;         // threads (stations) per block
__device__ __forceinline__ float& at(float4& v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }
__device__ __forceinline__ float get(const float4& v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }
__device__ __forceinline__ uint32_t get(const uint4& v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }

// One station's step.  V2G: signed levels (clip_power_v2g), the station
// battery at the root (its level after the chargers' in the action array, or
// drawn at charger index n), signed limits (|sum| <= eta * I), discharge
// energy after the port loss, two-case profit and degradation penalty.
//
// The chargers are walked in chunks of four with 16-byte loads, the next
// chunk loaded before the current one is used.  Pass (i) draws each
// charger's level once, clips it and keeps the clipped power in a per-thread
// array (local memory: consecutive threads' copies of one element are
// adjacent, so a warp's accesses are coalesced); the node passes and the
// charge pass read it from there.  Group scales live in this thread's column
// of a block-wide shared array (gscale[g * kPlainThreads]).  Sums run charger
// by charger in index order.
template <bool V2G>
__device__ __forceinline__ void step_station(const DevBatch& b, const DevParams& p, const int8_t* __restrict__ actions,
                                             long long lda, float* __restrict__ reward, uint8_t* __restrict__ done,
                                             int s, float* __restrict__ gscale)
{
    const int uid = b.user_id[s];
    if (uid < 0) return;
    const int c = class_of_slot(b, s);
    const int C = 8 << c;
    const long long pb = b.cls_port_base[c] + (long long)(s - b.cls_env_base[c]) * C;
    const int n = b.n_ports[s];
    const int nv = (n + 3) >> 2;                        // chunks of four chargers (inside the slot)
    const uint32_t g = b.gstep[s];
    const int t = b.tod[s];
    const uint32_t k0 = b.key0[s], k1 = b.key1[s];
    const long long aoff = b.user_port_off[s] + (V2G ? uid : 0);   // the station's first action

    auto level_of = [&](int q) -> int {                 // action level of charger q (q = n: battery)
        int lvl;
        if (actions) {
            lvl = actions[(aoff + q) * lda];
            if (lvl < 0 || lvl >= p.n_levels) {
                atomicOr(b.err, kErrActionRange);
                lvl = min(max(lvl, 0), p.n_levels - 1);
            }
        } else {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)uid, g >> 3, (uint32_t)q, kPurposeAction), k0, k1);
            lvl = random_level(w, g, p.n_levels);
        }
        return lvl;
    };

    // -- (i) apply actions: per-charger clip, then group sums (Eq. ArchConst)
    __align__(16) float Pst[kMaxPorts];                 // clipped (requested) power of each charger
    // gscale[g * kPlainThreads]: scale of group slot g (this thread's column
    // of a block-wide shared array: no bank conflicts, no local memory)
    float S = 0.f, Se = 0.f, Sn = 0.f, s_raw = 0.f, s_grp = 0.f, se_grp = 0.f, sn_grp = 0.f, over_max = 0.f;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint4 zu4 = make_uint4(0u, 0u, 0u, 0u);
    float4 xso = ld4(b.soc + pb), xer = ld4(b.erem + pb), xca = ld4(b.cap + pb), xrb = ld4(b.rbar + pb),
           xpl = ld4(b.pw + pb), xgc = ld4(b.gcap + pb), xgi = ld4(b.ginv_eta + pb);
    uint4 xme = __ldg(reinterpret_cast<const uint4*>(b.meta + pb));
    uint32_t xtr = *reinterpret_cast<const uint32_t*>(b.trem + pb);
    for (int v = 0; v < nv; ++v) {                      // chunk v + 1 is loaded before chunk v is computed
        const long long i0 = pb + 4 * v;
        const float4 so = xso, er = xer, ca = xca, rb = xrb, pl = xpl, gc4 = xgc, gi4 = xgi;
        const uint4 me = xme;
        const uint32_t tr4 = xtr;
        if (v + 1 < nv) {
            xso = ld4(b.soc + i0 + 4); xer = ld4(b.erem + i0 + 4); xca = ld4(b.cap + i0 + 4);
            xrb = ld4(b.rbar + i0 + 4); xpl = ld4(b.pw + i0 + 4);
            xgc = ld4(b.gcap + i0 + 4); xgi = ld4(b.ginv_eta + i0 + 4);   // group limits, read at group tails
            xme = __ldg(reinterpret_cast<const uint4*>(b.meta + i0 + 4));
            xtr = *reinterpret_cast<const uint32_t*>(b.trem + i0 + 4);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = 4 * v + j;
            if (q >= n) break;
            const uint32_t m = get(me, j);
            const bool dc = m & kMetaDC;
            float P = 0.f;
            if ((tr4 >> (8 * j)) & 0xFFu) {
                const float preq = request(level_of(q), dc ? p.lvl1 : p.lvl0, get(pl, j), p);
                P = V2G ? clip_power_v2g(preq, dc, get(so, j), get(er, j), get(ca, j), get(rb, j), p)
                        : clip_power(preq, dc, get(so, j), get(er, j), get(ca, j), get(rb, j), p);
            }
            Pst[q] = P;
            S += P;
            if (V2G) {
                if (P >= 0.f) Se += P * (dc ? p.inv_eta1 : p.inv_eta0);
                else Sn += P * (dc ? p.eta1 : p.eta0);
            } else {
                Se += P * (dc ? p.inv_eta1 : p.inv_eta0);
            }
            s_raw += P;
            if (m & kMetaTail) {
                const float gc = get(gc4, j);
                const float mag = V2G ? fabsf(S) : S;
                const float sc = mag > gc ? __fdividef(gc, mag) : 1.0f;
                gscale[((m >> kMetaGroupShift) & 31) * kPlainThreads] = sc;
                over_max = fmaxf(over_max, (mag - gc) * get(gi4, j));
                s_grp += S * sc;
                se_grp += Se * sc;
                sn_grp += Sn * sc;
                S = 0.f;
                Se = 0.f;
                Sn = 0.f;
            }
        }
    }
    // deeper trees: the nodes above the groups, level by level (deepest
    // first), each node rescaling its chargers' (already group-rescaled)
    // power; then the root sums over the fully rescaled powers
    float uscale[kMaxUpperDepth][32];
    const int TL = p.tree_levels;
    auto upper_mult = [&](long long i, int levels) -> float {
        float f = 1.f;
        for (int j = 0; j < levels; ++j) f *= uscale[j][(b.meta2[i] >> (8 * j + 2)) & 31u];
        return f;
    };
    if (TL > 0) {
        for (int j = 0; j < TL; ++j) {
            float Su = 0.f, Sr = 0.f;
            for (int q = 0; q < n; ++q) {
                const long long i = pb + q;
                const uint32_t m = b.meta[i], m2 = b.meta2[i] >> (8 * j);
                const float Pr = Pst[q];
                if (m2 & 1u) {
                    Su = 0.f;
                    Sr = 0.f;
                }
                Su += Pr * gscale[((m >> kMetaGroupShift) & 31) * kPlainThreads] * upper_mult(i, j);
                Sr += Pr;
                if (m2 & 2u) {
                    const float cap_u = b.ucap[(long long)j * b.port_slots + i];
                    const float mag = V2G ? fabsf(Su) : Su;
                    uscale[j][(m2 >> 2) & 31u] = mag > cap_u ? __fdividef(cap_u, mag) : 1.0f;
                    over_max = fmaxf(over_max, ((V2G ? fabsf(Sr) : Sr) - cap_u) * b.uinv[(long long)j * b.port_slots + i]);
                }
            }
        }
        s_grp = 0.f;
        se_grp = 0.f;
        sn_grp = 0.f;
        for (int q = 0; q < n; ++q) {
            const long long i = pb + q;
            if (b.trem[i] == 0) continue;
            const uint32_t m = b.meta[i];
            const bool dc = m & kMetaDC;
            const float P = Pst[q] * gscale[((m >> kMetaGroupShift) & 31) * kPlainThreads] * upper_mult(i, TL);
            s_grp += P;
            if (V2G) {
                if (P >= 0.f) se_grp += P * (dc ? p.inv_eta1 : p.inv_eta0);
                else sn_grp += P * (dc ? p.eta1 : p.eta0);
            } else {
                se_grp += P * (dc ? p.inv_eta1 : p.inv_eta0);
            }
        }
    }

    // station battery (a leaf of the root), then the root node
    float Pb = 0.f, bsoc = 0.f;
    if (V2G) {
        bsoc = b.bsoc[s];
        Pb = clip_battery(request(level_of(n), p.batt_lvl, b.bp[s], p), bsoc, p);
    }
    const float grid_cap = b.grid_cap[s];
    const float s_tot = s_grp + Pb, mag = V2G ? fabsf(s_tot) : s_tot;
    const float s_root = mag > grid_cap ? __fdividef(grid_cap, mag) : 1.0f;
    const float raw = V2G ? fabsf(s_raw + Pb) : s_raw;
    const float c_con = fmaxf(fmaxf(over_max, (raw - grid_cap) * b.grid_inv_eta[s]), 0.0f);

    // -- (ii) charge, time advance, (iii) departures; chunk v + 1 is loaded
    // before chunk v is stored
    float c_sat = 0.f, c_sat1 = 0.f;
    int n_free = 0;
    unsigned long long free_lo = 0ull, free_hi = 0ull;  // free chargers 0-63, 64-127
    float4 so = z4, er = z4, ca = z4, ps = z4;
    uint4 me = zu4;
    uint32_t tr4 = 0;
    if (nv > 0) {
        so = ld4(b.soc + pb); er = ld4(b.erem + pb); ca = ld4(b.cap + pb);
        ps = *reinterpret_cast<const float4*>(Pst);
        me = __ldg(reinterpret_cast<const uint4*>(b.meta + pb));
        tr4 = *reinterpret_cast<const uint32_t*>(b.trem + pb);
    }
    for (int v = 0; v < nv; ++v) {
        const long long i0 = pb + 4 * v;
        float4 so1 = z4, er1 = z4, ca1 = z4, ps1 = z4;
        uint4 me1 = zu4;
        uint32_t tr41 = 0;
        if (v + 1 < nv) {
            so1 = ld4(b.soc + i0 + 4); er1 = ld4(b.erem + i0 + 4); ca1 = ld4(b.cap + i0 + 4);
            ps1 = *reinterpret_cast<const float4*>(Pst + 4 * v + 4);
            me1 = __ldg(reinterpret_cast<const uint4*>(b.meta + i0 + 4));
            tr41 = *reinterpret_cast<const uint32_t*>(b.trem + i0 + 4);
        }
        float4 pw4 = make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t tr_out = tr4;
        bool any_leave = false;
        uint32_t leave_bits = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = 4 * v + j;
            if (q >= n) break;
            const long long i = i0 + j;
            const uint32_t m = get(me, j);
            int tr = (tr4 >> (8 * j)) & 0xFFu;
            float P = 0.f;
            if (tr > 0) {
                float soc = at(so, j), erem = at(er, j);
                const float cap = at(ca, j);
                P = get(ps, j) * gscale[((m >> kMetaGroupShift) & 31) * kPlainThreads];
                if (TL > 0) P *= upper_mult(i, TL);
                P *= s_root;
                const float dE = P * p.dt;
                soc = fminf(soc + __fdividef(dE, cap), 1.0f);
                if (V2G) soc = fmaxf(soc, 0.0f);
                erem = fmaxf(erem - dE, 0.0f);
                bool leave;
                if (p.cs_share && tr == kTremCS) {
                    // charge-sensitive: one step nearer the desired departure;
                    // leaves once the demand is met (c_Sat,1: overdue - beta early)
                    const int d = (int)b.due[i] - 1;
                    leave = erem <= p.eps * cap;     // demand met: target SoC within eps
                    if (leave) {
                        c_sat1 += (float)max(-d, 0) - p.beta * (float)max(d, 0);
                        tr = 0;
                        b.due[i] = 0;
                    } else {
                        b.due[i] = (int16_t)d;
                    }
                } else {
                    tr -= 1;
                    leave = tr == 0;
                    if (leave) c_sat += erem;
                }
                if (leave) {
                    soc = 0.f;
                    erem = 0.f;
                    at(ca, j) = 0.f;
                    leave_bits |= 1u << j;
                    any_leave = true;
                }
                at(so, j) = soc;
                at(er, j) = erem;
                tr_out = (tr_out & ~(0xFFu << (8 * j))) | ((uint32_t)tr << (8 * j));
            }
            // Delta form: a departed car's charger drops to 0, the next car's base
            at(pw4, j) = (p.delta && tr == 0) ? 0.f : P;
            if (tr == 0) {
                ++n_free;
                if (q < 64) free_lo |= 1ull << q;
                else free_hi |= 1ull << (q - 64);
            }
        }
        st4(b.soc + i0, so);
        st4(b.erem + i0, er);
        st4(b.pw + i0, pw4);
        *reinterpret_cast<uint32_t*>(b.trem + i0) = tr_out;
        if (any_leave) {
            st4(b.cap + i0, ca);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (leave_bits & (1u << j)) b.rbar[i0 + j] = 0.f;
        }
        so = so1; er = er1; ca = ca1; ps = ps1; me = me1; tr4 = tr41;
    }
    const float e_net = s_grp * s_root * p.dt;
    const float e_grid = se_grp * s_root * p.dt;
    float e_to = 0.f, e_b = 0.f;
    if (V2G) {
        e_to = sn_grp * s_root * p.dt;
        const float pb_applied = Pb * s_root;
        e_b = pb_applied * p.dt;
        b.bsoc[s] = fminf(fmaxf(bsoc + e_b * p.inv_batt_cap, 0.0f), 1.0f);
        b.bp[s] = pb_applied;
    }

    // -- (iv) arrivals: Poisson count, first come first served (free chargers
    // in ascending index)
    const int M = arrivals(b, p, (uint32_t)uid, g, t, b.arrival_class[s], k0, k1);
    const int m_adm = min(M, n_free);
    const uint32_t ncar = b.ncar[s];
    for (int w = 0, j = 0; w < 2 && j < m_adm; ++w) {
        unsigned long long fm = w == 0 ? free_lo : free_hi;
        while (fm && j < m_adm) {
            const int q = 64 * w + __ffsll((long long)fm) - 1;
            fm &= fm - 1;
            const long long i = pb + q;
            const Car car = car_from_words(car_words((uint32_t)uid, ncar + (uint32_t)j, k0, k1), b.meta[i] & kMetaDC, p);
            b.cap[i] = car.cap; b.soc[i] = car.soc; b.erem[i] = car.erem; b.rbar[i] = car.rbar;
            if (car.cs) {                  // charge-sensitive user: stays until charged
                b.trem[i] = (uint8_t)kTremCS;
                b.due[i] = (int16_t)car.stay;
            } else {
                b.trem[i] = (uint8_t)car.stay;
            }
            ++j;
        }
    }

    // -- reward, Appendix A.3: E_grid,net = bought + pushed into the grid + battery
    const float price = __ldg(b.price + (size_t)b.day[s] * (size_t)p.ep_len + (size_t)t);
    float r;
    if (V2G) {
        const float e_gn = e_grid + e_to + e_b;
        const float pg = e_gn > 0.f ? price : p.sell_grid_ratio * price;
        const float degrad = fmaxf(-e_b, 0.0f) - e_to;
        r = p.p_sell * e_net - pg * e_gn - p.c_fixed - p.a_sat * c_sat - p.a_decl * (float)(M - m_adm) -
            p.a_con * c_con - p.a_degrad * degrad;
    } else {
        const float profit = p.p_sell * e_net - price * e_grid - p.c_fixed;
        r = profit - p.a_sat * c_sat - p.a_decl * (float)(M - m_adm) - p.a_con * c_con;
    }
    if (p.cs_share) r -= p.a_sat1 * c_sat1;

    b.ncar[s] = ncar + (uint32_t)m_adm;
    b.st_arrived[s] += (uint32_t)m_adm;
    b.st_rejected[s] += (uint32_t)(M - m_adm);
    b.st_missing[s] += c_sat;
    b.st_charged[s] += e_net;
    float ret = b.ep_ret[s] + r;
    int t1 = t + 1;
    uint8_t fin = 0;
    if (t1 >= p.ep_len) {
        fin = 1;
        b.last_ret[s] = ret;
        ret = 0.f;
        b.n_episodes[s] += 1u;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = 0; q < C; q += 4) {
            const long long i = pb + q;
            st4(b.soc + i, z); st4(b.erem + i, z); st4(b.cap + i, z); st4(b.rbar + i, z); st4(b.pw + i, z);
            *reinterpret_cast<uint32_t*>(b.trem + i) = 0u;
            if (p.cs_share) *reinterpret_cast<uint2*>(b.due + i) = make_uint2(0u, 0u);
        }
        if (V2G) {
            b.bsoc[s] = p.batt_soc0;
            b.bp[s] = 0.f;
        }
        t1 = 0;
        b.day[s] = draw_day((uint32_t)uid, g, 0u, k0, k1, p.n_days);
    }
    b.ep_ret[s] = ret;
    b.tod[s] = t1;
    b.gstep[s] = g + 1u;
    if (reward) reward[uid] = r;
    if (done) done[uid] = fin;
}

template <bool V2G>
__global__ void __launch_bounds__(kPlainThreads) k_step_plain(DevBatch b, DevParams p, const int8_t* __restrict__ actions,
                                                    long long lda, float* __restrict__ reward,
                                                    uint8_t* __restrict__ done, const int* __restrict__ slot_list,
                                                    int n_list)
{
    __shared__ float gscale[32 * kPlainThreads];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (slot_list ? n_list : b.n_slots)) return;
    step_station<V2G>(b, p, actions, lda, reward, done, slot_list ? slot_list[idx] : idx, gscale + threadIdx.x);
}

void launch_step_plain(const DevBatch& b, const DevParams& p, const int8_t* actions, long long lda, float* reward,
                       uint8_t* done, const int* slot_list, int n_list, cudaStream_t st)
{
    const int n = slot_list ? n_list : b.n_slots;
    if (n <= 0) return;
    const int threads = kPlainThreads;
    if (p.v2g)
        k_step_plain<true><<<(n + threads - 1) / threads, threads, 0, st>>>(b, p, actions, lda, reward, done, slot_list,
                                                                              n_list);
    else
        k_step_plain<false><<<(n + threads - 1) / threads, threads, 0, st>>>(b, p, actions, lda, reward, done,
                                                                               slot_list, n_list);
}

}  // namespace chx
