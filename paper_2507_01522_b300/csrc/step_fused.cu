// step_fused.cu -- the fused form of the step: K transitions per launch.
//
// A persistent kernel.  Each warp repeatedly takes a tile from a global work
// counter (tiles of the largest stations first), loads the tile's state into
// registers, runs K steps without touching HBM except for the per-step
// reward/done outputs, and stores the state back.  A lane holds PPL
// consecutive chargers of one station (PPL = 2 for the classes of 8..64
// chargers, 4 for 128), so a tile is 32 * PPL charger slots: 8, 4, 2 or 1
// stations of 8, 16, 32 or 64 chargers, or one station of 128.
//
// Reductions over chargers (Eq. ArchConst and the reward sums) are warp
// shuffles: a segmented inclusive scan gives each group node's power at its
// last charger, whose scale is broadcast through 32 floats of shared memory;
// station totals use an xor butterfly inside the station's aligned lane
// segment.  Both depend only on a charger's position inside its station, so a
// station's result does not depend on which tile or lane offset it runs in.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <type_traits>

#include "chx_device.cuh"
#include "chx_kernels.h"

namespace chx {

template <int C>
struct Shape {
    static constexpr int CI = C == 8 ? 0 : (C == 16 ? 1 : (C == 32 ? 2 : (C == 64 ? 3 : 4)));
    static constexpr int PPL = tile_ppl(CI);         // chargers per lane
    static constexpr int LPE = tile_lpe(CI);         // lanes per station
    static constexpr int EPW = tile_epw(CI);         // stations per warp
};

template <int N>
__device__ __forceinline__ void ld_vec(const float* src, float (&d)[N])
{
    if constexpr (N == 1) {
        d[0] = src[0];
    } else if constexpr (N == 2) {
        const float2 v = *reinterpret_cast<const float2*>(src);
        d[0] = v.x; d[1] = v.y;
    } else {
        const float4 v = *reinterpret_cast<const float4*>(src);
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    }
}
template <int N>
__device__ __forceinline__ void st_vec(float* dst, const float (&d)[N])
{
    if constexpr (N == 1) {
        dst[0] = d[0];
    } else if constexpr (N == 2) {
        *reinterpret_cast<float2*>(dst) = make_float2(d[0], d[1]);
    } else {
        *reinterpret_cast<float4*>(dst) = make_float4(d[0], d[1], d[2], d[3]);
    }
}
template <int N>
__device__ __forceinline__ void ld_vec_u32(const uint32_t* src, uint32_t (&d)[N])
{
    if constexpr (N == 1) {
        d[0] = src[0];
    } else if constexpr (N == 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(src);
        d[0] = v.x; d[1] = v.y;
    } else {
        const uint4 v = *reinterpret_cast<const uint4*>(src);
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    }
}
template <int N>
__device__ __forceinline__ void ld_u8(const uint8_t* src, int (&d)[N])
{
    if constexpr (N == 1) {
        d[0] = src[0];
    } else if constexpr (N == 2) {
        const uint16_t v = *reinterpret_cast<const uint16_t*>(src);
        d[0] = v & 0xFF; d[1] = v >> 8;
    } else {
        const uint32_t v = *reinterpret_cast<const uint32_t*>(src);
        d[0] = v & 0xFF; d[1] = (v >> 8) & 0xFF; d[2] = (v >> 16) & 0xFF; d[3] = v >> 24;
    }
}
template <int N>
__device__ __forceinline__ void ld_i16(const int16_t* src, int (&d)[N])
{
    if constexpr (N == 1) {
        d[0] = src[0];
    } else if constexpr (N == 2) {
        const uint32_t v = *reinterpret_cast<const uint32_t*>(src);
        d[0] = (int16_t)(v & 0xFFFFu); d[1] = (int16_t)(v >> 16);
    } else {
        const uint2 v = *reinterpret_cast<const uint2*>(src);
        d[0] = (int16_t)(v.x & 0xFFFFu); d[1] = (int16_t)(v.x >> 16);
        d[2] = (int16_t)(v.y & 0xFFFFu); d[3] = (int16_t)(v.y >> 16);
    }
}
template <int N>
__device__ __forceinline__ void st_i16(int16_t* dst, const int (&d)[N])
{
    if constexpr (N == 1) {
        dst[0] = (int16_t)d[0];
    } else if constexpr (N == 2) {
        *reinterpret_cast<uint32_t*>(dst) = (uint32_t)(d[0] & 0xFFFF) | ((uint32_t)d[1] << 16);
    } else {
        *reinterpret_cast<uint2*>(dst) = make_uint2((uint32_t)(d[0] & 0xFFFF) | ((uint32_t)d[1] << 16),
                                                    (uint32_t)(d[2] & 0xFFFF) | ((uint32_t)d[3] << 16));
    }
}
template <int N>
__device__ __forceinline__ void st_u8(uint8_t* dst, const int (&d)[N])
{
    if constexpr (N == 1) {
        dst[0] = (uint8_t)d[0];
    } else if constexpr (N == 2) {
        *reinterpret_cast<uint16_t*>(dst) = (uint16_t)(d[0] | (d[1] << 8));
    } else {
        *reinterpret_cast<uint32_t*>(dst) = (uint32_t)(d[0] | (d[1] << 8) | (d[2] << 16) | (d[3] << 24));
    }
}

// sum over the LPE lanes of a station (aligned segment), identical in all of them
template <int LPE>
__device__ __forceinline__ float seg_sum(float v)
{
#pragma unroll
    for (int o = LPE / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
template <int LPE>
__device__ __forceinline__ float seg_max(float v)
{
#pragma unroll
    for (int o = LPE / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

// Distance, in lanes, from this lane back to the lane holding the head of the
// group that this lane's last charger belongs to (0 if that head is in this
// lane).  Groups are static, so this is computed once per tile: a prefix
// maximum of "this lane holds a head" over the station's lanes.
template <int PPL, int LPE>
__device__ __forceinline__ int head_distance(const uint32_t (&meta)[PPL], int le)
{
    bool any_head = false;
#pragma unroll
    for (int q = 0; q < PPL; ++q) any_head = any_head || (meta[q] & kMetaHead);
    int hl = any_head ? le : 0;            // lane 0 of a station always holds a head
#pragma unroll
    for (int d = 1; d < LPE; d <<= 1) {
        const int o = __shfl_up_sync(0xFFFFFFFFu, hl, d);
        if (le >= d) hl = max(hl, o);
    }
    return le - hl;
}

// Inclusive segmented scan of v over the chargers of the warp in charger
// order (lane-major, PPL per lane); a head bit starts a new group.  The lane
// aggregates are scanned with the static head distance dh: in the round of
// offset d a lane adds the partial of lane - d only while d <= dh, which keeps
// every sum inside its group (and its station).
template <int PPL, int LPE>
__device__ __forceinline__ void seg_scan(float (&v)[PPL], const uint32_t (&meta)[PPL], int le, int dh)
{
#pragma unroll
    for (int q = 1; q < PPL; ++q)
        if (!(meta[q] & kMetaHead)) v[q] += v[q - 1];
    float x = v[PPL - 1];
#pragma unroll
    for (int d = 1; d < LPE; d <<= 1) {
        const float xu = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (d <= dh) x += xu;
    }
    if constexpr (PPL == 1) {
        v[0] = x;
    } else {
        float carry = __shfl_up_sync(0xFFFFFFFFu, x, 1);
        if (le == 0) carry = 0.f;
        bool seen = false;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            seen = seen || (meta[q] & kMetaHead);
            if (!seen) v[q] += carry;
        }
    }
}

// Poisson count (see poisson_count) searched by the station's lanes in
// parallel: lane le tests CDF entry base + le; the entries <= u form a prefix
// because the CDF is nondecreasing, so their number is the count.
template <int LPE>
__device__ __forceinline__ int poisson_count_warp(const float* __restrict__ F, uint32_t w, int le, unsigned env_mask)
{
    const float u = __fmul_rn(__uint2float_rn(w >> 8), 0x1p-24f);
    int M = 0;
    bool more = true;
#pragma unroll 1
    for (int base = 0; base < kCdfLen; base += LPE) {
        const bool ok = more && u >= __ldg(F + base + le);
        const int cnt = __popc(__ballot_sync(0xFFFFFFFFu, ok) & env_mask);
        if (more) {
            M = base + cnt;
            more = cnt == LPE;
        }
        if (!__any_sync(0xFFFFFFFFu, more)) break;
    }
    return M;
}

// Per-warp shared memory: group scales and limits by group slot, the running
// statistics of the warp's stations, and the Philox action words of its
// chargers (kept here instead of registers).
struct WarpSmem {
    float scale[64];                       // group slots: station ew's group g at ew * min(C, 32) + g
    float gcap[64];
    float ginv[64];
    float st_f[8][4];                      // per station: missing kWh, charged kWh, last return
    uint32_t st_u[8][4];                   // per station: admitted, rejected, episodes, episode ended
    uint32_t arrw[4][32];                  // arrival words: word w of block (blk0 + x - station's first lane) at [w][x]
    uint32_t aw[4][32 * 4];                // action words: word w of charger slot q*32 + lane
    uint32_t carw[5][128];                 // pre-drawn cars, station ew's i-th buffered car at ew*C + i:
                                           // capacity, SoC, demand (FP32 bits), stay | u << 8, rate word
};

// extended instances: also the nodes above the groups, per level, at the
// group slots' indexing (station ew's node slot k at ew * min(C, 32) + k)
struct WarpSmemExt : WarpSmem {
    float ucap[kMaxUpperDepth][64];
    float uinv[kMaxUpperDepth][64];
    float uscale[kMaxUpperDepth][64];
    uint32_t m2[4][32];                    // per lane: its chargers' meta2 words
    int dhu[kMaxUpperDepth][32];           // per lane: head distance at each level
};

// level j's byte of meta2 in the layout of the group bits of meta
__device__ __forceinline__ uint32_t level_meta(uint32_t m2, int j)
{
    const uint32_t b8 = (m2 >> (8 * j)) & 0xFFu;
    return ((b8 & 1u) ? kMetaHead : 0u) | ((b8 & 2u) ? kMetaTail : 0u) | (((b8 >> 2) & 31u) << kMetaGroupShift);
}

// A given action level: action slot a at step k of the launch (int8, or a
// nibble of two-per-byte packed levels)
__device__ __forceinline__ int given_level(const FusedIO& io, long long a, int k)
{
    const long long i = a * io.lda + (long long)k * io.lda_step;
    if (io.act_bits == 4) {
        const uint32_t byte = reinterpret_cast<const uint8_t*>(io.actions)[i >> 1];
        return (int)((i & 1) ? byte >> 4 : byte & 15u);
    }
    return io.actions[i];
}

// V2G: signed levels, the station battery at the root (state in the
// station's lanes, its level after the chargers' or drawn at charger index
// n), signed limits, discharge energy after the port loss, two-case profit,
// degradation penalty; observation with the battery features.
template <int C, bool V2G, bool EXT, bool TREE, class SM>
__device__ __forceinline__ void run_tile(const DevBatch& b, const DevParams& p, const FusedIO& io, int tile,
                                         SM* ws)
{
    using S = Shape<C>;
    constexpr int PPL = S::PPL, LPE = S::LPE;
    constexpr int GPS = C < 32 ? C : 32;   // group slots per station (at most 32 groups)
    constexpr int CI = C == 8 ? 0 : (C == 16 ? 1 : (C == 32 ? 2 : (C == 64 ? 3 : 4)));
    const int lane = threadIdx.x & 31;
    const int ew = lane / LPE;            // station within the warp
    const int le = lane % LPE;            // lane within the station
    // the station this lane works on: the tile's own slots, or (gather mode)
    // the slots a caller listed, with their own action/output/observation offsets
    int s, act_base, out_idx, obs_w = 0;
    if (io.gather) {
        const int4 en = io.gather[io.gather_base[CI] + tile * S::EPW + ew];
        s = en.x;
        act_base = en.y;
        out_idx = en.z;
        obs_w = en.w;
    } else {
        s = b.cls_env_base[CI] + tile * S::EPW + ew;
        act_base = b.user_port_off[s];
        out_idx = b.user_id[s];
        if (V2G) act_base += out_idx;     // one more action (the battery's) per station before this one
    }
    const long long pb = b.cls_port_base[CI] + (long long)(s - b.cls_env_base[CI]) * C + le * PPL;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned env_mask = (LPE == 32) ? 0xFFFFFFFFu : (((1u << LPE) - 1u) << (ew * LPE));

    // per-station state (identical in the station's lanes)
    const int uid = b.user_id[s];
    const bool live = uid >= 0;
    const uint32_t uidu = (uint32_t)(live ? uid : 0);
    const int cls_row = b.arrival_class[s];
    const float grid_cap = b.grid_cap[s];
    const uint32_t k0 = b.key0[s], k1 = b.key1[s];
    int t = b.tod[s], day = b.day[s];
    uint32_t g = b.gstep[s];
    float ret = b.ep_ret[s];
    // station battery (V2G): the same values in all the station's lanes
    float bsoc = 0.f, bpw = 0.f;
    uint4 bwords = make_uint4(0, 0, 0, 0);
    if (V2G) {
        bsoc = b.bsoc[s];
        bpw = b.bp[s];
    }
    // cars: the station's next C car profiles are drawn in one lane-parallel
    // pass into shared memory and handed out as cars arrive
    uint32_t ncar = b.ncar[s], cend = ncar;

    // per-charger state
    float soc[PPL], erem[PPL], cap[PPL], rbar[PPL], pw[PPL];
    int trem[PPL];
    uint32_t meta[PPL];
    ld_vec(b.soc + pb, soc);
    ld_vec(b.erem + pb, erem);
    ld_vec(b.cap + pb, cap);
    ld_vec(b.rbar + pb, rbar);
    ld_vec(b.pw + pb, pw);
    ld_u8(b.trem + pb, trem);
    // charge-sensitive users (EXT instances): Delta t_remain per charger
    const bool cs_on = EXT && p.cs_share > 0;
    int due[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) due[q] = 0;
    if (cs_on) ld_i16(b.due + pb, due);
    ld_vec_u32(b.meta + pb, meta);
    {
        float gc[PPL], gi[PPL];
        ld_vec(b.gcap + pb, gc);
        ld_vec(b.ginv_eta + pb, gi);
#pragma unroll
        for (int q = 0; q < PPL; ++q)
            if (meta[q] & kMetaTail) {
                const int gs = ew * GPS + (int)((meta[q] >> kMetaGroupShift) & 31u);
                ws->gcap[gs] = gc[q];
                ws->ginv[gs] = gi[q];
            }
    }
    if (le == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ws->st_f[ew][i] = 0.f;
            ws->st_u[ew][i] = 0u;
        }
    }
    // deeper trees (extended instances): per level the chargers' node bits,
    // its head distance, and the nodes' limits at their tails
    // (kept in shared memory per lane: live for the whole tile)
    const int TL = TREE ? p.tree_levels : 0;
    if constexpr (TREE) {
        if (TL > 0) {
            uint32_t m2[PPL];
            ld_vec_u32(b.meta2 + pb, m2);
#pragma unroll
            for (int q = 0; q < PPL; ++q) ws->m2[q][lane] = m2[q];
#pragma unroll
            for (int j = 0; j < kMaxUpperDepth; ++j) {
                if (j >= TL) break;
                uint32_t lm[PPL];
#pragma unroll
                for (int q = 0; q < PPL; ++q) {
                    lm[q] = level_meta(m2[q], j);
                    if (lm[q] & kMetaTail) {
                        const int us = ew * GPS + (int)((lm[q] >> kMetaGroupShift) & 31u);
                        ws->ucap[j][us] = b.ucap[(long long)j * b.port_slots + pb + q];
                        ws->uinv[j][us] = b.uinv[(long long)j * b.port_slots + pb + q];
                    }
                }
                ws->dhu[j][lane] = head_distance<PPL, LPE>(lm, le);
            }
        }
    }
    __syncwarp();
    const bool random_actions = io.actions == nullptr || act_base < 0;
    const int dh = head_distance<PPL, LPE>(meta, le);
    // Arrival words are prefetched lane-parallel: lane le of a station holds the
    // Philox block (blk0 + le), i.e. the words of steps 4*(blk0+le)..+3, so one
    // pass covers 4*LPE steps.
    uint32_t blk0 = 0;

    for (int k = 0; k < io.k_steps; ++k) {
        // ---- (i) apply actions: per-charger clip
        float P[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            const int port = le * PPL + q;
            int lvl = 0;
            if (random_actions) {
                const int j = q * 32 + lane;
                if (k == 0 || (g & 7u) == 0u) {
                    const uint4 w = philox4x32_10(make_uint4(uidu, g >> 3, (uint32_t)port, kPurposeAction), k0, k1);
                    ws->aw[0][j] = w.x;
                    ws->aw[1][j] = w.y;
                    ws->aw[2][j] = w.z;
                    ws->aw[3][j] = w.w;
                }
                const uint32_t word = ws->aw[(g >> 1) & 3u][j];
                const uint32_t half = (g & 1u) ? (word >> 16) : (word & 0xFFFFu);
                lvl = (int)((half * (uint32_t)p.n_levels) >> 16);
            } else if (trem[q] > 0) {
                lvl = given_level(io, (long long)act_base + port, k);
                if (lvl < 0 || lvl >= p.n_levels) {
                    atomicOr(b.err, kErrActionRange);
                    lvl = min(max(lvl, 0), p.n_levels - 1);
                }
            }
            const bool dc = meta[q] & kMetaDC;
            const float preq = EXT ? request(lvl, dc ? p.lvl1 : p.lvl0, pw[q], p)
                                   : request_t<V2G, false>(lvl, dc ? p.lvl1 : p.lvl0, pw[q], p);
            if (V2G)
                P[q] = trem[q] > 0 ? clip_power_v2g(preq, dc, soc[q], erem[q], cap[q], rbar[q], p) : 0.f;
            else
                P[q] = trem[q] > 0 ? clip_power(preq, dc, soc[q], erem[q], cap[q], rbar[q], p) : 0.f;
        }
        // the battery's request (V2G; computed alike in every lane of the station)
        float Pb = 0.f;
        if (V2G) {
            const int n_st = b.n_ports[s];
            int lvl;
            if (random_actions) {
                if (k == 0 || (g & 7u) == 0u)
                    bwords = philox4x32_10(make_uint4(uidu, g >> 3, (uint32_t)n_st, kPurposeAction), k0, k1);
                lvl = random_level(bwords, g, p.n_levels);
            } else {
                lvl = given_level(io, (long long)act_base + n_st, k);
                if (lvl < 0 || lvl >= p.n_levels) {
                    atomicOr(b.err, kErrActionRange);
                    lvl = min(max(lvl, 0), p.n_levels - 1);
                }
            }
            Pb = clip_battery(EXT ? request(lvl, p.batt_lvl, bpw, p) : request_t<true, false>(lvl, p.batt_lvl, bpw, p),
                              bsoc, p);
        }

        // ---- architecture constraint: group nodes (segmented scan), then root
        float Sg[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) Sg[q] = P[q];
        seg_scan<PPL, LPE>(Sg, meta, le, dh);
        float over = 0.f;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            if (meta[q] & kMetaTail) {
                const int gs = ew * GPS + (int)((meta[q] >> kMetaGroupShift) & 31u);
                const float gc = ws->gcap[gs];
                const float mag = V2G ? fabsf(Sg[q]) : Sg[q];
                const float sc = mag > gc ? __fdividef(gc, mag) : 1.0f;
                ws->scale[gs] = sc;
                if (p.a_con != 0.f) over = fmaxf(over, (mag - gc) * ws->ginv[gs]);
            }
        }
        __syncwarp();
        if constexpr (TREE) {
            // the upper nodes' penalty, on the requested power (P still is)
            if (TL > 0 && p.a_con != 0.f) {
#pragma unroll
                for (int j = 0; j < kMaxUpperDepth; ++j) {
                    if (j >= TL) break;
                    uint32_t lm[PPL];
                    float Sr[PPL];
#pragma unroll
                    for (int q = 0; q < PPL; ++q) {
                        lm[q] = level_meta(ws->m2[q][lane], j);
                        Sr[q] = P[q];
                    }
                    seg_scan<PPL, LPE>(Sr, lm, le, ws->dhu[j][lane]);
#pragma unroll
                    for (int q = 0; q < PPL; ++q)
                        if (lm[q] & kMetaTail) {
                            const int us = ew * GPS + (int)((lm[q] >> kMetaGroupShift) & 31u);
                            over = fmaxf(over, ((V2G ? fabsf(Sr[q]) : Sr[q]) - ws->ucap[j][us]) * ws->uinv[j][us]);
                        }
                }
            }
        }
        float raw = 0.f, sp = 0.f, se = 0.f, sn = 0.f;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            raw += P[q];
            P[q] *= ws->scale[ew * GPS + (int)((meta[q] >> kMetaGroupShift) & 31u)];
            sp += P[q];
            const bool dcq = meta[q] & kMetaDC;
            if (V2G) {
                if (P[q] >= 0.f) se += P[q] * (dcq ? p.inv_eta1 : p.inv_eta0);
                else sn += P[q] * (dcq ? p.eta1 : p.eta0);
            } else {
                se += P[q] * (dcq ? p.inv_eta1 : p.inv_eta0);
            }
        }
        if constexpr (TREE) {
            if (TL > 0) {
                // the upper levels, deepest first: each node rescales its
                // chargers' power, then the station sums are taken again
#pragma unroll
                for (int j = 0; j < kMaxUpperDepth; ++j) {
                    if (j >= TL) break;
                    uint32_t lm[PPL];
                    float Su[PPL];
#pragma unroll
                    for (int q = 0; q < PPL; ++q) {
                        lm[q] = level_meta(ws->m2[q][lane], j);
                        Su[q] = P[q];
                    }
                    seg_scan<PPL, LPE>(Su, lm, le, ws->dhu[j][lane]);
#pragma unroll
                    for (int q = 0; q < PPL; ++q) {
                        if (lm[q] & kMetaTail) {
                            const int us = ew * GPS + (int)((lm[q] >> kMetaGroupShift) & 31u);
                            const float cu = ws->ucap[j][us];
                            const float mag = V2G ? fabsf(Su[q]) : Su[q];
                            ws->uscale[j][us] = mag > cu ? __fdividef(cu, mag) : 1.0f;
                        }
                    }
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < PPL; ++q)
                        P[q] *= ws->uscale[j][ew * GPS + (int)((lm[q] >> kMetaGroupShift) & 31u)];
                    __syncwarp();
                }
                sp = 0.f;
                se = 0.f;
                sn = 0.f;
#pragma unroll
                for (int q = 0; q < PPL; ++q) {
                    sp += P[q];
                    const bool dcq = meta[q] & kMetaDC;
                    if (V2G) {
                        if (P[q] >= 0.f) se += P[q] * (dcq ? p.inv_eta1 : p.inv_eta0);
                        else sn += P[q] * (dcq ? p.eta1 : p.eta0);
                    } else {
                        se += P[q] * (dcq ? p.inv_eta1 : p.inv_eta0);
                    }
                }
            }
        }
        __syncwarp();
        sp = seg_sum<LPE>(sp);
        se = seg_sum<LPE>(se);
        if (V2G) sn = seg_sum<LPE>(sn);
        float c_con = 0.f;
        if (p.a_con != 0.f) {
            raw = seg_sum<LPE>(raw);
            over = seg_max<LPE>(over);
            const float raw_root = V2G ? fabsf(raw + Pb) : raw;
            c_con = fmaxf(fmaxf(over, (raw_root - grid_cap) * b.grid_inv_eta[s]), 0.f);
        }
        const float s_tot = V2G ? sp + Pb : sp;
        const float mag_root = V2G ? fabsf(s_tot) : s_tot;
        const float s_root = mag_root > grid_cap ? __fdividef(grid_cap, mag_root) : 1.0f;

        // ---- (ii) charge, time advance, (iii) departures
        bool any_leave = false;
        uint32_t leave = 0, leave_cs = 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            const float Pq = P[q] * s_root;
            pw[q] = Pq;
            if (trem[q] > 0) {
                const float dE = Pq * p.dt;
                soc[q] = fminf(soc[q] + __fdividef(dE, cap[q]), 1.0f);
                if (V2G) soc[q] = fmaxf(soc[q], 0.0f);
                erem[q] = fmaxf(erem[q] - dE, 0.0f);
                if (cs_on && trem[q] == kTremCS) {   // charge-sensitive: leaves once charged
                    due[q] -= 1;
                    if (erem[q] <= p.eps * cap[q]) leave_cs |= 1u << q;
                } else {
                    trem[q] -= 1;
                    if (trem[q] == 0) leave |= 1u << q;
                }
            }
        }
        leave |= leave_cs;
        any_leave = leave != 0;
        const float e_net = sp * s_root * p.dt;
        const float e_grid = se * s_root * p.dt;
        float e_to = 0.f, e_b = 0.f;
        if (V2G) {
            e_to = sn * s_root * p.dt;
            bpw = Pb * s_root;
            e_b = bpw * p.dt;
            bsoc = fminf(fmaxf(bsoc + e_b * p.inv_batt_cap, 0.0f), 1.0f);
        }
        float c_sat = 0.f, c_sat1 = 0.f;
        if (__any_sync(0xFFFFFFFFu, any_leave)) {
            float v = 0.f, v1 = 0.f;
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                if (leave & (1u << q)) {
                    if (EXT && (leave_cs & (1u << q))) {
                        // c_Sat,1: steps overdue minus beta x steps early
                        v1 += (float)max(-due[q], 0) - p.beta * (float)max(due[q], 0);
                        trem[q] = 0;
                        due[q] = 0;
                    } else {
                        v += erem[q];
                    }
                    soc[q] = 0.f; erem[q] = 0.f; cap[q] = 0.f; rbar[q] = 0.f;
                    if (EXT && p.delta) pw[q] = 0.f;   // Delta form: the next car starts from 0
                }
            }
            c_sat = seg_sum<LPE>(v);
            if (cs_on) c_sat1 = seg_sum<LPE>(v1);
        }

        // ---- (iv) arrivals: Poisson count, first come first served
        const uint32_t blk = g >> 2;
        if (k == 0 || blk - blk0 >= (uint32_t)LPE) {   // first step, or past the prefetched blocks
            blk0 = blk;
            const uint4 w = arrival_words(uidu, (blk + (uint32_t)le) << 2, k0, k1);
            ws->arrw[0][lane] = w.x;
            ws->arrw[1][lane] = w.y;
            ws->arrw[2][lane] = w.z;
            ws->arrw[3][lane] = w.w;
        }
        __syncwarp();
        const int M = poisson_count_warp<LPE>(b.cdf + ((size_t)cls_row * (size_t)p.ep_len + (size_t)t) * kCdfLen,
                                              ws->arrw[g & 3u][ew * LPE + (int)(blk - blk0)], le, env_mask);
        int n_free = 0, before = 0;
        uint32_t fr = 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            const bool f = (meta[q] & kMetaValid) && trem[q] == 0;
            fr |= (f ? 1u : 0u) << q;
            const unsigned bq = __ballot_sync(0xFFFFFFFFu, f) & env_mask;
            n_free += __popc(bq);
            before += __popc(bq & lt_mask);
        }
        const int m_adm = min(M, n_free);
        if (__any_sync(0xFFFFFFFFu, m_adm > 0)) {
            if (ncar + (uint32_t)m_adm > cend) {   // buffer exhausted: draw cars ncar .. ncar+C-1
#pragma unroll
                for (int q = 0; q < PPL; ++q) {   // profiles computed here, in one dense pass
                    const int i = q * LPE + le;
                    const uint4 w = car_words(uidu, ncar + (uint32_t)i, k0, k1);
                    const Car core = car_core(w, p);
                    ws->carw[0][ew * C + i] = __float_as_uint(core.cap);
                    ws->carw[1][ew * C + i] = __float_as_uint(core.soc);
                    ws->carw[2][ew * C + i] = __float_as_uint(core.erem);
                    ws->carw[3][ew * C + i] = (uint32_t)core.stay | (core.cs ? 1u << 8 : 0u);
                    ws->carw[4][ew * C + i] = w.w;
                }
                cend = ncar + (uint32_t)C;
            }
            __syncwarp();
            const int x0 = ew * C + (int)(ncar - (cend - (uint32_t)C));   // buffer slot of car ncar
            int rank = before;
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                const bool f = fr & (1u << q);
                if (f && rank < m_adm) {
                    const int x = x0 + rank;
                    cap[q] = __uint_as_float(ws->carw[0][x]);
                    soc[q] = __uint_as_float(ws->carw[1][x]);
                    erem[q] = __uint_as_float(ws->carw[2][x]);
                    rbar[q] = car_rbar(ws->carw[4][x], meta[q] & kMetaDC, p);
                    const uint32_t su = ws->carw[3][x];
                    if (EXT && (su >> 8)) {   // charge-sensitive user: stays until charged
                        trem[q] = kTremCS;
                        due[q] = (int)(su & 0xFFu);
                    } else {
                        trem[q] = (int)(su & 0xFFu);
                    }
                }
                rank += f ? 1 : 0;
            }
            ncar += (uint32_t)m_adm;
        }

        // ---- reward, Appendix A.3
        const float price = __ldg(b.price + (size_t)day * (size_t)p.ep_len + (size_t)t);
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
        if (EXT) r -= p.a_sat1 * c_sat1;
        ret += r;
        t += 1;
        const bool fin = t >= p.ep_len;
        if (le == 0) {                     // station statistics, one lane per station
            ws->st_u[ew][0] += (uint32_t)m_adm;
            ws->st_u[ew][1] += (uint32_t)(M - m_adm);
            ws->st_f[ew][0] += c_sat;
            ws->st_f[ew][1] += e_net;
            if (fin) {
                ws->st_f[ew][2] = ret;
                ws->st_u[ew][2] += 1u;
                ws->st_u[ew][3] = 1u;
            }
            if (live) {
                if (io.reward) io.reward[(long long)out_idx * io.ld_out + (long long)k * io.ld_step] = r;
                if (io.done) io.done[(long long)out_idx * io.ld_out + (long long)k * io.ld_step] = fin ? 1 : 0;
            }
        }
        if (fin) {                         // episode end: start a new one
            ret = 0.f;
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                soc[q] = 0.f; erem[q] = 0.f; cap[q] = 0.f; rbar[q] = 0.f; pw[q] = 0.f; trem[q] = 0;
                due[q] = 0;
            }
            t = 0;
            day = draw_day(uidu, g, 0u, k0, k1, p.n_days);
            if (V2G) {
                bsoc = p.batt_soc0;
                bpw = 0.f;
            }
        }
        g += 1u;
    }

    // ---- write back
    if (live) {                            // padding stations never write
        st_vec(b.soc + pb, soc);
        st_vec(b.erem + pb, erem);
        st_vec(b.cap + pb, cap);
        st_vec(b.rbar + pb, rbar);
        st_vec(b.pw + pb, pw);
        st_u8(b.trem + pb, trem);
        if (cs_on) st_i16(b.due + pb, due);
    }
    __syncwarp();
    if (le == 0 && live) {
        b.tod[s] = t;
        b.day[s] = day;
        b.gstep[s] = g;
        b.ncar[s] = ncar;
        b.ep_ret[s] = ret;
        if (ws->st_u[ew][3]) b.last_ret[s] = ws->st_f[ew][2];
        b.n_episodes[s] += ws->st_u[ew][2];
        b.st_arrived[s] += ws->st_u[ew][0];
        b.st_rejected[s] += ws->st_u[ew][1];
        b.st_missing[s] += ws->st_f[ew][0];
        b.st_charged[s] += ws->st_f[ew][1];
        if (V2G) {
            b.bsoc[s] = bsoc;
            b.bp[s] = bpw;
        }
    }
    if (io.obs) {                          // uniform across the warp
        int occ_l = 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q) occ_l += trem[q] > 0;
        const int occ = (int)seg_sum<LPE>((float)occ_l);
        if (live && obs_w >= 0) {
            const int n = b.n_ports[s];
            const int QP = EXT ? p.obs_port : 6;   // features per charger
            float* ob = io.obs + (io.gather ? (long long)obs_w
                                            : (long long)p.obs_env * uid + (long long)QP * b.user_port_off[s]);
            if (le == 0) obs_env(ob, t, day, occ, n, bsoc, bpw, b, p);
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                const int port = le * PPL + q;
                if (port < n)
                    obs_port<EXT>(ob + p.obs_env + QP * port, trem[q], due[q], soc[q], erem[q], rbar[q], pw[q],
                             meta[q] & kMetaDC, p);
            }
        }
    }
    __syncwarp();
}

// Persistent work loop over a schedule of classes in [CLO, CHI]: one
// instantiation for the 128-charger class (4 chargers per lane, more
// registers), one for the others, so the smaller classes keep more warps
// resident.
template <int CLO, int CHI, int MINB, bool V2G, bool EXT, bool TREE>
__global__ void __launch_bounds__(256, MINB) k_step_fused(DevBatch b, DevParams p, FusedIO io)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using SM = std::conditional_t<TREE, WarpSmemExt, WarpSmem>;
    SM* ws = reinterpret_cast<SM*>(smem_raw) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < 64; i += 32) {   // padding chargers read defined values
        ws->scale[i] = 1.0f;
        ws->gcap[i] = 0.f;
        ws->ginv[i] = 1.f;
        if constexpr (TREE) {
            for (int j = 0; j < kMaxUpperDepth; ++j) {
                ws->uscale[j][i] = 1.0f;
                ws->ucap[j][i] = FLT_MAX;
                ws->uinv[j][i] = 1.f;
            }
        }
    }
    __syncwarp();
    for (;;) {
        int tile_id = 0;
        if (lane == 0) tile_id = atomicAdd(io.counter, 1);
        tile_id = __shfl_sync(0xFFFFFFFFu, tile_id, 0);
        int cls = -1, tile = 0;
        if (io.dcount) {                   // device-side schedule: classes CHI down to CLO
            int rest = tile_id;
#pragma unroll
            for (int c = CHI; c >= CLO; --c) {
                const int nt = (__ldg(io.dcount + c) + tile_epw(c) - 1) / tile_epw(c);
                if (cls < 0 && rest < nt) {
                    cls = c;
                    tile = rest;
                }
                rest -= nt;
            }
            if (cls < 0) break;
        } else {
            if (tile_id >= io.total_tiles) break;
#pragma unroll
            for (int i = 0; i < kNumClasses; ++i) {
                if (i < io.n_sched && tile_id >= io.sched_tile_base[i] && tile_id < io.sched_tile_base[i + 1]) {
                    cls = io.sched_cls[i];
                    tile = tile_id - io.sched_tile_base[i];
                }
            }
        }
        if (CLO <= 0 && 0 <= CHI && cls == 0) run_tile<8, V2G, EXT, TREE>(b, p, io, tile, ws);
        if (CLO <= 1 && 1 <= CHI && cls == 1) run_tile<16, V2G, EXT, TREE>(b, p, io, tile, ws);
        if (CLO <= 2 && 2 <= CHI && cls == 2) run_tile<32, V2G, EXT, TREE>(b, p, io, tile, ws);
        if (CLO <= 3 && 3 <= CHI && cls == 3) run_tile<64, V2G, EXT, TREE>(b, p, io, tile, ws);
        if (CLO <= 4 && 4 <= CHI && cls == 4) run_tile<128, V2G, EXT, TREE>(b, p, io, tile, ws);
    }
}

namespace {

// [v2g | ext << 1 | tree << 2]: charge-only / vehicle-to-grid; ext instances
// add, switched at run time, the Delta-current form and charge-sensitive
// users, tree instances the levels of nodes above the groups
constexpr int kForms = 8;
constexpr size_t smem_per_warp(int v) { return (v & 4) ? sizeof(WarpSmemExt) : sizeof(WarpSmem); }
#define CHX_FORMS(CLO, CHI, MINB)                                                                              \
    {&k_step_fused<CLO, CHI, MINB, false, false, false>, &k_step_fused<CLO, CHI, MINB, true, false, false>,  \
     &k_step_fused<CLO, CHI, MINB, false, true, false>, &k_step_fused<CLO, CHI, MINB, true, true, false>,    \
     &k_step_fused<CLO, CHI, MINB, false, false, true>, &k_step_fused<CLO, CHI, MINB, true, false, true>,    \
     &k_step_fused<CLO, CHI, MINB, false, true, true>, &k_step_fused<CLO, CHI, MINB, true, true, true>}
// The instances by class range.  The V2G and extended forms run the
// 64-charger class in an instance of its own (measured: 4 % faster with
// fewer spills in each); the charge-only and tree forms keep it with the
// smaller classes (their split instances measured 1 % slower).
constexpr bool split64(int v) { return (v & 4) == 0 && (v & 3) != 0; }
constexpr int kRanges = 3;                 // 8..32 or 8..64, 64 (split forms), 128 chargers
using FusedKernel = void (*)(DevBatch, DevParams, FusedIO);
const FusedKernel kSmall[kForms] = CHX_FORMS(0, 3, 3);
const FusedKernel kSmall32[kForms] = CHX_FORMS(0, 2, 3);
const FusedKernel kMid[kForms] = CHX_FORMS(3, 3, 3);
const FusedKernel kLarge[kForms] = CHX_FORMS(4, 4, 3);
#undef CHX_FORMS
FusedKernel fused_kernel(int r, int v)
{
    if (r == 2) return kLarge[v];
    if (r == 1) return split64(v) ? kMid[v] : nullptr;
    return split64(v) ? kSmall32[v] : kSmall[v];
}
constexpr int range_lo(int r) { return r == 0 ? 0 : (r == 1 ? 3 : 4); }
constexpr int range_hi(int r, int v) { return r == 0 ? (split64(v) ? 2 : 3) : (r == 1 ? 3 : 4); }

// the part of a schedule whose classes lie in [clo, chi], tiles renumbered
FusedIO sub_schedule(const FusedIO& io, int clo, int chi, int* counter)
{
    FusedIO o = io;
    o.n_sched = 0;
    int tb = 0;
    for (int i = 0; i < io.n_sched; ++i) {
        const int c = io.sched_cls[i];
        if (c < clo || c > chi) continue;
        o.sched_cls[o.n_sched] = c;
        o.sched_tile_base[o.n_sched] = tb;
        o.n_sched++;
        tb += io.sched_tile_base[i + 1] - io.sched_tile_base[i];
    }
    o.sched_tile_base[o.n_sched] = tb;
    o.total_tiles = tb;
    o.counter = counter;
    return o;
}

// allow each kernel the dynamic shared memory of 8 warps (above the 48 KB default)
bool raise_smem_limit()
{
    static const bool ok = [] {
        for (int r = 0; r < kRanges; ++r)
            for (int v = 0; v < kForms; ++v)
                if (fused_kernel(r, v) &&
                    cudaFuncSetAttribute((const void*)fused_kernel(r, v), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8 * (int)smem_per_warp(v)) != cudaSuccess)
                    return false;
        return true;
    }();
    return ok;
}

int blocks_per_sm(const void* kernel, int v, int threads)
{
    if (!raise_smem_limit()) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, (threads / 32) * smem_per_warp(v)) !=
        cudaSuccess)
        return 0;
    return n;
}

// blocks_per_sm of a range's kernel, asked of the runtime once per (range,
// form, block size): launches on the serving path happen every tick
int blocks_per_sm_memo(int r, int v, int threads)
{
    static std::atomic<int> memo[kRanges][kForms][9] = {};
    std::atomic<int>& m = memo[r][v][std::min(std::max(threads / 32, 0), 8)];
    int n = m.load(std::memory_order_relaxed);
    if (n <= 0) {
        n = blocks_per_sm((const void*)fused_kernel(r, v), v, threads);
        if (n > 0) m.store(n, std::memory_order_relaxed);
    }
    return n;
}

}  // namespace

bool fused_block_size_ok(int threads)
{
    if (threads < 32 || threads > 256 || threads % 32 != 0) return false;
    for (int r = 0; r < kRanges; ++r)
        for (int v = 0; v < kForms; ++v)
            if (fused_kernel(r, v) && blocks_per_sm((const void*)fused_kernel(r, v), v, threads) <= 0) return false;
    return true;
}

void launch_step_fused(const DevBatch& b, const DevParams& p, const FusedIO& io, int threads, int sm_count,
                       cudaStream_t st, const FusedSide* side)
{
    const int warps = threads / 32;
    const int v = (p.v2g ? 1 : 0) | ((p.delta || p.cs_share) ? 2 : 0) | (p.tree_levels ? 4 : 0);
    const size_t smem = (size_t)warps * smem_per_warp(v);
    // per range (8..32 or 8..64, 64, 128 chargers): its schedule and a tile
    // bound for the grid.  Device-side schedule: the grids come from the
    // host's bounds; the kernels read the tile counts.
    FusedIO o[kRanges];
    int tiles[kRanges];
    for (int r = 0; r < kRanges; ++r) {
        if (!fused_kernel(r, v)) {
            tiles[r] = 0;
        } else if (io.dcount) {
            o[r] = io;
            o[r].counter = io.counter + r;
            tiles[r] = r == 0 ? io.dmax_small : (r == 1 ? io.dmax_mid : io.dmax_large);
        } else {
            o[r] = sub_schedule(io, range_lo(r), range_hi(r, v), io.counter + r);
            tiles[r] = o[r].total_tiles;
        }
    }
    // the 128- and 64-charger classes first, beside the others when a side
    // stream is given (their few stations would otherwise run alone on a
    // mostly idle GPU at the end)
    const bool fork = side && side->aux && tiles[0] > 0 && (tiles[1] > 0 || tiles[2] > 0);
    cudaStream_t sb = st;
    if (fork) {
        cudaEventRecord(side->fork, st);
        cudaStreamWaitEvent(side->aux, side->fork, 0);
        sb = side->aux;
    }
    auto launch = [&](int r, cudaStream_t s) {
        const int blocks = std::max(1, std::min(blocks_per_sm_memo(r, v, threads) * sm_count,
                                                (tiles[r] + warps - 1) / warps));
        fused_kernel(r, v)<<<blocks, threads, smem, s>>>(b, p, o[r]);
    };
    if (tiles[2] > 0) launch(2, sb);
    if (tiles[1] > 0) launch(1, sb);
    if (fork) cudaEventRecord(side->join, side->aux);
    if (tiles[0] > 0) launch(0, st);
    if (fork) cudaStreamWaitEvent(st, side->join, 0);
}

}  // namespace chx
