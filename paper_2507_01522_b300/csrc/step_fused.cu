// step_fused.cu -- the fused form of the step: K transitions per launch.
//
// A persistent kernel.  Each warp repeatedly takes a tile from a global work
// counter (tiles of the largest stations first), loads the tile's state into
// registers, runs K steps without touching HBM except for the per-step
// reward/done outputs, and stores the state back.  A tile is 32 charger slots
// per lane-column: 32/C stations of size class C <= 32 (one charger per
// lane), or one station of C = 64/128 (2/4 consecutive chargers per lane).
//
// Reductions over chargers (Eq. ArchConst and the reward sums) are warp
// shuffles: a segmented inclusive scan gives each group node's power at its
// last charger, whose scale is broadcast through 32 floats of shared memory;
// station totals use an xor butterfly inside the station's aligned lane
// segment.  Both depend only on a charger's position inside its station, so a
// station's result does not depend on which tile or lane offset it runs in.
#include "chx_device.cuh"
#include "chx_kernels.h"

namespace chx {

template <int C>
struct Shape {
    static constexpr int PPL = C > 32 ? C / 32 : 1;   // chargers per lane
    static constexpr int LPE = C > 32 ? 32 : C;       // lanes per station
    static constexpr int EPW = 32 / LPE;              // stations per warp
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

// Inclusive segmented scan of v over the chargers of the warp in charger
// order (lane-major, PPL per lane); a set head bit starts a new segment.
template <int PPL, int LPE>
__device__ __forceinline__ void seg_scan(float (&v)[PPL], const uint32_t (&meta)[PPL], int le)
{
    bool any_head = meta[0] & kMetaHead;
#pragma unroll
    for (int q = 1; q < PPL; ++q) {
        if (!(meta[q] & kMetaHead)) v[q] += v[q - 1];
        any_head = any_head || (meta[q] & kMetaHead);
    }
    float x = v[PPL - 1];
    int f = any_head ? 1 : 0;
#pragma unroll
    for (int d = 1; d < LPE; d <<= 1) {
        const float xu = __shfl_up_sync(0xFFFFFFFFu, x, d);
        const int fu = __shfl_up_sync(0xFFFFFFFFu, f, d);
        if (le >= d) {
            if (!f) x += xu;
            f |= fu;
        }
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

template <int C>
__device__ __forceinline__ void run_tile(const DevBatch& b, const DevParams& p, const FusedIO& io, int cls, int tile,
                                         float* sw)
{
    using S = Shape<C>;
    constexpr int PPL = S::PPL, LPE = S::LPE;
    constexpr int CI = C == 8 ? 0 : (C == 16 ? 1 : (C == 32 ? 2 : (C == 64 ? 3 : 4)));
    const int lane = threadIdx.x & 31;
    const int ew = lane / LPE;            // station within the warp
    const int le = lane % LPE;            // lane within the station
    // the station this lane works on: the tile's own slots, or (gather mode)
    // the slots a caller listed, with their own action/output/observation offsets
    int s;
    long long act_base, out_idx, obs_off;
    if (io.gather) {
        const int4 en = io.gather[io.gather_base[CI] + tile * S::EPW + ew];
        s = en.x;
        act_base = en.y;
        out_idx = en.z;
        obs_off = en.w;
    } else {
        s = b.cls_env_base[CI] + tile * S::EPW + ew;
        act_base = b.user_port_off[s];
        out_idx = b.user_id[s];
        obs_off = 8LL * out_idx + 6LL * act_base;
    }
    const long long pb = b.cls_port_base[CI] + (long long)(s - b.cls_env_base[CI]) * C + le * PPL;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned env_mask = (LPE == 32) ? 0xFFFFFFFFu : (((1u << LPE) - 1u) << (ew * LPE));

    // per-station state (identical in the station's lanes)
    const int uid = b.user_id[s];
    const bool live = uid >= 0;
    const uint32_t uidu = (uint32_t)(live ? uid : 0);
    const int cls_row = b.arrival_class[s];
    const float grid_cap = b.grid_cap[s], grid_inv_eta = b.grid_inv_eta[s];
    const uint32_t k0 = b.key0[s], k1 = b.key1[s];
    int t = b.tod[s], day = b.day[s];
    uint32_t g = b.gstep[s];
    float ret = b.ep_ret[s], last_ret = 0.f;
    uint32_t n_ep = 0, arrived = 0, rejected = 0;
    float missing = 0.f, charged = 0.f;
    bool had_end = false;

    // per-charger state
    float soc[PPL], erem[PPL], cap[PPL], rbar[PPL], pw[PPL];
    int trem[PPL];
    uint32_t meta[PPL];
    float gcap[PPL], ginv[PPL];
    ld_vec(b.soc + pb, soc);
    ld_vec(b.erem + pb, erem);
    ld_vec(b.cap + pb, cap);
    ld_vec(b.rbar + pb, rbar);
    ld_vec(b.pw + pb, pw);
    ld_u8(b.trem + pb, trem);
    ld_vec_u32(b.meta + pb, meta);
    ld_vec(b.gcap + pb, gcap);
    ld_vec(b.ginv_eta + pb, ginv);
    int gslot[PPL];
#pragma unroll
    for (int q = 0; q < PPL; ++q) gslot[q] = ew * LPE + (int)((meta[q] >> kMetaGroupShift) & 31u);

    uint4 aw[PPL];                        // Philox words of the current 8-step action block
    const bool random_actions = io.actions == nullptr;

    for (int k = 0; k < io.k_steps; ++k) {
        // ---- (i) apply actions: per-charger clip
        float P[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            const int port = le * PPL + q;
            int lvl = 0;
            if (random_actions) {
                if (k == 0 || (g & 7u) == 0u)
                    aw[q] = philox4x32_10(make_uint4(uidu, g >> 3, (uint32_t)port, kPurposeAction), k0, k1);
                lvl = random_level(aw[q], g, p.n_levels);
            } else if (trem[q] > 0) {
                lvl = io.actions[(act_base + port) * io.lda + k];
                if (lvl < 0 || lvl >= p.n_levels) {
                    atomicOr(b.err, kErrActionRange);
                    lvl = min(max(lvl, 0), p.n_levels - 1);
                }
            }
            const bool dc = meta[q] & kMetaDC;
            P[q] = trem[q] > 0 ? clip_power(lvl, dc, soc[q], erem[q], cap[q], rbar[q], p) : 0.f;
        }

        // ---- architecture constraint: group nodes (segmented scan), then root
        float Sg[PPL];
#pragma unroll
        for (int q = 0; q < PPL; ++q) Sg[q] = P[q];
        seg_scan<PPL, LPE>(Sg, meta, le);
        float over = 0.f;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            if (meta[q] & kMetaTail) {
                const float sc = Sg[q] > gcap[q] ? gcap[q] / Sg[q] : 1.0f;
                sw[gslot[q]] = sc;
                over = fmaxf(over, (Sg[q] - gcap[q]) * ginv[q]);
            }
        }
        __syncwarp();
        float raw = 0.f, sp = 0.f, se = 0.f;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            raw += P[q];
            P[q] *= sw[gslot[q]];
            sp += P[q];
            se += P[q] * ((meta[q] & kMetaDC) ? p.inv_eta1 : p.inv_eta0);
        }
        __syncwarp();
        sp = seg_sum<LPE>(sp);
        se = seg_sum<LPE>(se);
        float c_con = 0.f;
        if (p.a_con != 0.f) {
            raw = seg_sum<LPE>(raw);
            over = seg_max<LPE>(over);
            c_con = fmaxf(fmaxf(over, (raw - grid_cap) * grid_inv_eta), 0.f);
        }
        const float s_root = sp > grid_cap ? grid_cap / sp : 1.0f;

        // ---- (ii) charge, time advance, (iii) departures
        bool leave[PPL];
        bool any_leave = false;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            const float Pq = P[q] * s_root;
            pw[q] = Pq;
            leave[q] = false;
            if (trem[q] > 0) {
                const float dE = Pq * p.dt;
                soc[q] = fminf(soc[q] + dE / cap[q], 1.0f);
                erem[q] = fmaxf(erem[q] - dE, 0.0f);
                trem[q] -= 1;
                leave[q] = trem[q] == 0;
                any_leave = any_leave || leave[q];
            }
        }
        const float e_net = sp * s_root * p.dt;
        const float e_grid = se * s_root * p.dt;
        float c_sat = 0.f;
        if (__any_sync(0xFFFFFFFFu, any_leave)) {
            float v = 0.f;
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                if (leave[q]) {
                    v += erem[q];
                    soc[q] = 0.f; erem[q] = 0.f; cap[q] = 0.f; rbar[q] = 0.f;
                }
            }
            c_sat = seg_sum<LPE>(v);
        }

        // ---- (iv) arrivals: Poisson count, first come first served
        const int M = arrivals(b, p, uidu, g, t, cls_row, k0, k1);
        bool fr[PPL];
        int n_free = 0, before = 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q) {
            fr[q] = (meta[q] & kMetaValid) && trem[q] == 0;
            const unsigned bq = __ballot_sync(0xFFFFFFFFu, fr[q]) & env_mask;
            n_free += __popc(bq);
            before += __popc(bq & lt_mask);
        }
        const int m_adm = min(M, n_free);
        if (__any_sync(0xFFFFFFFFu, m_adm > 0)) {
            int rank = before;
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                if (fr[q] && rank < m_adm) {
                    const Car car = draw_car(uidu, g, (uint32_t)rank, k0, k1, meta[q] & kMetaDC, p);
                    cap[q] = car.cap; soc[q] = car.soc; erem[q] = car.erem; rbar[q] = car.rbar;
                    trem[q] = car.stay;
                }
                rank += fr[q] ? 1 : 0;
            }
        }

        // ---- reward, Appendix A.3
        const float price = __ldg(b.price + (size_t)day * (size_t)p.ep_len + (size_t)t);
        const float profit = p.p_sell * e_net - price * e_grid - p.c_fixed;
        const float r = profit - p.a_sat * c_sat - p.a_decl * (float)(M - m_adm) - p.a_con * c_con;
        arrived += (uint32_t)m_adm;
        rejected += (uint32_t)(M - m_adm);
        missing += c_sat;
        charged += e_net;
        ret += r;
        t += 1;
        uint8_t fin = 0;
        if (t >= p.ep_len) {               // episode end: record and start a new one
            fin = 1;
            last_ret = ret;
            had_end = true;
            ret = 0.f;
            n_ep += 1u;
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                soc[q] = 0.f; erem[q] = 0.f; cap[q] = 0.f; rbar[q] = 0.f; pw[q] = 0.f; trem[q] = 0;
            }
            t = 0;
            day = draw_day(uidu, g, 0u, k0, k1, p.n_days);
        }
        g += 1u;
        if (live && le == 0) {
            if (io.reward) io.reward[out_idx * io.ld_out + k] = r;
            if (io.done) io.done[out_idx * io.ld_out + k] = fin;
        }
    }

    // ---- write back
    if (live) {                            // padding stations never write
        st_vec(b.soc + pb, soc);
        st_vec(b.erem + pb, erem);
        st_vec(b.cap + pb, cap);
        st_vec(b.rbar + pb, rbar);
        st_vec(b.pw + pb, pw);
        st_u8(b.trem + pb, trem);
    }
    if (le == 0 && live) {
        b.tod[s] = t;
        b.day[s] = day;
        b.gstep[s] = g;
        b.ep_ret[s] = ret;
        if (had_end) b.last_ret[s] = last_ret;
        b.n_episodes[s] += n_ep;
        b.st_arrived[s] += arrived;
        b.st_rejected[s] += rejected;
        b.st_missing[s] += missing;
        b.st_charged[s] += charged;
    }
    if (io.obs) {                          // uniform across the warp
        int occ_l = 0;
#pragma unroll
        for (int q = 0; q < PPL; ++q) occ_l += trem[q] > 0;
        const int occ = (int)seg_sum<LPE>((float)occ_l);
        if (live) {
            const int n = b.n_ports[s];
            float* ob = io.obs + obs_off;
            if (le == 0) obs_env(ob, t, day, occ, n, b, p);
#pragma unroll
            for (int q = 0; q < PPL; ++q) {
                const int port = le * PPL + q;
                if (port < n)
                    obs_port(ob + 8 + 6 * port, trem[q], soc[q], erem[q], rbar[q], pw[q], meta[q] & kMetaDC, p);
            }
        }
    }
}

__global__ void __launch_bounds__(256, 2) k_step_fused(DevBatch b, DevParams p, FusedIO io)
{
    extern __shared__ float smem[];
    float* sw = smem + (threadIdx.x >> 5) * 32;
    const int lane = threadIdx.x & 31;
    sw[lane] = 1.0f;                       // group scales; padding chargers read a defined value
    __syncwarp();
    for (;;) {
        int tile_id = 0;
        if (lane == 0) tile_id = atomicAdd(io.counter, 1);
        tile_id = __shfl_sync(0xFFFFFFFFu, tile_id, 0);
        if (tile_id >= io.total_tiles) break;
        int cls = 0, tile = 0;
#pragma unroll
        for (int i = 0; i < kNumClasses; ++i) {
            if (i < io.n_sched && tile_id >= io.sched_tile_base[i] && tile_id < io.sched_tile_base[i + 1]) {
                cls = io.sched_cls[i];
                tile = tile_id - io.sched_tile_base[i];
            }
        }
        switch (cls) {
            case 0: run_tile<8>(b, p, io, cls, tile, sw); break;
            case 1: run_tile<16>(b, p, io, cls, tile, sw); break;
            case 2: run_tile<32>(b, p, io, cls, tile, sw); break;
            case 3: run_tile<64>(b, p, io, cls, tile, sw); break;
            default: run_tile<128>(b, p, io, cls, tile, sw); break;
        }
    }
}

int fused_max_blocks_per_sm(int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_fused, threads, (threads / 32) * 32 * sizeof(float)) !=
        cudaSuccess)
        return 0;
    return n;
}

void launch_step_fused(const DevBatch& b, const DevParams& p, const FusedIO& io, int blocks, int threads,
                       cudaStream_t st)
{
    k_step_fused<<<blocks, threads, (threads / 32) * 32 * sizeof(float), st>>>(b, p, io);
}

}  // namespace chx
