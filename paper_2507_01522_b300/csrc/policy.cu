// policy.cu -- the on-device policy: a 3-layer MLP
// obs (D = 8 + 6N) -> 256 -> 256 -> N x L logits (ReLU between layers; the
// actor of the PPO agent of the paper's Sec. 5, randomly initialised), BF16
// operands, FP32 accumulation, on the 5th-generation tensor cores, with the
// categorical sample of every charger's action level fused into the last
// layer's epilogue.  Two kernels share it:
//
//   k_policy   actions of every env from given observations (one MLP pass
//              per 128-env tile);
//   k_rollout  the fused rollout: one CTA owns 128 envs for all T steps and
//              alternates "observe -> MLP -> sample -> environment step"
//              without leaving the SM.  The env state lives in TMEM next to
//              the accumulators (lane = env, see kCol*); the environment step
//              runs one thread per env.
//
// Roles (both kernels, 10 warps):
//   warp 0, lane 0   TMA producer: streams the weights, one 128-row x 64-col
//                    BF16 box (16 KB) per stage, through a ring of stages;
//   warp 1           owns the TMEM allocation (512 columns); lane 0 issues
//                    every tcgen05.mma (M = 128, N <= 128 per part, K = 16);
//   warps 2..9       "workers": write the layer-1 operand, run the epilogues
//                    (bias, ReLU, BF16 into the next layer's operand) and the
//                    sampling.  Worker warp w reads TMEM lanes 32 (w % 4) ..
//                    +31 (one env per thread); warps 2-5 take accumulator
//                    columns 0-127, warps 6-9 columns 128-255 (chargers 0-15
//                    and 16-31 in the sampling).  In k_rollout warps 2-5 also
//                    own the env rows of their lane quadrant.
//
// One operand buffer A (128 x 256 BF16, swizzled) holds the observations,
// then h1, then h2: an epilogue writes A only after every MMA of its layer
// has finished.  Every wait is bounded (kWaitCycles); a timeout sets
// kErrPolicyWait and a shared flag that makes every role skip its remaining
// waits and asynchronous work, so the kernel always ends.
#include <cuda.h>

#include "chx_kernels.h"
#include "chx_tc.cuh"

namespace chx {

namespace {

using namespace tc;

constexpr int kM = 128;                    // envs per tile (MMA M, TMEM lanes)
constexpr int kChunkBytes = kM * 128;      // 128 rows x 64 BF16
constexpr int kActBytes = 4 * kChunkBytes; // 128 x 256 BF16 operand
constexpr int kStageRows = 256;            // weight rows (MMA N) per stage
constexpr int kStageBytes = kStageRows * 128; // 256 weight rows x 64 BF16
constexpr int kWorkerWarps = 8;
constexpr int kWorkers = kWorkerWarps * 32;
constexpr int kThreads = (2 + kWorkerWarps) * 32;
constexpr uint32_t kTmemCols = 512;
constexpr int kPolStages = 4;              // weight ring of k_policy
constexpr int kRollStages = 3;             // weight ring of k_rollout
constexpr int kMaxStages = kPolStages;
constexpr int kBarWorkers = 1;             // named barrier of the worker warps

// k_rollout: TMEM columns of the env state, 32 per field (charger c at +c)
constexpr int kColSoc = 352, kColErem = 384, kColCap = 416, kColRbar = 448;
constexpr int kColPack = 480;              // remaining stay | meta << 8
constexpr int kColPw = 0;                  // last applied power, parked in accumulator columns between MLP passes

struct Sync {
    uint64_t full[kMaxStages], empty[kMaxStages];
    uint64_t acc;                          // a layer is accumulated (3 completions per pass)
    uint64_t xrdy;                         // layer-1 operand written (kWorkers arrivals)
    uint64_t hrdy;                         // h1 / h2 written (kWorkers arrivals, 2 per pass)
    uint64_t fin;                          // every MMA of the CTA finished
    uint32_t tmem;
    int bad;                               // a wait timed out: skip everything
};

__device__ __forceinline__ bool is_bad(const Sync& S) { return *reinterpret_cast<const volatile int*>(&S.bad) != 0; }

// bounded wait; on timeout raise the error and the shared flag; returns
// immediately (false) once the flag is set
// (kSleep: after a short spin the waiting thread sleeps with exponential
// backoff, so that long waits leave the issue slots to the warps doing the
// work; the single producer and MMA threads spin, their waits are on the
// critical path)
template <bool kSleep = true>
__device__ __forceinline__ bool wait_sync(uint64_t* bar, uint32_t parity, Sync& S, uint32_t* err)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    unsigned ns = 0;
    for (int i = 0;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (is_bad(S)) return false;
        if (clock64() - t0 > kWaitCycles) {
            *reinterpret_cast<volatile int*>(&S.bad) = 1;
            atomicOr(err, kErrPolicyWait);
            return false;
        }
        if (kSleep && i >= 8) {
            ns = ns ? (ns < 256u ? 2u * ns : 256u) : 32u;
            __nanosleep(ns);
        }
    }
}

__device__ __forceinline__ void init_sync(Sync& S, int n_stages)
{
    for (int s = 0; s < n_stages; ++s) {
        mbar_init(&S.full[s], 1);
        mbar_init(&S.empty[s], 1);             // the MMA commit that has read the stage
    }
    mbar_init(&S.acc, 1);
    mbar_init(&S.fin, 1);
    mbar_init(&S.xrdy, kWorkers);
    mbar_init(&S.hrdy, kWorkers);
    S.bad = 0;
    mbar_fence_init();
}

// ---- TMA producer: n_passes MLP passes worth of weight stages ------------
// A stage is one 64-column K chunk of one layer part: 256 weight rows (the
// MMA's N), or n3_last rows for the last part of layer 3.
// Every CTA loads its own stages (the 0.44 MB of weights stay in L2); a slot
// is refilled once the MMAs that read it have completed.
__device__ __forceinline__ int part_rows(const PolicyArgs& a, int L, int p)
{
    return (L == 2 && p == a.parts3 - 1) ? a.n3_last : kStageRows;
}

template <int NS>
__device__ void produce(const WMaps* wm, const PolicyArgs& a, unsigned char* ring, Sync& S, int n_passes)
{
    uint32_t s = 0;
    int last[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) last[j] = -1;
    for (int it = 0; it < n_passes; ++it)
        for (int L = 0; L < 3; ++L) {
            const int parts = L < 2 ? 1 : a.parts3;
            const int chunks = L == 0 ? a.ch1 : 4;
            for (int p = 0; p < parts; ++p) {
                const int rows = part_rows(a, L, p);
                const CUtensorMap* map = rows == kStageRows ? &wm->main : &wm->tail;
                for (int k = 0; k < chunks; ++k, ++s) {
                    const uint32_t slot = s % NS;
                    if (s >= (uint32_t)NS) wait_sync<false>(&S.empty[slot], ((s / NS) - 1) & 1, S, a.err);
                    if (is_bad(S)) continue;
                    mbar_arrive_expect_tx(&S.full[slot], (uint32_t)rows * 128u);
                    tma_load_2d(ring + slot * kStageBytes, map, k * 64, L * 256 + p * kStageRows, &S.full[slot]);
#pragma unroll
                    for (int j = 0; j < NS; ++j)
                        if (j == (int)slot) last[j] = (int)s;
                }
            }
        }
    // nothing may still be landing in shared memory when the CTA exits
#pragma unroll
    for (int j = 0; j < NS; ++j)
        if (last[j] >= 0 && !mbar_wait(&S.full[j], ((uint32_t)last[j] / NS) & 1)) atomicOr(a.err, kErrPolicyWait);
}

// ---- MMA issuer ------------------------------------------------------------
template <int NS>
__device__ void issue(const PolicyArgs& a, unsigned char* A, unsigned char* ring, Sync& S, uint32_t tmem,
                      int n_passes)
{
    uint32_t s = 0;
    for (int it = 0; it < n_passes; ++it) {
        wait_sync<false>(&S.xrdy, it & 1, S, a.err);
        fence_after();
        for (int L = 0; L < 3; ++L) {
            if (L > 0) {
                wait_sync<false>(&S.hrdy, (2 * it + L - 1) & 1, S, a.err);
                fence_after();
            }
            const int parts = L < 2 ? 1 : a.parts3;
            const int chunks = L == 0 ? a.ch1 : 4;
            for (int p = 0; p < parts; ++p) {
                const uint32_t id = idesc_bf16_f32(kM, part_rows(a, L, p));
                for (int k = 0; k < chunks; ++k, ++s) {
                    const uint32_t slot = s % NS;
                    wait_sync<false>(&S.full[slot], (s / NS) & 1, S, a.err);
                    fence_after();
                    if (is_bad(S)) continue;
                    const int nks = (L == 0 && k == chunks - 1) ? a.ks1_last : 4;
                    unsigned char* bst = ring + slot * kStageBytes;
                    for (int j = 0; j < nks; ++j)          // onto the bias the workers placed in TMEM
                        mma_bf16(tmem + (uint32_t)(p * kStageRows), sdesc_sw128(A + k * kChunkBytes + j * 32),
                                 sdesc_sw128(bst + j * 32), id, true);
                    mma_commit(&S.empty[slot]);
                }
            }
            if (!is_bad(S)) mma_commit(&S.acc);
        }
    }
    mma_commit(&S.fin);
    if (!mbar_wait(&S.fin, 0)) atomicOr(a.err, kErrPolicyWait);
}

// ---- bias rows into TMEM: every accumulator of a layer starts at its bias --
// 32 columns [c0, c0 + 32) of the warp's 32 lanes := bias[c0 .. c0 + 31]
__device__ __forceinline__ void bias_to_tmem(uint32_t taddr, const float* bias)
{
    uint32_t v[32];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 b = reinterpret_cast<const float4*>(bias)[j];
        v[4 * j] = __float_as_uint(b.x);
        v[4 * j + 1] = __float_as_uint(b.y);
        v[4 * j + 2] = __float_as_uint(b.z);
        v[4 * j + 3] = __float_as_uint(b.w);
    }
    tmem_st32(taddr, v);
}

// Bias of layer L (0, 1: 256 columns; 2: n_out_pad columns) into the
// accumulator columns this worker warp may write: half h takes hidden
// columns 128h .. 128h+127 and, for layer 3, 48 of columns 256 .. 351 as
// well (columns it does not read in the layer-2 epilogue).
__device__ __forceinline__ void layer_bias(const PolicyArgs& a, const float* bias_s, uint32_t tl, int L, int h)
{
    const float* b = bias_s + kPolicyHidden * L;
    const int n = L < 2 ? kPolicyHidden : a.n_out_pad;
#pragma unroll 1
    for (int c = 128 * h; c < 128 * h + 128; c += 32)
        if (c < n) bias_to_tmem(tl + (uint32_t)c, b + c);
    if (L == 2)
#pragma unroll 1
        for (int c = 256 + 64 * h; c < 256 + 64 * h + 64; c += 32)
            if (c < n) bias_to_tmem(tl + (uint32_t)c, b + c);
    tmem_wait_st();
}

// ---- epilogue of layers 1 and 2: ReLU, BF16 into A ------------------------
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, uint32_t abase, int row, int col0)
{
#pragma unroll 1
    for (int blk = 0; blk < 4; ++blk) {
        const int c = col0 + 32 * blk;
        uint32_t v[32];
        tmem_ld32(taddr + (uint32_t)(32 * blk), v);
        tmem_wait_ld();
        uint32_t q[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
            q[j] = pack_bf16x2(fmaxf(__uint_as_float(v[2 * j]), 0.f), fmaxf(__uint_as_float(v[2 * j + 1]), 0.f));
        const int unit0 = (c & 63) >> 3;
        const uint32_t rbase = abase + (uint32_t)((c >> 6) * kChunkBytes + row * 128);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            st_shared_v4(rbase + ((uint32_t)((unit0 + u) ^ (row & 7)) << 4), q[4 * u], q[4 * u + 1], q[4 * u + 2],
                         q[4 * u + 3]);
    }
}

// ---- sampling ----------------------------------------------------------------
// Inverse transform of the softmax of charger c's logits l_0..l_{L-1}:
// level = #{j < L-1 : e_0 + .. + e_j <= u S}, e_j = exp(l_j - max l),
// S = sum e_j, u from word c % 4 of the policy Philox block (env, step, c / 4).
template <int LT>
__device__ __forceinline__ uint32_t sample4(const uint32_t (&v)[48], int c0, int n_ports, int n_levels, uint4 words,
                                           float* logits_out)
{
    const int L = LT ? LT : n_levels;
    uint32_t packed = 0;
#pragma unroll
    for (int ci = 0; ci < 4; ++ci) {
        const int c = c0 + ci;
        if (c >= n_ports) break;
        float l[kPolicyGroup];
        float m = -INFINITY;
#pragma unroll
        for (int j = 0; j < kPolicyGroup; ++j) {
            l[j] = j < L ? __uint_as_float(v[L * ci + j]) : 0.f;
            if (j < L) m = fmaxf(m, l[j]);
        }
        float e[kPolicyGroup], S = 0.f;
#pragma unroll
        for (int j = 0; j < kPolicyGroup; ++j) {
            e[j] = j < L ? __expf(l[j] - m) : 0.f;
            S += e[j];
        }
        const float T = unit_of(word_of(words, (uint32_t)ci)) * S;
        float cum = 0.f;
        int level = 0;
#pragma unroll
        for (int j = 0; j < kPolicyGroup - 1; ++j) {
            cum += e[j];
            level += (j < L - 1 && cum <= T) ? 1 : 0;
        }
        packed |= (uint32_t)level << (8 * ci);
        if (logits_out)
#pragma unroll
            for (int j = 0; j < kPolicyGroup; ++j)
                if (j < L) logits_out[(long long)ci * L + j] = l[j];
    }
    return packed;
}

// Levels of chargers 16h .. 16h+15 of the env in TMEM lane `tl`, four per
// block; returns them packed 4 per word.
template <int LT>
__device__ __forceinline__ void sample_row(const PolicyArgs& a, uint32_t tl, int h, long long env, bool live,
                                           uint32_t g, uint32_t k0, uint32_t k1, float* logits_env,
                                           uint32_t (&packed)[4])
{
    const int L = LT ? LT : a.n_levels;
    uint4 words[4];                                    // the four Philox blocks of chargers 16h .. 16h+15
#pragma unroll
    for (int blk = 0; blk < 4; ++blk)
        words[blk] = philox4x32_10(make_uint4((uint32_t)env, g, (uint32_t)(4 * h + blk), kPurposePolicy), k0, k1);
#pragma unroll 1
    for (int blk = 0; blk < 4; ++blk) {
        packed[blk] = 0;
        const int c0 = 16 * h + 4 * blk;
        if (c0 >= a.n_ports) break;                    // uniform across the warp
        uint32_t v[48];
        tmem_ld32(tl + (uint32_t)(L * c0), *reinterpret_cast<uint32_t(*)[32]>(v));
        tmem_ld16(tl + (uint32_t)(L * c0 + 32), v + 32);
        tmem_wait_ld();
        if (!live) continue;
        const uint4 w = blk == 0 ? words[0] : blk == 1 ? words[1] : blk == 2 ? words[2] : words[3];
        packed[blk] = sample4<LT>(v, c0, a.n_ports, a.n_levels, w,
                                  logits_env ? logits_env + (long long)c0 * L : nullptr);
    }
}

__device__ __forceinline__ void store_levels(int8_t* dst, int h, int n_ports, const uint32_t (&packed)[4])
{
    if (n_ports == 32) {
        *reinterpret_cast<uint4*>(dst + 16 * h) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int c = 16 * h + j;
            if (c < n_ports) dst[c] = (int8_t)((packed[j >> 2] >> (8 * (j & 3))) & 0xFFu);
        }
    }
}

// ---- common prologue / epilogue of both kernels ------------------------------
__device__ __forceinline__ unsigned char* aligned_smem(unsigned char* raw)
{
    return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~static_cast<uintptr_t>(1023));
}

__device__ __forceinline__ void worker_arrive(uint64_t* bar)
{
    fence_proxy_async();
    fence_before();
    mbar_arrive(bar);
}

// =============================================================================
// k_policy: actions of every env from observations
// =============================================================================
template <int LT>
__global__ void __launch_bounds__(kThreads, 1) k_policy(const __grid_constant__ WMaps wm, const PolicyArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* A = aligned_smem(smem_raw);
    unsigned char* ring = A + kActBytes;
    __shared__ Sync S;
    __shared__ __align__(16) float bias_s[2 * kPolicyHidden + kPolicyMaxPorts * kPolicyGroup];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < 2 * kPolicyHidden + a.n_out_pad; j += blockDim.x) bias_s[j] = a.bias[j];
    if (threadIdx.x == 0) init_sync(S, kPolStages);
    if (warp == 1) tmem_alloc(&S.tmem, kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem;
    const int n_tiles = (a.E + kM - 1) / kM;
    const int my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (warp == 0) {
        if (lane == 0) produce<kPolStages>(&wm, a, ring, S, my_tiles);
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) issue<kPolStages>(a, A, ring, S, tmem, my_tiles);
        __syncwarp();
    } else {
        const int ew = warp - 2, q = warp & 3, h = ew >> 2;
        const int row = 32 * q + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
        const uint32_t abase = smem_addr(A);
        const int D = a.obs_dim;
        const int pairs = ((D + 15) & ~15) >> 1;     // K padded to the MMA's 16
        for (int i = 0; i < my_tiles; ++i) {
            const int tile = (int)blockIdx.x + i * (int)gridDim.x;
            // (1) observations -> BF16 operand (rows ew, ew + 8, ...); kRowBatch
            // rows x 4 column pairs per lane are loaded before any is stored
            constexpr int kRowBatch = 4;
            for (int r0 = ew; r0 < kM; r0 += kWorkerWarps * kRowBatch) {
                float2 x[kRowBatch][4];
#pragma unroll
                for (int j = 0; j < kRowBatch; ++j) {
                    const int r = r0 + j * kWorkerWarps;
                    const long long e = (long long)tile * kM + r;
                    const float* src = a.obs + e * D;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = 2 * (lane + 32 * u);
                        x[j][u] = make_float2(0.f, 0.f);
                        if (r < kM && e < a.E && k < D) x[j][u] = __ldg(reinterpret_cast<const float2*>(src + k));
                    }
                }
#pragma unroll
                for (int j = 0; j < kRowBatch; ++j) {
                    const int r = r0 + j * kWorkerWarps;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int pr = lane + 32 * u;
                        if (r < kM && pr < pairs)
                            st_shared_u32(abase + sw128_offset(r, 2 * pr, kChunkBytes),
                                          pack_bf16x2(x[j][u].x, x[j][u].y));
                    }
                }
            }
            named_sync(kBarWorkers, kWorkers);       // the previous tile's sampling has left TMEM
            layer_bias(a, bias_s, tl, 0, h);
            worker_arrive(&S.xrdy);

            const long long env = (long long)tile * kM + row;
            const bool live = env < a.E;
            uint32_t g = 0, k0 = 0, k1 = 0;
            if (live) {
                const int slot = a.user_to_slot[env];
                g = a.gstep[slot];
                k0 = a.key0[slot];
                k1 = a.key1[slot];
            }
            // (2) hidden layers
            for (int L = 0; L < 2; ++L) {
                wait_sync(&S.acc, (3 * i + L) & 1, S, a.err);
                fence_after();
                hidden_epilogue(tl + (uint32_t)(128 * h), abase, row, 128 * h);
                layer_bias(a, bias_s, tl, L + 1, h);
                worker_arrive(&S.hrdy);
            }
            // (3) logits -> levels
            wait_sync(&S.acc, (3 * i + 2) & 1, S, a.err);
            fence_after();
            uint32_t packed[4];
            sample_row<LT>(a, tl, h, env, live, g, k0, k1,
                           (a.logits && live) ? a.logits + env * a.n_ports * a.n_levels : nullptr, packed);
            fence_before();
            if (live) store_levels(a.actions + env * a.n_ports, h, a.n_ports, packed);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// =============================================================================
// k_rollout: observe -> MLP -> sample -> environment step, T times
// =============================================================================

// Per-station state, held in registers by BOTH worker threads of a station
// (warps 2-5 take its chargers 0-15, warps 6-9 chargers 16-31: "half" 0 and
// 1).  Both halves apply the same station-level updates from the same
// exchanged totals, so their copies stay identical; half 0 writes the
// station's outputs.
struct Owner {
    long long e;
    bool live;
    int half, slot, t, day, cls_row, occ;
    long long pb;
    uint32_t uid, k0, k1, g, ncar, ablk;
    uint4 aw;
    float grid_cap, grid_inv_eta, ret, price;
    uint32_t st_arr, st_rej, st_eps;
    float st_miss, st_chg, last_ret;
    bool ended;
};

// Observation staging: one 8-charger chunk (plus the 8 station features in
// chunk 0) of 16 rows per worker warp; row stride kStageRow floats.
constexpr int kStageRow = 8 + 48 + 4;      // 16-byte aligned rows
constexpr int kObsRows = 16;               // rows per staging round

// values the two halves of a station exchange during a step (per row)
struct Xchg {
    float trail[kM];                       // half 0: power of the group still open after charger 15
    float lead[kM];                        // half 1: power up to its first tail charger
    int first_gs[kM];                      // half 1: group slot of that tail (-1: none)
    float raw[2][kM], over[2][kM], sp[2][kM], se[2][kM], csat[2][kM];
    int nfree[2][kM], occ[2][kM];
};

struct RollSmem {
    float gcap[32 * kM];                   // group slot x row: eta_H * I_H of the group of a tail charger
    union {                                // the step's group scales, then the observation staging
        float gscale[32 * kM];             // group slot x row
        float stage[kWorkerWarps][kObsRows * kStageRow];
    } u;
    Xchg x;
    uint32_t act[kM * kPolicyMaxPorts / 4]; // sampled levels, row-major [row][charger] bytes
    uint32_t gstep[kM], key0[kM], key1[kM];
};

__device__ __forceinline__ uint32_t taddr_of(uint32_t tl, int col) { return tl + (uint32_t)col; }

// car words for the rare step with more than kPreCars arrivals (kept out of line)
__device__ __noinline__ uint4 car_words_late(uint32_t uid, uint32_t n, uint32_t k0, uint32_t k1)
{
    return car_words(uid, n, k0, k1);
}

// Load the station's state (both halves: station fields; each half: its 16
// chargers into TMEM).  Ends with the workers' named barrier (occupancy).
__device__ __forceinline__ void owner_load(Owner& o, const RolloutArgs& R, int tile, int row, int half, uint32_t tl,
                                           RollSmem& rs)
{
    const DevBatch& b = R.b;
    o.e = (long long)tile * kM + row;
    o.live = o.e < R.pol.E;
    o.half = half;
    o.slot = 0; o.pb = 0; o.uid = 0; o.k0 = o.k1 = o.g = o.ncar = 0;
    o.t = 0; o.day = 0; o.cls_row = 0; o.occ = 0;
    o.grid_cap = 1.f; o.grid_inv_eta = 1.f; o.ret = 0.f; o.price = 0.f;
    o.st_arr = o.st_rej = o.st_eps = 0; o.st_miss = o.st_chg = 0.f; o.last_ret = 0.f; o.ended = false;
    o.ablk = 0xFFFFFFFFu;
    o.aw = make_uint4(0, 0, 0, 0);
    if (o.live) {
        o.slot = R.pol.user_to_slot[o.e];
        o.pb = R.port_base + (long long)(o.slot - R.env_base) * R.C;
        o.uid = (uint32_t)b.user_id[o.slot];
        o.k0 = b.key0[o.slot];
        o.k1 = b.key1[o.slot];
        o.g = b.gstep[o.slot];
        o.ncar = b.ncar[o.slot];
        o.t = b.tod[o.slot];
        o.day = b.day[o.slot];
        o.cls_row = b.arrival_class[o.slot];
        o.grid_cap = b.grid_cap[o.slot];
        o.grid_inv_eta = b.grid_inv_eta[o.slot];
        o.ret = b.ep_ret[o.slot];
        o.price = __ldg(b.price + (size_t)o.day * (size_t)R.p.ep_len + (size_t)o.t);
    }
    int occ = 0;
#pragma unroll 1
    for (int kk = 0; kk < 2; ++kk) {
        const int k = 2 * half + kk;
        uint32_t vs[8], ve[8], vc[8], vr[8], vp[8], vw[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = 8 * k + i;
            vs[i] = ve[i] = vc[i] = vr[i] = vp[i] = vw[i] = 0u;
            if (o.live && c < R.C) {
                const long long x = o.pb + c;
                vs[i] = __float_as_uint(b.soc[x]);
                ve[i] = __float_as_uint(b.erem[x]);
                vc[i] = __float_as_uint(b.cap[x]);
                vr[i] = __float_as_uint(b.rbar[x]);
                vw[i] = __float_as_uint(b.pw[x]);
                const uint32_t meta = b.meta[x];
                vp[i] = (uint32_t)b.trem[x] | (meta << 8);
                occ += b.trem[x] > 0 ? 1 : 0;
                if (meta & kMetaTail) rs.gcap[((meta >> kMetaGroupShift) & 31u) * kM + row] = b.gcap[x];
            }
        }
        tmem_st8(taddr_of(tl, kColSoc + 8 * k), vs);
        tmem_st8(taddr_of(tl, kColErem + 8 * k), ve);
        tmem_st8(taddr_of(tl, kColCap + 8 * k), vc);
        tmem_st8(taddr_of(tl, kColRbar + 8 * k), vr);
        tmem_st8(taddr_of(tl, kColPack + 8 * k), vp);
        tmem_st8(taddr_of(tl, kColPw + 8 * k), vw);
    }
    tmem_wait_st();
    rs.x.occ[half][row] = occ;
    if (half == 0) {
        rs.gstep[row] = o.g;
        rs.key0[row] = o.k0;
        rs.key1[row] = o.k1;
    }
    fence_before();
    named_sync(kBarWorkers, kWorkers);
    fence_after();
    o.occ = rs.x.occ[0][row] + rs.x.occ[1][row];
}

// One environment step of the station with this step's sampled levels
// (Appendix A.2 then A.3; the operations of the fused step kernel), this
// thread's half of the chargers, three exchanges with the other half.
__device__ __forceinline__ void owner_step(Owner& o, const RolloutArgs& R, int it, int row, uint32_t tl, RollSmem& rs)
{
    const DevParams& p = R.p;
    const DevBatch& b = R.b;
    const int h = o.half;
    // arrival count of this step (Philox word, Poisson CDF row)
    const uint32_t blk = o.g >> 2;
    if (blk != o.ablk) {
        o.aw = arrival_words(o.uid, o.g, o.k0, o.k1);
        o.ablk = blk;
    }
    const float* F = b.cdf + ((size_t)o.cls_row * (size_t)p.ep_len + (size_t)o.t) * kCdfLen;
    const float4 f0 = __ldg(reinterpret_cast<const float4*>(F));
    const float4 f1 = __ldg(reinterpret_cast<const float4*>(F + 4));
    uint32_t lv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) lv[j] = rs.act[row * (kPolicyMaxPorts / 4) + 4 * h + j];

    // (i) per-charger clip; sums of the groups whose tail is in this half
    float P[16];
    float gacc = 0.f, raw = 0.f, over = 0.f;
    int nfree = 0, last_tail = -1, first_tail = -1, first_gs = -1;
    float lead = 0.f;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const int k = 2 * h + kk;
        uint32_t vs[8], ve[8], vc[8], vr[8], vp[8];
        tmem_ld8(taddr_of(tl, kColSoc + 8 * k), vs);
        tmem_ld8(taddr_of(tl, kColErem + 8 * k), ve);
        tmem_ld8(taddr_of(tl, kColCap + 8 * k), vc);
        tmem_ld8(taddr_of(tl, kColRbar + 8 * k), vr);
        tmem_ld8(taddr_of(tl, kColPack + 8 * k), vp);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int ci = 8 * kk + i;
            const int trem = (int)(vp[i] & 0xFFu);
            const uint32_t meta = vp[i] >> 8;
            const int lvl = (int)((lv[ci >> 2] >> (8 * (ci & 3))) & 0xFFu);
            const bool dc = meta & kMetaDC;
            P[ci] = trem > 0 ? clip_power((float)lvl * (dc ? p.lvl1 : p.lvl0), dc, __uint_as_float(vs[i]), __uint_as_float(ve[i]),
                                          __uint_as_float(vc[i]), __uint_as_float(vr[i]), p)
                             : 0.f;
            raw += P[ci];
            gacc += P[ci];
            nfree += ((meta & kMetaValid) && trem <= 1) ? 1 : 0;    // free once this step's departures left
            if (meta & kMetaTail) {
                const int gs = (int)((meta >> kMetaGroupShift) & 31u);
                if (h == 1 && first_tail < 0) {                      // may close a group opened in half 0
                    first_tail = ci;
                    first_gs = gs;
                    lead = gacc;
                } else {
                    const float gc = rs.gcap[gs * kM + row];
                    rs.u.gscale[gs * kM + row] = gacc > gc ? __fdividef(gc, gacc) : 1.0f;
                    if (p.a_con != 0.f) over = fmaxf(over, (gacc - gc) * __ldg(b.ginv_eta + o.pb + 16 * h + ci));
                }
                last_tail = ci;
                gacc = 0.f;
            }
        }
    }
    if (h == 0) rs.x.trail[row] = gacc;
    else {
        rs.x.lead[row] = lead;
        rs.x.first_gs[row] = first_gs;
    }
    rs.x.raw[h][row] = raw;
    rs.x.over[h][row] = over;
    rs.x.nfree[h][row] = nfree;
    named_sync(kBarWorkers, kWorkers);                               // exchange A

    // the group that closes at half 1's first tail charger (it may have
    // started in half 0): both halves compute its scale
    const int sgs = rs.x.first_gs[row];
    float s_scale = 1.f, s_over = 0.f;
    if (sgs >= 0) {
        const float S = rs.x.trail[row] + rs.x.lead[row];
        const float gc = rs.gcap[sgs * kM + row];
        s_scale = S > gc ? __fdividef(gc, S) : 1.0f;
        // its tail charger is half 1's first tail (an index only half 1 has)
        if (h == 1 && p.a_con != 0.f) s_over = (S - gc) * __ldg(b.ginv_eta + o.pb + 16 + first_tail);
    }
    const int nfree0 = rs.x.nfree[0][row], nfree1 = rs.x.nfree[1][row];
    // architecture constraint: charger power scaled by its group
    float sp = 0.f;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const int k = 2 * h + kk;
        uint32_t vp[8];
        tmem_ld8(taddr_of(tl, kColPack + 8 * k), vp);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int ci = 8 * kk + i;
            const uint32_t meta = vp[i] >> 8;
            const bool in_split = h == 0 ? ci > last_tail : (first_tail >= 0 && ci <= first_tail);
            float sc = 1.f;
            if (in_split) sc = s_scale;
            else if (meta & kMetaValid) sc = rs.u.gscale[((meta >> kMetaGroupShift) & 31u) * kM + row];
            P[ci] *= sc;
            sp += P[ci];
        }
    }
    rs.x.sp[h][row] = sp;
    named_sync(kBarWorkers, kWorkers);                               // exchange B
    const float sp_all = rs.x.sp[0][row] + rs.x.sp[1][row];
    const float raw_all = rs.x.raw[0][row] + rs.x.raw[1][row];
    const float s_root = sp_all > o.grid_cap ? __fdividef(o.grid_cap, sp_all) : 1.0f;
    float c_con = 0.f;
    if (p.a_con != 0.f) {
        // s_over was formed by half 1 with the right tail; half 0 takes it from the exchange
        if (h == 1) rs.x.over[1][row] = fmaxf(rs.x.over[1][row], s_over);
    }

    // Poisson count: the smallest k with u < F_k (F nondecreasing, F_127 = inf)
    const uint32_t word = word_of(o.aw, o.g & 3u);
    const float u = __fmul_rn(__uint2float_rn(word >> 8), 0x1p-24f);
    int M = (u >= f0.x) + (u >= f0.y) + (u >= f0.z) + (u >= f0.w) + (u >= f1.x) + (u >= f1.y) + (u >= f1.z) +
            (u >= f1.w);
    if (M == 8)
        while (u >= __ldg(F + M)) ++M;
    // first come first served: half 0's free chargers take the first cars
    const int adm0 = min(M, nfree0), adm1 = min(M - adm0, nfree1);
    const int quota = h == 0 ? adm0 : adm1;
    const uint32_t car0 = o.ncar + (uint32_t)(h == 0 ? 0 : adm0);
    constexpr int kPreCars = 4;
    uint4 cw[kPreCars];
#pragma unroll
    for (int j = 0; j < kPreCars; ++j)
        cw[j] = j < quota ? car_words(o.uid, car0 + (uint32_t)j, o.k0, o.k1) : make_uint4(0, 0, 0, 0);

    // (ii) charge, (iii) departures, (iv) arrivals, and the episode end
    const bool fin = o.t + 1 >= p.ep_len;
    float se = 0.f, c_sat = 0.f;
    int adm = 0, occ = 0;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const int k = 2 * h + kk;
        uint32_t vs[8], ve[8], vc[8], vr[8], vp[8], vw[8];
        tmem_ld8(taddr_of(tl, kColSoc + 8 * k), vs);
        tmem_ld8(taddr_of(tl, kColErem + 8 * k), ve);
        tmem_ld8(taddr_of(tl, kColCap + 8 * k), vc);
        tmem_ld8(taddr_of(tl, kColRbar + 8 * k), vr);
        tmem_ld8(taddr_of(tl, kColPack + 8 * k), vp);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int ci = 8 * kk + i;
            int trem = (int)(vp[i] & 0xFFu);
            const uint32_t meta = vp[i] >> 8;
            const bool dc = meta & kMetaDC;
            float soc = __uint_as_float(vs[i]), erem = __uint_as_float(ve[i]);
            float cap = __uint_as_float(vc[i]), rbar = __uint_as_float(vr[i]);
            const float Pq = P[ci] * s_root;
            se += P[ci] * (dc ? p.inv_eta1 : p.inv_eta0);
            float pw = Pq;
            if (trem > 0) {
                const float dE = Pq * p.dt;
                soc = fminf(soc + __fdividef(dE, cap), 1.0f);
                erem = fmaxf(erem - dE, 0.0f);
                trem -= 1;
                if (trem == 0) {
                    c_sat += erem;
                    soc = 0.f; erem = 0.f; cap = 0.f; rbar = 0.f;
                }
            }
            if ((meta & kMetaValid) && trem == 0 && adm < quota) {
                const uint4 w = adm == 0 ? cw[0]
                              : adm == 1 ? cw[1]
                              : adm == 2 ? cw[2]
                              : adm == 3 ? cw[3]
                                         : car_words_late(o.uid, car0 + (uint32_t)adm, o.k0, o.k1);
                const Car car = car_from_words(w, dc, p);
                cap = car.cap; soc = car.soc; erem = car.erem; rbar = car.rbar;
                trem = car.stay;
                ++adm;
            }
            if (fin) {
                soc = 0.f; erem = 0.f; cap = 0.f; rbar = 0.f; pw = 0.f;
                trem = 0;
            }
            occ += trem > 0 ? 1 : 0;
            vs[i] = __float_as_uint(soc);
            ve[i] = __float_as_uint(erem);
            vc[i] = __float_as_uint(cap);
            vr[i] = __float_as_uint(rbar);
            vp[i] = (uint32_t)trem | (meta << 8);
            vw[i] = __float_as_uint(pw);
        }
        tmem_st8(taddr_of(tl, kColSoc + 8 * k), vs);
        tmem_st8(taddr_of(tl, kColErem + 8 * k), ve);
        tmem_st8(taddr_of(tl, kColCap + 8 * k), vc);
        tmem_st8(taddr_of(tl, kColRbar + 8 * k), vr);
        tmem_st8(taddr_of(tl, kColPack + 8 * k), vp);
        tmem_st8(taddr_of(tl, kColPw + 8 * k), vw);
    }
    tmem_wait_st();
    rs.x.se[h][row] = se;
    rs.x.csat[h][row] = c_sat;
    rs.x.occ[h][row] = occ;
    named_sync(kBarWorkers, kWorkers);                               // exchange C
    const float se_all = rs.x.se[0][row] + rs.x.se[1][row];
    const float csat_all = rs.x.csat[0][row] + rs.x.csat[1][row];
    const int adm_all = adm0 + adm1;
    if (p.a_con != 0.f) {
        const float over_all = fmaxf(rs.x.over[0][row], rs.x.over[1][row]);
        c_con = fmaxf(fmaxf(over_all, (raw_all - o.grid_cap) * o.grid_inv_eta), 0.f);
    }
    o.occ = rs.x.occ[0][row] + rs.x.occ[1][row];

    // reward, Appendix A.3
    const float e_net = sp_all * s_root * p.dt;
    const float e_grid = se_all * s_root * p.dt;
    o.ncar += (uint32_t)adm_all;
    const float profit = p.p_sell * e_net - o.price * e_grid - p.c_fixed;
    const float r = profit - p.a_sat * csat_all - p.a_decl * (float)(M - adm_all) - p.a_con * c_con;
    o.ret += r;
    o.t += 1;
    o.st_arr += (uint32_t)adm_all;
    o.st_rej += (uint32_t)(M - adm_all);
    o.st_miss += csat_all;
    o.st_chg += e_net;
    if (fin) {
        o.last_ret = o.ret;
        o.ended = true;
        o.st_eps += 1u;
        o.ret = 0.f;
        o.t = 0;
        o.day = draw_day(o.uid, o.g, 0u, o.k0, o.k1, p.n_days);
    }
    o.g += 1u;
    if (o.live) {
        if (h == 0) {
            const long long out = (long long)it * R.pol.E + o.e;
            if (R.reward) R.reward[out] = r;
            if (R.done) R.done[out] = fin ? 1 : 0;
        }
        o.price = __ldg(b.price + (size_t)o.day * (size_t)p.ep_len + (size_t)o.t);
    }
    if (h == 0) rs.gstep[row] = o.g;
}

// Observation after the step: this half's chunks (half 0 also the 8 station
// features), every lane on its own row; BF16 into the layer-1 operand, FP32
// to HBM through the warp's staging buffer, 16 rows at a time, each row's
// chunk a contiguous, 16-byte aligned run.
__device__ __forceinline__ void owner_observe(const Owner& o, const RolloutArgs& R, int it, int q, int lane, uint32_t tl,
                                              uint32_t abase, float* stage)
{
    const DevParams& p = R.p;
    const int D = R.pol.obs_dim, N = R.pol.n_ports;
    const int row = 32 * q + lane;
    const long long e0 = o.e - lane;                        // env of the warp's first row
    const int n_chunks = (N + 7) >> 3;
#pragma unroll 1
    for (int kk = 0; kk < 2; ++kk) {
        const int k = 2 * o.half + kk;
        if (k >= n_chunks) break;                           // uniform across the warp
        uint32_t vs[8], ve[8], vr[8], vp[8], vw[8];
        tmem_ld8(taddr_of(tl, kColSoc + 8 * k), vs);
        tmem_ld8(taddr_of(tl, kColErem + 8 * k), ve);
        tmem_ld8(taddr_of(tl, kColRbar + 8 * k), vr);
        tmem_ld8(taddr_of(tl, kColPack + 8 * k), vp);
        tmem_ld8(taddr_of(tl, kColPw + 8 * k), vw);
        tmem_wait_ld();
        // features [f0, f1): the station's 8 in chunk 0, then 6 per charger
        const int f0 = k == 0 ? 0 : 8 + 48 * k;
        const int f1 = min(8 + 48 * (k + 1), D);
        float st8[8], cf[48];
        if (k == 0 && o.live) obs_env(st8, o.t, o.day, o.occ, N, 0.f, 0.f, R.b, p);   // charge-only mode
        else
#pragma unroll
            for (int f = 0; f < 8; ++f) st8[f] = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = 8 * k + i;
            if (o.live && c < N) {
                obs_port<false>(cf + 6 * i, (int)(vp[i] & 0xFFu), 0, __uint_as_float(vs[i]), __uint_as_float(ve[i]),
                         __uint_as_float(vr[i]), __uint_as_float(vw[i]), (vp[i] >> 8) & kMetaDC, p);
            } else {
#pragma unroll
                for (int x = 0; x < 6; ++x) cf[6 * i + x] = 0.f;
            }
        }
        // feature f0 + j (j a compile-time index after unrolling)
        auto V = [&](int j) -> float {
            if (k == 0) return j < 8 ? st8[j < 8 ? j : 0] : cf[j >= 8 && j < 56 ? j - 8 : 0];
            return j < 48 ? cf[j < 48 ? j : 0] : 0.f;
        };
        // BF16 into the operand (pairs; the K padding up to 16 is zero)
        const int n_f = f1 - f0;
        const bool last = k == n_chunks - 1;
        const int n_fp = last ? (((D + 15) & ~15) - f0) : n_f;
#pragma unroll
        for (int j = 0; j < 56; j += 2) {
            if (j < n_fp) {
                const float x0 = j < n_f ? V(j) : 0.f, x1 = j + 1 < n_f ? V(j + 1) : 0.f;
                st_shared_u32(abase + sw128_offset(row, f0 + j, kChunkBytes), pack_bf16x2(x0, x1));
            }
        }
        if (last && n_fp > 56) {                             // padding beyond the chunk's own width
            for (int j = 56; j < n_fp; j += 2) st_shared_u32(abase + sw128_offset(row, f0 + j, kChunkBytes), 0u);
        }
        if (R.obs_out) {
#pragma unroll 1
            for (int half_rows = 0; half_rows < 2; ++half_rows) {
                if ((lane >> 4) == half_rows) {
                    float* srow = stage + (lane & 15) * kStageRow;
#pragma unroll
                    for (int j = 0; j < 56; j += 4)
                        if (j < n_f)
                            *reinterpret_cast<float4*>(srow + j) = make_float4(V(j), V(j + 1), V(j + 2), V(j + 3));
                }
                __syncwarp();
                const long long eb = e0 + 16 * half_rows;
                const int n_rows = (int)min(16LL, max(0LL, (long long)R.pol.E - eb));
                float* dst0 = R.obs_out + ((long long)it * R.pol.E + eb) * D + f0;
                // two rows per pass, 16 lanes per row (a row's run is at most 14 float4)
                const int cl = lane & 15;
                if ((D & 3) == 0) {
                    if (4 * cl < n_f)
#pragma unroll 4
                        for (int r = lane >> 4; r < n_rows; r += 2)
                            *reinterpret_cast<float4*>(dst0 + (long long)r * D + 4 * cl) =
                                *reinterpret_cast<const float4*>(stage + r * kStageRow + 4 * cl);
                } else {
#pragma unroll 4
                    for (int r = lane >> 4; r < n_rows; r += 2)
                        for (int c2 = cl; 2 * c2 < n_f; c2 += 16)
                            *reinterpret_cast<float2*>(dst0 + (long long)r * D + 2 * c2) =
                                *reinterpret_cast<const float2*>(stage + r * kStageRow + 2 * c2);
                }
                __syncwarp();
            }
        }
    }
}

// State back to HBM: each half its chargers, half 0 the station fields.
__device__ __forceinline__ void owner_store(const Owner& o, const RolloutArgs& R, uint32_t tl)
{
    const DevBatch& b = R.b;
#pragma unroll 1
    for (int kk = 0; kk < 2; ++kk) {
        const int k = 2 * o.half + kk;
        uint32_t vs[8], ve[8], vc[8], vr[8], vp[8], vw[8];
        tmem_ld8(taddr_of(tl, kColSoc + 8 * k), vs);
        tmem_ld8(taddr_of(tl, kColErem + 8 * k), ve);
        tmem_ld8(taddr_of(tl, kColCap + 8 * k), vc);
        tmem_ld8(taddr_of(tl, kColRbar + 8 * k), vr);
        tmem_ld8(taddr_of(tl, kColPack + 8 * k), vp);
        tmem_ld8(taddr_of(tl, kColPw + 8 * k), vw);
        tmem_wait_ld();
        if (!o.live) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = 8 * k + i;
            if (c < R.C) {
                const long long x = o.pb + c;
                b.soc[x] = __uint_as_float(vs[i]);
                b.erem[x] = __uint_as_float(ve[i]);
                b.cap[x] = __uint_as_float(vc[i]);
                b.rbar[x] = __uint_as_float(vr[i]);
                b.pw[x] = __uint_as_float(vw[i]);
                b.trem[x] = (uint8_t)(vp[i] & 0xFFu);
            }
        }
    }
    if (!o.live || o.half != 0) return;
    const int s = o.slot;
    b.tod[s] = o.t;
    b.day[s] = o.day;
    b.gstep[s] = o.g;
    b.ncar[s] = o.ncar;
    b.ep_ret[s] = o.ret;
    if (o.ended) b.last_ret[s] = o.last_ret;
    b.n_episodes[s] += o.st_eps;
    b.st_arrived[s] += o.st_arr;
    b.st_rejected[s] += o.st_rej;
    b.st_missing[s] += o.st_miss;
    b.st_charged[s] += o.st_chg;
}

template <int LT>
__global__ void __launch_bounds__(kThreads, 1) k_rollout(const __grid_constant__ WMaps wm, const RolloutArgs R)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* A = aligned_smem(smem_raw);
    unsigned char* ring = A + kActBytes;
    RollSmem& rs = *reinterpret_cast<RollSmem*>(ring + kRollStages * kStageBytes);
    __shared__ Sync S;
    __shared__ __align__(16) float bias_s[2 * kPolicyHidden + kPolicyMaxPorts * kPolicyGroup];
    const PolicyArgs& a = R.pol;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < 2 * kPolicyHidden + a.n_out_pad; j += blockDim.x) bias_s[j] = a.bias[j];
    if (threadIdx.x == 0) init_sync(S, kRollStages);
    if (warp == 1) tmem_alloc(&S.tmem, kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem;
    const int tile = blockIdx.x;
    if (warp == 0) {
        if (lane == 0) produce<kRollStages>(&wm, a, ring, S, R.T);
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) issue<kRollStages>(a, A, ring, S, tmem, R.T);
        __syncwarp();
    } else {
        const int ew = warp - 2, q = warp & 3, h = ew >> 2;
        const int row = 32 * q + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
        const uint32_t abase = smem_addr(A);
        const long long env = (long long)tile * kM + row;
        const bool live = env < a.E;
        Owner o;
        owner_load(o, R, tile, row, h, tl, rs);
        owner_observe(o, R, 0, q, lane, tl, abase, rs.u.stage[ew]);
        for (int it = 0; it < R.T; ++it) {
            fence_before();
            named_sync(kBarWorkers, kWorkers);     // every observation (and its parked power) written
            fence_after();
            layer_bias(a, bias_s, tl, 0, h);
            worker_arrive(&S.xrdy);
            for (int L = 0; L < 2; ++L) {
                wait_sync(&S.acc, (3 * it + L) & 1, S, a.err);
                fence_after();
                hidden_epilogue(tl + (uint32_t)(128 * h), abase, row, 128 * h);
                layer_bias(a, bias_s, tl, L + 1, h);
                worker_arrive(&S.hrdy);
            }
            wait_sync(&S.acc, (3 * it + 2) & 1, S, a.err);
            fence_after();
            uint32_t packed[4];
            sample_row<LT>(a, tl, h, env, live, rs.gstep[row], rs.key0[row], rs.key1[row],
                           (a.logits && live) ? a.logits + ((long long)it * a.E + env) * a.n_ports * a.n_levels
                                              : nullptr,
                           packed);
#pragma unroll
            for (int j = 0; j < 4; ++j) rs.act[row * (kPolicyMaxPorts / 4) + 4 * h + j] = packed[j];
            if (live) store_levels(a.actions + ((long long)it * a.E + env) * a.n_ports, h, a.n_ports, packed);
            fence_before();
            named_sync(kBarWorkers, kWorkers);
            fence_after();
            owner_step(o, R, it, row, tl, rs);
            named_sync(kBarWorkers, kWorkers);                 // group scales done: the staging may overwrite them
            if (it + 1 < R.T) owner_observe(o, R, it + 1, q, lane, tl, abase, rs.u.stage[ew]);
        }
        owner_store(o, R, tl);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

constexpr int kPolicySmem = 1024 + kActBytes + kPolStages * kStageBytes;
constexpr int kRolloutSmem = 1024 + kActBytes + kRollStages * kStageBytes + (int)sizeof(RollSmem);
static_assert(kPolicySmem <= 227 * 1024 - 256, "k_policy shared memory");
static_assert(kRolloutSmem + (2 * kPolicyHidden + kPolicyMaxPorts * kPolicyGroup) * 4 <= 227 * 1024 - 256,
              "k_rollout shared memory");

// Bounded-wait self-test: one thread runs the kernels' wait on an mbarrier
// that nothing arrives on.  The wait must give up after kWaitCycles, raise
// the error flag and return; out = {gave up, shared flag set, elapsed cycles
// / 2^20}.
__global__ void k_wait_selftest(uint32_t* err, int* out)
{
    __shared__ Sync S;
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    S.bad = 0;
    mbar_fence_init();
    const long long t0 = clock64();
    const bool done = wait_sync<true>(&bar, 0, S, err);
    out[0] = done ? 0 : 1;
    out[1] = is_bad(S) ? 1 : 0;
    out[2] = (int)((clock64() - t0) >> 20);
}

}  // namespace

cudaError_t wait_selftest(uint32_t* err, int* d_out, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(err, d_out);
    return cudaGetLastError();
}

int policy_smem_bytes() { return kPolicySmem; }

cudaError_t policy_prepare()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_policy<11>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPolicySmem))) return e;
    if ((e = cudaFuncSetAttribute(k_policy<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPolicySmem))) return e;
    if ((e = cudaFuncSetAttribute(k_rollout<11>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRolloutSmem)))
        return e;
    return cudaFuncSetAttribute(k_rollout<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRolloutSmem);
}

cudaError_t launch_policy(const WMaps& wm, const PolicyArgs& a, int sm_count, cudaStream_t st)
{
    const int n_tiles = (a.E + kM - 1) / kM;
    const int grid = n_tiles < sm_count ? n_tiles : sm_count;
    if (grid <= 0) return cudaSuccess;
    if (a.n_levels == 11)
        k_policy<11><<<grid, kThreads, kPolicySmem, st>>>(wm, a);
    else
        k_policy<0><<<grid, kThreads, kPolicySmem, st>>>(wm, a);
    return cudaGetLastError();
}

bool rollout_fits(int n_out_pad) { return n_out_pad <= kColSoc; }
int policy_stage_rows() { return kStageRows; }

cudaError_t launch_rollout(const WMaps& wm, const RolloutArgs& r, cudaStream_t st)
{
    const int n_tiles = (r.pol.E + kM - 1) / kM;
    if (n_tiles <= 0 || r.T <= 0) return cudaSuccess;
    if (r.pol.n_levels == 11)
        k_rollout<11><<<n_tiles, kThreads, kRolloutSmem, st>>>(wm, r);
    else
        k_rollout<0><<<n_tiles, kThreads, kRolloutSmem, st>>>(wm, r);
    return cudaGetLastError();
}

}  // namespace chx
