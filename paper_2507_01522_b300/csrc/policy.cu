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
constexpr int kRollStages = 4;             // weight ring of k_rollout
constexpr int kMaxStages = kPolStages;
constexpr int kBarWorkers = 1;             // named barrier of the worker warps

// k_rollout: TMEM columns of the env state, 32 per field (charger c at +c)
constexpr int kColSoc = 352, kColErem = 384, kColCap = 416, kColRbar = 448;
constexpr int kColPack = 480;              // remaining stay | meta << 8
// k_rollout: the next observation's BF16 operand rows, packed in pairs,
// parked by the environment step (columns the output layer's accumulator
// has left free) until the observation pass copies them into the operand;
// part k's run at columns kColObs + 32 k ..
constexpr int kColObs = 0;

struct Sync {
    uint64_t full[kMaxStages], empty[kMaxStages];
    uint64_t acc;                          // a layer is accumulated (3 completions per pass)
    uint64_t xrdy;                         // layer-1 operand written (one arrival per worker thread)
    uint64_t hrdy;                         // h1 / h2 written (one arrival per worker thread, 2 per pass)
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

__device__ __forceinline__ void init_sync(Sync& S, int n_stages, int n_workers)
{
    for (int s = 0; s < n_stages; ++s) {
        mbar_init(&S.full[s], 1);
        mbar_init(&S.empty[s], 1);             // the MMA commit that has read the stage
    }
    mbar_init(&S.acc, 1);
    mbar_init(&S.fin, 1);
    mbar_init(&S.xrdy, n_workers);
    mbar_init(&S.hrdy, n_workers);
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
// kBiasTmem: every layer accumulates onto the bias the workers placed in
// TMEM; else each layer's first MMA overwrites the accumulator and the
// workers add the bias when they read it.
template <int NS, bool kBiasTmem = true>
__device__ void issue(const PolicyArgs& a, unsigned char* A, unsigned char* ring, Sync& S, uint32_t tmem,
                      int n_passes)
{
    // descriptors of the operand's and the ring's first rows; a K = 16 step
    // (32 bytes) or a chunk / stage further is an offset in 16-byte units
    // (both buffers lie far below the field's 256 KB limit)
    const uint64_t a0 = sdesc_sw128(A), r0 = sdesc_sw128(ring);
    uint32_t s = 0;
    for (int it = 0; it < n_passes; ++it) {
        wait_sync<false>(&S.xrdy, it & 1, S, a.err);
        fence_after();
#pragma unroll
        for (int L = 0; L < 3; ++L) {      // unrolled: the issue sequence of each layer is straight-line code
            if (L > 0) {
                wait_sync<false>(&S.hrdy, (2 * it + L - 1) & 1, S, a.err);
                fence_after();
            }
            const int parts = L < 2 ? 1 : a.parts3;
            const int chunks = L == 0 ? a.ch1 : 4;
            for (int p = 0; p < parts; ++p) {
                const uint32_t id = idesc_bf16_f32(kM, part_rows(a, L, p));
                const uint32_t dt = tmem + (uint32_t)(p * kStageRows);
                for (int k = 0; k < chunks; ++k, ++s) {
                    const uint32_t slot = s % NS;
                    wait_sync<false>(&S.full[slot], (s / NS) & 1, S, a.err);
                    fence_after();
                    if (is_bad(S)) continue;
                    const int nks = (L == 0 && k == chunks - 1) ? a.ks1_last : 4;
                    const uint64_t ad = a0 + (uint64_t)((k * kChunkBytes) >> 4);
                    const uint64_t bd = r0 + (uint64_t)((slot * kStageBytes) >> 4);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (j < nks) mma_bf16(dt, ad + 2 * j, bd + 2 * j, id, kBiasTmem || k > 0 || j > 0);
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

// ---- epilogue of layers 1 and 2: ReLU, BF16 into A (NB blocks of 32 columns)
// bias (layer's bias vector, or nullptr when it is already in TMEM) is
// added to the accumulator before the ReLU
template <int NB>
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, uint32_t abase, int row, int col0,
                                                const float* bias = nullptr)
{
#pragma unroll 1
    for (int blk = 0; blk < NB; ++blk) {
        const int c = col0 + 32 * blk;
        uint32_t v[32];
        tmem_ld32(taddr + (uint32_t)(32 * blk), v);
        tmem_wait_ld();
        if (bias) {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = __float_as_uint(__uint_as_float(v[j]) + bias[c + j]);
        }
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
    if (threadIdx.x == 0) init_sync(S, kPolStages, kWorkers);
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
                hidden_epilogue<4>(tl + (uint32_t)(128 * h), abase, row, 128 * h);
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
//
// Sixteen worker warps: warp 2 + w serves TMEM lane quadrant (2 + w) % 4 and
// part p = w / 4 of every station row there: chargers 8p .. 8p + 7 in the
// sampling, the environment step and the observation, and hidden columns
// 64p .. 64p + 63 in the epilogues.  So a station is served by four threads,
// and every CUDA-core phase has twice the warps of k_policy to hide latency.

constexpr int kRollWorkerWarps = 16;
constexpr int kRollWorkers = kRollWorkerWarps * 32;
constexpr int kRollThreads = (2 + kRollWorkerWarps) * 32;
constexpr int kParts = 4;                  // threads per station
constexpr int kBarQuad = 2;                // named barriers 2..5: the four warps that share rows 32q .. 32q + 31
constexpr int kPartPorts = 8;              // chargers per part
static_assert(kParts * kPartPorts == 32, "a part's chargers tile the 32 columns of a station's state block");

// A station's scalars between steps, one record per row in shared memory:
// part 0 writes it at the end of a step, every part reads it (the phases are
// barrier-separated), so registers hold them only inside the step.
struct RowState {
    int slot[kM], t[kM], day[kM], occ[kM], cls_row[kM];
    uint32_t uid[kM], k0[kM], k1[kM], g[kM], ncar[kM], ablk[kM];
    uint4 aw[kM];
    float ret[kM];
};

// The station's state during a step, in the registers of all four threads
// of the station.  They apply the same station-level updates from the same
// exchanged totals, so their copies stay identical; part 0 writes the
// station's outputs and its record.
struct Owner {
    long long e;
    bool live;
    int part, slot, t, day, cls_row, occ;
    long long pb;
    uint32_t uid, k0, k1, g, ncar, ablk;
    uint4 aw;
    float grid_cap, grid_inv_eta, ret, price;
};

// the station's running statistics of the rollout, kept by part 0
struct RowStats {
    uint32_t arr[kM], rej[kM], eps[kM], ended[kM];
    float miss[kM], chg[kM], last_ret[kM];
};

// values the four parts of a station exchange during a step (per part, row);
// the second members of the unions are written only after every read of the
// first (the exchanges are barrier-separated)
struct Xchg {
    union { float lead[kParts][kM]; float sp[kParts][kM]; };      // sum up to the part's first tail when
                                                                   // that group began earlier | scaled sum
    union { float trail[kParts][kM]; float se[kParts][kM]; };     // sum after the part's last tail (all of
                                                                   // the part if it has none) | grid energy
    union { int first_gs[kParts][kM]; float csat[kParts][kM]; };  // slot of that first tail (-1) | c_sat
    union { int has_tail[kParts][kM]; int occ[kParts][kM]; };
    float raw[kParts][kM], over[kParts][kM];
    int nfree[kParts][kM];
};

// What the sampling and the environment step share, placed in the
// activation operand: from the completion of a step's last layer (the
// tensor core has read the operand) until the next observation is written
// into it (after the workers' barrier that ends the step), the operand
// holds nothing live.
struct StepScratch {
    float gscale[32 * kM];                 // group slot x row
    Xchg x;
    uint32_t act[kM * kPolicyMaxPorts / 4]; // sampled levels, row-major [row][charger] bytes
};
static_assert(sizeof(StepScratch) <= kActBytes, "the step's scratch fits in the activation operand");

// per-CTA state that lives for the whole rollout
struct RollSmem {
    RowStats st;
    RowState rw;
    float pw[kPolicyMaxPorts * kM];        // charger x row: the last applied power
};

// the station's record -> registers (every part, at the start of a step)
__device__ __forceinline__ void owner_get(Owner& o, const RolloutArgs& R, long long e, int row, int part,
                                          const RollSmem& rs)
{
    const DevBatch& b = R.b;
    const RowState& w = rs.rw;
    o.e = e;
    o.live = e < R.pol.E;
    o.part = part;
    o.slot = w.slot[row];
    o.t = w.t[row];
    o.day = w.day[row];
    o.occ = w.occ[row];
    o.cls_row = w.cls_row[row];
    o.uid = w.uid[row];
    o.k0 = w.k0[row];
    o.k1 = w.k1[row];
    o.g = w.g[row];
    o.ncar = w.ncar[row];
    o.ablk = w.ablk[row];
    o.aw = w.aw[row];
    o.ret = w.ret[row];
    o.pb = R.port_base + (long long)(o.slot - R.env_base) * R.C;
    o.grid_cap = o.live ? __ldg(b.grid_cap + o.slot) : 1.f;
    o.grid_inv_eta = o.live ? __ldg(b.grid_inv_eta + o.slot) : 1.f;
    o.price = o.live ? __ldg(b.price + (size_t)o.day * (size_t)R.p.ep_len + (size_t)o.t) : 0.f;
}

// registers -> the station's record (part 0)
__device__ __forceinline__ void owner_put(const Owner& o, int row, RollSmem& rs)
{
    RowState& w = rs.rw;
    w.slot[row] = o.slot;
    w.t[row] = o.t;
    w.day[row] = o.day;
    w.occ[row] = o.occ;
    w.cls_row[row] = o.cls_row;
    w.uid[row] = o.uid;
    w.k0[row] = o.k0;
    w.k1[row] = o.k1;
    w.g[row] = o.g;
    w.ncar[row] = o.ncar;
    w.ablk[row] = o.ablk;
    w.aw[row] = o.aw;
    w.ret[row] = o.ret;
}

__device__ __forceinline__ uint32_t taddr_of(uint32_t tl, int col) { return tl + (uint32_t)col; }

// car words beyond the pre-drawn ones (kept out of line)
__device__ __noinline__ uint4 car_words_late(uint32_t uid, uint32_t n, uint32_t k0, uint32_t k1)
{
    return car_words(uid, n, k0, k1);
}

// Levels of chargers 8 part .. 8 part + 7 of the env in TMEM lane `tl`, four
// per block; returns them packed 4 per word.
template <int LT>
__device__ __forceinline__ void sample_part(const PolicyArgs& a, uint32_t tl, int part, long long env, bool live,
                                            uint32_t g, uint32_t k0, uint32_t k1, float* logits_env,
                                            uint32_t (&packed)[2], const float* bias3)
{
    const int L = LT ? LT : a.n_levels;
    uint4 words[2];
#pragma unroll
    for (int blk = 0; blk < 2; ++blk)
        words[blk] = philox4x32_10(make_uint4((uint32_t)env, g, (uint32_t)(2 * part + blk), kPurposePolicy), k0, k1);
#pragma unroll 1
    for (int blk = 0; blk < 2; ++blk) {
        packed[blk] = 0;
        const int c0 = 8 * part + 4 * blk;
        if (c0 >= a.n_ports) break;                    // uniform across the warp
        uint32_t v[48];
        tmem_ld32(tl + (uint32_t)(L * c0), *reinterpret_cast<uint32_t(*)[32]>(v));
        tmem_ld16(tl + (uint32_t)(L * c0 + 32), v + 32);
        tmem_wait_ld();
        if (!live) continue;
#pragma unroll
        for (int j = 0; j < 4 * kPolicyGroup; ++j)     // the output layer's bias (columns past the last used: 0)
            if (j < 4 * L) v[j] = __float_as_uint(__uint_as_float(v[j]) + bias3[L * c0 + j]);
        packed[blk] = sample4<LT>(v, c0, a.n_ports, a.n_levels, blk == 0 ? words[0] : words[1],
                                  logits_env ? logits_env + (long long)c0 * L : nullptr);
    }
}

__device__ __forceinline__ void store_levels_part(int8_t* dst, int part, int n_ports, const uint32_t (&packed)[2])
{
    if (n_ports == 32) {
        *reinterpret_cast<uint2*>(dst + 8 * part) = make_uint2(packed[0], packed[1]);
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 8 * part + j;
            if (c < n_ports) dst[c] = (int8_t)((packed[j >> 2] >> (8 * (j & 3))) & 0xFFu);
        }
    }
}

// Load the station's state (every part: station fields; each part: its 8
// chargers into TMEM).  Ends with the workers' named barrier (occupancy).
__device__ __forceinline__ void owner_load(Owner& o, const RolloutArgs& R, int tile, int row, int part, uint32_t tl,
                                           RollSmem& rs, StepScratch& sx)
{
    const DevBatch& b = R.b;
    o.e = (long long)tile * kM + row;
    o.live = o.e < R.pol.E;
    o.part = part;
    o.slot = 0; o.pb = 0; o.uid = 0; o.k0 = o.k1 = o.g = o.ncar = 0;
    o.t = 0; o.day = 0; o.cls_row = 0; o.occ = 0;
    o.grid_cap = 1.f; o.grid_inv_eta = 1.f; o.ret = 0.f; o.price = 0.f;
    o.ablk = 0xFFFFFFFFu;
    if (part == 0) {
        rs.st.arr[row] = rs.st.rej[row] = rs.st.eps[row] = rs.st.ended[row] = 0u;
        rs.st.miss[row] = rs.st.chg[row] = rs.st.last_ret[row] = 0.f;
    }
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
    uint32_t vs[8], ve[8], vc[8], vr[8], vp[8], vw[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = 8 * part + i;
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
        }
    }
    tmem_st8(taddr_of(tl, kColSoc + 8 * part), vs);
    tmem_st8(taddr_of(tl, kColErem + 8 * part), ve);
    tmem_st8(taddr_of(tl, kColCap + 8 * part), vc);
    tmem_st8(taddr_of(tl, kColRbar + 8 * part), vr);
    tmem_st8(taddr_of(tl, kColPack + 8 * part), vp);
#pragma unroll
    for (int i = 0; i < 8; ++i) rs.pw[(8 * part + i) * kM + row] = __uint_as_float(vw[i]);
    tmem_wait_st();
    sx.x.occ[part][row] = occ;
    fence_before();
    named_sync(kBarWorkers, kRollWorkers);
    fence_after();
    o.occ = 0;
#pragma unroll
    for (int j = 0; j < kParts; ++j) o.occ += sx.x.occ[j][row];
    if (part == 0) owner_put(o, row, rs);
    named_sync(kBarWorkers, kRollWorkers);           // every read done: the operand may be written
}

// FP32 observation rows as 32-byte sectors: the row length and the buffer
// keep every part's run, and each half of it, 32-byte aligned (uniform for
// the launch).  The environment step then writes the next observation's
// rows itself while its state is in registers.
__device__ __forceinline__ bool obs_sectors(const RolloutArgs& R)
{
    return R.obs_out && (R.pol.obs_dim & 7) == 0 && (reinterpret_cast<uintptr_t>(R.obs_out) & 31) == 0;
}

// The environment step parks the next observation's operand rows in TMEM
// when every half part (4 chargers, 24 features) is complete or empty.
// (The FP32 rows then come from the environment step too, or are not asked for.)
__device__ __forceinline__ bool obs_parked(const RolloutArgs& R)
{
    return (R.pol.n_ports & 3) == 0 && (R.obs_out == nullptr || obs_sectors(R));
}

// One environment step of the station with this step's sampled levels
// (Appendix A.2 then A.3; the operations of the fused step kernel), this
// thread's 8 chargers, four exchanges with the other parts (each a barrier
// of the four warps that hold these rows only).
__device__ __forceinline__ void owner_step(const RolloutArgs& R, long long e, int part, int it, int row, uint32_t tl,
                                           RollSmem& rs, StepScratch& sx)
{
    Owner o;
    owner_get(o, R, e, row, part, rs);
    const DevParams& p = R.p;
    const DevBatch& b = R.b;
    const int h = o.part;
    // arrival count of this step (Philox word, Poisson CDF row)
    const uint32_t blk = o.g >> 2;
    if (blk != o.ablk) {
        o.aw = arrival_words(o.uid, o.g, o.k0, o.k1);
        o.ablk = blk;
    }
    const float* F = b.cdf + ((size_t)o.cls_row * (size_t)p.ep_len + (size_t)o.t) * kCdfLen;
    const float4 f0 = __ldg(reinterpret_cast<const float4*>(F));
    const float4 f1 = __ldg(reinterpret_cast<const float4*>(F + 4));
    const uint32_t lv0 = sx.act[row * (kPolicyMaxPorts / 4) + 2 * h];
    const uint32_t lv1 = sx.act[row * (kPolicyMaxPorts / 4) + 2 * h + 1];

    // (i) per-charger clip; sums of the groups that close in this part
    float P[8];
    float gacc = 0.f, raw = 0.f, over = 0.f, lead = 0.f;
    int nfree = 0, first_gs = -1, first_tail = -1;
    bool head_seen = h == 0, any_tail = false;   // part 0 starts at the station's first group head
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        uint32_t vs[4], ve[4], vc[4], vr[4], vp[4];
        const int c4 = 8 * h + 4 * hh;
        tmem_ld4(taddr_of(tl, kColSoc + c4), vs);
        tmem_ld4(taddr_of(tl, kColErem + c4), ve);
        tmem_ld4(taddr_of(tl, kColCap + c4), vc);
        tmem_ld4(taddr_of(tl, kColRbar + c4), vr);
        tmem_ld4(taddr_of(tl, kColPack + c4), vp);
        tmem_wait_ld();
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
            const int i = 4 * hh + ii;
            const int trem = (int)(vp[ii] & 0xFFu);
            const uint32_t meta = vp[ii] >> 8;
            const int lvl = (int)(((hh == 0 ? lv0 : lv1) >> (8 * ii)) & 0xFFu);
            const bool dc = meta & kMetaDC;
            P[i] = trem > 0 ? clip_power((float)lvl * (dc ? p.lvl1 : p.lvl0), dc, __uint_as_float(vs[ii]),
                                         __uint_as_float(ve[ii]), __uint_as_float(vc[ii]), __uint_as_float(vr[ii]), p)
                            : 0.f;
            raw += P[i];
            if (meta & kMetaHead) head_seen = true;
            gacc += P[i];
            nfree += ((meta & kMetaValid) && trem <= 1) ? 1 : 0;    // free once this step's departures left
            if (meta & kMetaTail) {
                const int gs = (int)((meta >> kMetaGroupShift) & 31u);
                if (!head_seen) {                                    // closes a group begun in an earlier part
                    first_gs = gs;
                    first_tail = i;
                    lead = gacc;
                } else {
                    const float gc = __ldg(b.gcap + o.pb + 8 * h + i);
                    sx.gscale[gs * kM + row] = gacc > gc ? __fdividef(gc, gacc) : 1.0f;
                    if (p.a_con != 0.f) over = fmaxf(over, (gacc - gc) * __ldg(b.ginv_eta + o.pb + 8 * h + i));
                }
                any_tail = true;
                head_seen = false;                                   // until the next group's head
                gacc = 0.f;
            }
        }
    }
    sx.x.lead[h][row] = lead;
    sx.x.trail[h][row] = gacc;
    sx.x.first_gs[h][row] = first_gs;
    sx.x.has_tail[h][row] = any_tail ? 1 : 0;
    sx.x.raw[h][row] = raw;
    sx.x.nfree[h][row] = nfree;
    named_sync(kBarQuad + (row >> 5), kParts * 32);                  // exchange A

    // a group that closes here but began in an earlier part: its sum is this
    // part's lead plus the open sums of the parts back to the one it began in
    if (first_gs >= 0) {
        float S = lead;
        for (int j = h - 1; j >= 0; --j) {
            S += sx.x.trail[j][row];
            if (sx.x.has_tail[j][row]) break;
        }
        const float gc = __ldg(b.gcap + o.pb + 8 * h + first_tail);
        sx.gscale[first_gs * kM + row] = S > gc ? __fdividef(gc, S) : 1.0f;
        if (p.a_con != 0.f) over = fmaxf(over, (S - gc) * __ldg(b.ginv_eta + o.pb + 8 * h + first_tail));
    }
    sx.x.over[h][row] = over;
    int nfree_all = 0, before = 0;
#pragma unroll
    for (int j = 0; j < kParts; ++j) {
        const int nf = sx.x.nfree[j][row];
        nfree_all += nf;
        before += j < h ? nf : 0;
    }
    float raw_all = 0.f;
#pragma unroll
    for (int j = 0; j < kParts; ++j) raw_all += sx.x.raw[j][row];
    named_sync(kBarQuad + (row >> 5), kParts * 32);                  // exchange B: every group's scale

    // architecture constraint: charger power scaled by its group
    float sp = 0.f;
    {
        uint32_t vp[8];
        tmem_ld8(taddr_of(tl, kColPack + 8 * h), vp);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t meta = vp[i] >> 8;
            if (meta & kMetaValid) P[i] *= sx.gscale[((meta >> kMetaGroupShift) & 31u) * kM + row];
            sp += P[i];
        }
    }
    sx.x.sp[h][row] = sp;
    named_sync(kBarQuad + (row >> 5), kParts * 32);                  // exchange C
    float sp_all = 0.f;
#pragma unroll
    for (int j = 0; j < kParts; ++j) sp_all += sx.x.sp[j][row];
    const float s_root = sp_all > o.grid_cap ? __fdividef(o.grid_cap, sp_all) : 1.0f;
    float c_con = 0.f;
    if (p.a_con != 0.f) {
        float over_all = 0.f;
#pragma unroll
        for (int j = 0; j < kParts; ++j) over_all = fmaxf(over_all, sx.x.over[j][row]);
        c_con = fmaxf(fmaxf(over_all, (raw_all - o.grid_cap) * o.grid_inv_eta), 0.f);
    }

    // Poisson count: the smallest k with u < F_k (F nondecreasing, F_127 = inf)
    const uint32_t word = word_of(o.aw, o.g & 3u);
    const float u = __fmul_rn(__uint2float_rn(word >> 8), 0x1p-24f);
    int M = (u >= f0.x) + (u >= f0.y) + (u >= f0.z) + (u >= f0.w) + (u >= f1.x) + (u >= f1.y) + (u >= f1.z) +
            (u >= f1.w);
    if (M == 8)
        while (u >= __ldg(F + M)) ++M;
    // first come first served: earlier parts' free chargers take the first cars
    const int adm_all = min(M, nfree_all);
    const int quota = max(0, min(adm_all - before, nfree));
    const uint32_t car0 = o.ncar + (uint32_t)min(before, adm_all);
    const uint4 cw0 = quota > 0 ? car_words(o.uid, car0, o.k0, o.k1) : make_uint4(0, 0, 0, 0);

    // (ii) charge, (iii) departures, (iv) arrivals, and the episode end
    const bool fin = o.t + 1 >= p.ep_len;
    // the next observation's FP32 rows go out from here (the BF16 operand is
    // written after the step's last barrier, when the scratch is free)
    const bool next_rows = o.live && it + 1 < R.T && obs_sectors(R);
    const bool park = it + 1 < R.T && obs_parked(R);   // uniform across the CTA
    float se = 0.f, c_sat = 0.f;
    int adm = 0, occ = 0;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        uint32_t vs[4], ve[4], vc[4], vr[4], vp[4], vw[4];
        const int c4 = 8 * h + 4 * hh;
        tmem_ld4(taddr_of(tl, kColSoc + c4), vs);
        tmem_ld4(taddr_of(tl, kColErem + c4), ve);
        tmem_ld4(taddr_of(tl, kColCap + c4), vc);
        tmem_ld4(taddr_of(tl, kColRbar + c4), vr);
        tmem_ld4(taddr_of(tl, kColPack + c4), vp);
        tmem_wait_ld();
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
            const int i = 4 * hh + ii;
            int trem = (int)(vp[ii] & 0xFFu);
            const uint32_t meta = vp[ii] >> 8;
            const bool dc = meta & kMetaDC;
            float soc = __uint_as_float(vs[ii]), erem = __uint_as_float(ve[ii]);
            float cap = __uint_as_float(vc[ii]), rbar = __uint_as_float(vr[ii]);
            const float Pq = P[i] * s_root;
            se += P[i] * (dc ? p.inv_eta1 : p.inv_eta0);
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
                const uint4 w = adm == 0 ? cw0 : car_words_late(o.uid, car0 + (uint32_t)adm, o.k0, o.k1);
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
            vs[ii] = __float_as_uint(soc);
            ve[ii] = __float_as_uint(erem);
            vc[ii] = __float_as_uint(cap);
            vr[ii] = __float_as_uint(rbar);
            vp[ii] = (uint32_t)trem | (meta << 8);
            vw[ii] = __float_as_uint(pw);
        }
        tmem_st4(taddr_of(tl, kColSoc + c4), vs);
        tmem_st4(taddr_of(tl, kColErem + c4), ve);
        tmem_st4(taddr_of(tl, kColCap + c4), vc);
        tmem_st4(taddr_of(tl, kColRbar + c4), vr);
        tmem_st4(taddr_of(tl, kColPack + c4), vp);
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) rs.pw[(c4 + ii) * kM + row] = __uint_as_float(vw[ii]);
        if (park && c4 < R.pol.n_ports) {  // BF16 pairs of chargers c4 .. c4 + 3
            uint32_t u[12];
#pragma unroll
            for (int x = 0; x < 12; ++x) {
                const int ia = (2 * x) / 6, fa = (2 * x) % 6, ib = (2 * x + 1) / 6, fb = (2 * x + 1) % 6;
                const float a0 = obs_port_feature(fa, (int)(vp[ia] & 0xFFu), __uint_as_float(vs[ia]), __uint_as_float(ve[ia]),
                                                  __uint_as_float(vr[ia]), __uint_as_float(vw[ia]), (vp[ia] >> 8) & kMetaDC, p);
                const float a1 = obs_port_feature(fb, (int)(vp[ib] & 0xFFu), __uint_as_float(vs[ib]), __uint_as_float(ve[ib]),
                                                  __uint_as_float(vr[ib]), __uint_as_float(vw[ib]), (vp[ib] >> 8) & kMetaDC, p);
                u[x] = o.live ? pack_bf16x2(a0, a1) : 0u;
            }
            const uint32_t col = kColObs + 32 * h + (h == 0 ? 4 : 0) + 12 * hh;
            tmem_st8(taddr_of(tl, col), *reinterpret_cast<const uint32_t(*)[8]>(u));
            tmem_st4(taddr_of(tl, col + 8), *reinterpret_cast<const uint32_t(*)[4]>(u + 8));
        }
        if (next_rows && c4 < R.pol.n_ports) {   // chargers c4 .. c4 + 3: one aligned run of 24 floats
            float* dst = R.obs_out + ((long long)(it + 1) * R.pol.E + o.e) * R.pol.obs_dim + 8 + 6 * c4;
#pragma unroll
            for (int j = 0; j < 24; j += 8) {
                float f[8];
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const int ii = (j + x) / 6, fx = (j + x) % 6;   // charger, feature (compile-time)
                    f[x] = obs_port_feature(fx, (int)(vp[ii] & 0xFFu), __uint_as_float(vs[ii]), __uint_as_float(ve[ii]),
                                            __uint_as_float(vr[ii]), __uint_as_float(vw[ii]), (vp[ii] >> 8) & kMetaDC, p);
                }
                st_global_v8(dst + j, f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7]);
            }
        }
    }
    tmem_wait_st();
    sx.x.se[h][row] = se;
    sx.x.csat[h][row] = c_sat;
    sx.x.occ[h][row] = occ;
    named_sync(kBarQuad + (row >> 5), kParts * 32);                  // exchange D
    float se_all = 0.f, csat_all = 0.f;
    int occ_all = 0;
#pragma unroll
    for (int j = 0; j < kParts; ++j) {
        se_all += sx.x.se[j][row];
        csat_all += sx.x.csat[j][row];
        occ_all += sx.x.occ[j][row];
    }
    o.occ = occ_all;

    // reward, Appendix A.3
    const float e_net = sp_all * s_root * p.dt;
    const float e_grid = se_all * s_root * p.dt;
    o.ncar += (uint32_t)adm_all;
    const float profit = p.p_sell * e_net - o.price * e_grid - p.c_fixed;
    const float r = profit - p.a_sat * csat_all - p.a_decl * (float)(M - adm_all) - p.a_con * c_con;
    o.ret += r;
    o.t += 1;
    if (h == 0) {
        rs.st.arr[row] += (uint32_t)adm_all;
        rs.st.rej[row] += (uint32_t)(M - adm_all);
        rs.st.miss[row] += csat_all;
        rs.st.chg[row] += e_net;
        if (fin) {
            rs.st.last_ret[row] = o.ret;
            rs.st.ended[row] = 1u;
            rs.st.eps[row] += 1u;
        }
    }
    if (fin) {
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
    if (h == 0 && (next_rows || park)) {   // the next observation's station features
        float st8[8];
        obs_env_at(st8, o.t, o.day, o.occ, R.pol.n_ports, 0.f, 0.f, o.price, p);   // charge-only mode
        if (next_rows)
            st_global_v8(R.obs_out + ((long long)(it + 1) * R.pol.E + o.e) * R.pol.obs_dim, st8[0], st8[1], st8[2],
                         st8[3], st8[4], st8[5], st8[6], st8[7]);
        if (park) {
            uint32_t u[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) u[x] = o.live ? pack_bf16x2(st8[2 * x], st8[2 * x + 1]) : 0u;
            tmem_st4(taddr_of(tl, kColObs), u);
            tmem_wait_st();
        }
    }
    if (h == 0) owner_put(o, row, rs);
}

// Observation after the step: this part's chunk (part 0 also the 8 station
// features), every lane on its own row: BF16 into the layer-1 operand, and
// the FP32 row's chunk straight to HBM as the lane's own contiguous run
// (32-byte sectors when the row length keeps them aligned).
__device__ __forceinline__ void owner_observe(const RolloutArgs& R, long long e, int part, int it, int q, int lane,
                                              uint32_t tl, uint32_t abase, const RollSmem& rs, bool fp32, bool parked)
{
    const DevParams& p = R.p;
    const int D = R.pol.obs_dim, N = R.pol.n_ports;
    const int row = 32 * q + lane;
    const bool live = e < R.pol.E;
    const int n_chunks = (N + 7) >> 3;
    const int k = part;
    if (k >= n_chunks) return;                              // uniform across the warp
    if (parked) {
        // the environment step left this part's BF16 pairs in TMEM: copy
        // them into the operand, zero units past the features (K padding)
        const int f0 = k == 0 ? 0 : 8 + 48 * k;
        const int n_f = min(8 + 48 * (k + 1), D) - f0;
        const int n_fp = k == n_chunks - 1 ? (((D + 15) & ~15) - f0) : n_f;
        uint32_t u[32];
        u[28] = u[29] = u[30] = u[31] = 0u;
        tmem_ld16(taddr_of(tl, kColObs + 32 * k), u);
        tmem_ld8(taddr_of(tl, kColObs + 32 * k + 16), *reinterpret_cast<uint32_t(*)[8]>(u + 16));
        tmem_ld4(taddr_of(tl, kColObs + 32 * k + 24), *reinterpret_cast<uint32_t(*)[4]>(u + 24));
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 64; j += 8)
            if (j < n_fp) {
                const bool in = j < n_f;
                st_shared_v4(abase + sw128_offset(row, f0 + j, kChunkBytes), in ? u[j >> 1] : 0u,
                             in ? u[(j >> 1) + 1] : 0u, in ? u[(j >> 1) + 2] : 0u, in ? u[(j >> 1) + 3] : 0u);
            }
        return;
    }
    uint32_t vs[8], ve[8], vr[8], vp[8];
    tmem_ld8(taddr_of(tl, kColSoc + 8 * k), vs);
    tmem_ld8(taddr_of(tl, kColErem + 8 * k), ve);
    tmem_ld8(taddr_of(tl, kColRbar + 8 * k), vr);
    tmem_ld8(taddr_of(tl, kColPack + 8 * k), vp);
    tmem_wait_ld();
    // features [f0, f1): the station's 8 in chunk 0, then 6 per charger
    const int f0 = k == 0 ? 0 : 8 + 48 * k;
    const int f1 = min(8 + 48 * (k + 1), D);
    float st8[8], cf[48];
    if (k == 0 && live) obs_env(st8, rs.rw.t[row], rs.rw.day[row], rs.rw.occ[row], N, 0.f, 0.f, R.b, p);   // charge-only mode
    else
#pragma unroll
        for (int f = 0; f < 8; ++f) st8[f] = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = 8 * k + i;
        if (live && c < N) {
            obs_port<false>(cf + 6 * i, (int)(vp[i] & 0xFFu), 0, __uint_as_float(vs[i]), __uint_as_float(ve[i]),
                            __uint_as_float(vr[i]), rs.pw[c * kM + row], (vp[i] >> 8) & kMetaDC, p);
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
    const int n_f = f1 - f0;
    // BF16 into the operand, one 16-byte swizzle unit (8 features) per store:
    // f0 and the padded width are multiples of 8, so units never straddle a
    // chunk; the K padding up to a multiple of 16 is zero
    const bool last = k == n_chunks - 1;
    const int n_fp = last ? (((D + 15) & ~15) - f0) : n_f;
    auto B = [&](int j) -> float { return j < n_f ? V(j) : 0.f; };
#pragma unroll
    for (int j = 0; j < 64; j += 8)
        if (j < n_fp)
            st_shared_v4(abase + sw128_offset(row, f0 + j, kChunkBytes), pack_bf16x2(B(j), B(j + 1)),
                         pack_bf16x2(B(j + 2), B(j + 3)), pack_bf16x2(B(j + 4), B(j + 5)),
                         pack_bf16x2(B(j + 6), B(j + 7)));
    if (fp32 && R.obs_out && live) {
        // the FP32 row's run of this part: full 32-byte sectors when the
        // row length keeps them aligned, else 8-byte pairs / single floats
        float* dst = R.obs_out + ((long long)it * R.pol.E + e) * D + f0;
        if (obs_sectors(R)) {
#pragma unroll
            for (int j = 0; j < 56; j += 8)
                if (j < n_f) st_global_v8(dst + j, V(j), V(j + 1), V(j + 2), V(j + 3), V(j + 4), V(j + 5), V(j + 6),
                                          V(j + 7));
        } else if ((D & 1) == 0) {
#pragma unroll
            for (int j = 0; j < 56; j += 2)
                if (j < n_f) *reinterpret_cast<float2*>(dst + j) = make_float2(V(j), V(j + 1));
        } else {
#pragma unroll
            for (int j = 0; j < 56; ++j)
                if (j < n_f) dst[j] = V(j);
        }
    }
}

// State back to HBM: each part its chargers, part 0 the station fields.
__device__ __forceinline__ void owner_store(const RolloutArgs& R, long long e, int part, uint32_t tl, int row,
                                            const RollSmem& rs)
{
    Owner o;
    owner_get(o, R, e, row, part, rs);
    const DevBatch& b = R.b;
    const int k = o.part;
    uint32_t vs[8], ve[8], vc[8], vr[8], vp[8];
    tmem_ld8(taddr_of(tl, kColSoc + 8 * k), vs);
    tmem_ld8(taddr_of(tl, kColErem + 8 * k), ve);
    tmem_ld8(taddr_of(tl, kColCap + 8 * k), vc);
    tmem_ld8(taddr_of(tl, kColRbar + 8 * k), vr);
    tmem_ld8(taddr_of(tl, kColPack + 8 * k), vp);
    tmem_wait_ld();
    if (!o.live) return;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = 8 * k + i;
        if (c < R.C) {
            const long long x = o.pb + c;
            b.soc[x] = __uint_as_float(vs[i]);
            b.erem[x] = __uint_as_float(ve[i]);
            b.cap[x] = __uint_as_float(vc[i]);
            b.rbar[x] = __uint_as_float(vr[i]);
            b.pw[x] = rs.pw[c * kM + row];
            b.trem[x] = (uint8_t)(vp[i] & 0xFFu);
        }
    }
    if (k != 0) return;
    const int s = o.slot;
    b.tod[s] = o.t;
    b.day[s] = o.day;
    b.gstep[s] = o.g;
    b.ncar[s] = o.ncar;
    b.ep_ret[s] = o.ret;
    if (rs.st.ended[row]) b.last_ret[s] = rs.st.last_ret[row];
    b.n_episodes[s] += rs.st.eps[row];
    b.st_arrived[s] += rs.st.arr[row];
    b.st_rejected[s] += rs.st.rej[row];
    b.st_missing[s] += rs.st.miss[row];
    b.st_charged[s] += rs.st.chg[row];
}

template <int LT>
__global__ void __launch_bounds__(kRollThreads, 1) k_rollout(const __grid_constant__ WMaps wm, const RolloutArgs R)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* A = aligned_smem(smem_raw);
    unsigned char* ring = A + kActBytes;
    RollSmem& rs = *reinterpret_cast<RollSmem*>(ring + kRollStages * kStageBytes);
    StepScratch& sx = *reinterpret_cast<StepScratch*>(A);
    __shared__ Sync S;
    __shared__ __align__(16) float bias_s[2 * kPolicyHidden + kPolicyMaxPorts * kPolicyGroup];
    const PolicyArgs& a = R.pol;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < 2 * kPolicyHidden + a.n_out_pad; j += blockDim.x) bias_s[j] = a.bias[j];
    if (threadIdx.x == 0) init_sync(S, kRollStages, kRollWorkers);
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
        if (lane == 0) issue<kRollStages, false>(a, A, ring, S, tmem, R.T);
        __syncwarp();
    } else {
        const int ew = warp - 2, q = warp & 3, part = ew >> 2;
        const int row = 32 * q + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
        const uint32_t abase = smem_addr(A);
        const long long env = (long long)tile * kM + row;
        const bool live = env < a.E;
        {
            Owner o;
            owner_load(o, R, tile, row, part, tl, rs, sx);
        }
        owner_observe(R, env, part, 0, q, lane, tl, abase, rs, true, false);
        for (int it = 0; it < R.T; ++it) {
            fence_before();
            named_sync(kBarWorkers, kRollWorkers);   // every observation operand written
            fence_after();
            worker_arrive(&S.xrdy);
            for (int L = 0; L < 2; ++L) {
                wait_sync(&S.acc, (3 * it + L) & 1, S, a.err);
                fence_after();
                hidden_epilogue<2>(tl + (uint32_t)(64 * part), abase, row, 64 * part, bias_s + kPolicyHidden * L);
                worker_arrive(&S.hrdy);
            }
            wait_sync(&S.acc, (3 * it + 2) & 1, S, a.err);
            fence_after();
            uint32_t packed[2];
            sample_part<LT>(a, tl, part, env, live, rs.rw.g[row], rs.rw.k0[row], rs.rw.k1[row],
                            (a.logits && live) ? a.logits + ((long long)it * a.E + env) * a.n_ports * a.n_levels
                                               : nullptr,
                            packed, bias_s + 2 * kPolicyHidden);
            sx.act[row * (kPolicyMaxPorts / 4) + 2 * part] = packed[0];
            sx.act[row * (kPolicyMaxPorts / 4) + 2 * part + 1] = packed[1];
            if (live) store_levels_part(a.actions + ((long long)it * a.E + env) * a.n_ports, part, a.n_ports, packed);
            fence_before();
            named_sync(kBarQuad + q, kParts * 32);              // the rows' sampled levels
            fence_after();
            owner_step(R, env, part, it, row, tl, rs, sx);
            named_sync(kBarWorkers, kRollWorkers);               // the step's scratch is read: the operand may be written
            if (it + 1 < R.T) owner_observe(R, env, part, it + 1, q, lane, tl, abase, rs, !obs_sectors(R), obs_parked(R));
        }
        owner_store(R, env, part, tl, row, rs);
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
        k_rollout<11><<<n_tiles, kRollThreads, kRolloutSmem, st>>>(wm, r);
    else
        k_rollout<0><<<n_tiles, kRollThreads, kRolloutSmem, st>>>(wm, r);
    return cudaGetLastError();
}

}  // namespace chx
