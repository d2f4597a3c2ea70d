// policy.cu -- the on-device policy of a rollout: a 3-layer MLP
// obs (D = 8 + 6N) -> 256 -> 256 -> N x L logits (ReLU between layers; the
// PPO actor of the paper's Table "PPO hyper-parameters" with its random
// initialisation), BF16 operands, FP32 accumulation, on the 5th-generation
// tensor cores, with the categorical sample of every charger's action level
// fused into the last layer's epilogue.
//
// One CTA per 128-env tile (persistent over tiles when there are more tiles
// than SMs).  Roles:
//   warp 0, lane 0   TMA producer: streams the weights, one 128-row x 64-col
//                    BF16 box (16 KB) per stage, through a kStages ring;
//   warp 1           owns the TMEM allocation (512 columns); lane 0 issues
//                    every tcgen05.mma (M = 128, N = 128 per part, K = 16);
//   warps 2..9       load the tile's observations (FP32 -> BF16, swizzled),
//                    run the epilogues (bias, ReLU, BF16 into the next
//                    layer's A operand) and the sampling.
// Epilogue warp w reads TMEM lanes 32 (w % 4) .. +31 (one env per thread);
// warps 2-5 take columns 0-127 of a layer (part 0), warps 6-9 columns
// 128-255 (part 1), so each half starts as soon as its part's MMAs finish,
// and the next layer's MMAs over K = 0..127 start as soon as half 0 is
// written.  Every wait is bounded (kWaitCycles); a timeout sets
// kErrPolicyWait and unwinds without hanging.
#include <cuda.h>

#include "chx_kernels.h"
#include "chx_tc.cuh"

namespace chx {

namespace {

using namespace tc;

constexpr int kM = 128;                    // envs per tile (MMA M, TMEM lanes)
constexpr int kChunkBytes = kM * 128;      // 128 rows x 64 BF16
constexpr int kActBytes = 4 * kChunkBytes; // 128 x 256 BF16 activation tile
constexpr int kStages = 5;
constexpr int kStageBytes = 128 * 128;     // 128 weight rows x 64 BF16
constexpr int kEpiWarps = 8;
constexpr int kThreads = (2 + kEpiWarps) * 32;
constexpr int kSmemBytes = 1024 + 2 * kActBytes + kStages * kStageBytes;
constexpr uint32_t kTmemCols = 512;
constexpr int kGroup = kPolicyGroup;

struct Bars {
    uint64_t full[kStages], empty[kStages];
    uint64_t accb[2];                      // layer 1/2 part p accumulated
    uint64_t acc3;                         // layer 3 accumulated
    uint64_t xrdy;                         // observations of the tile in act0
    uint64_t hrdy[2];                      // half h of the next layer's input written
    uint64_t fin;                          // every MMA of this CTA done
    uint32_t tmem;
};

__device__ __forceinline__ void raise(uint32_t* err) { atomicOr(err, kErrPolicyWait); }

// ---- TMA producer -------------------------------------------------------
__device__ void produce(const CUtensorMap* wmap, const PolicyArgs& a, unsigned char* ring, Bars& B, int n_tiles)
{
    uint32_t s = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x)
        for (int L = 0; L < 3 && ok; ++L) {
            const int parts = L < 2 ? 2 : a.parts3;
            const int chunks = L == 0 ? a.ch1 : 4;
            for (int p = 0; p < parts && ok; ++p)
                for (int k = 0; k < chunks; ++k, ++s) {
                    const uint32_t slot = s % kStages;
                    if (s >= (uint32_t)kStages && !mbar_wait(&B.empty[slot], ((s / kStages) - 1) & 1)) {
                        raise(a.err);
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&B.full[slot], kStageBytes);
                    tma_load_2d(ring + slot * kStageBytes, wmap, k * 64, L * 256 + p * 128, &B.full[slot]);
                }
        }
    // nothing may still be landing in shared memory when the CTA exits
    for (uint32_t j = s > (uint32_t)kStages ? s - kStages : 0; j < s; ++j)
        if (!mbar_wait(&B.full[j % kStages], (j / kStages) & 1)) raise(a.err);
}

// ---- MMA issuer ---------------------------------------------------------
__device__ void issue(const PolicyArgs& a, unsigned char* act0, unsigned char* act1, unsigned char* ring, Bars& B,
                      uint32_t tmem, int n_tiles)
{
    uint32_t s = 0;
    bool ok = true;
    const uint32_t id128 = idesc_bf16_f32(kM, 128);
    int i = 0;
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++i) {
        if (!mbar_wait(&B.xrdy, i & 1)) { ok = false; break; }
        fence_after();
        for (int L = 0; L < 3 && ok; ++L) {
            unsigned char* A = (L == 1) ? act1 : act0;
            const int parts = L < 2 ? 2 : a.parts3;
            const int chunks = L == 0 ? a.ch1 : 4;
            for (int p = 0; p < parts && ok; ++p) {
                const int n = (L == 2 && p == parts - 1) ? a.n3_last : 128;
                const uint32_t id = n == 128 ? id128 : idesc_bf16_f32(kM, n);
                for (int k = 0; k < chunks; ++k, ++s) {
                    // layers 2 and 3 read the previous epilogue's halves
                    if (L > 0 && p == 0 && (k == 0 || k == 2)) {
                        if (!mbar_wait(&B.hrdy[k >> 1], (2 * i + L - 1) & 1)) { ok = false; break; }
                        fence_after();
                    }
                    const uint32_t slot = s % kStages;
                    if (!mbar_wait(&B.full[slot], (s / kStages) & 1)) { ok = false; break; }
                    fence_after();
                    const int nks = (L == 0 && k == chunks - 1) ? a.ks1_last : 4;
                    unsigned char* bst = ring + slot * kStageBytes;
                    for (int j = 0; j < nks; ++j)
                        mma_bf16(tmem + (uint32_t)(p * 128), sdesc_sw128(A + k * kChunkBytes + j * 32),
                                 sdesc_sw128(bst + j * 32), id, (k | j) != 0);
                    mma_commit(&B.empty[slot]);
                }
                if (L < 2) mma_commit(&B.accb[p]);
            }
        }
        if (ok) mma_commit(&B.acc3);
    }
    if (!ok) raise(a.err);
    mma_commit(&B.fin);
    if (!mbar_wait(&B.fin, 0)) raise(a.err);
}

// ---- epilogue of layers 1 and 2: bias, ReLU, BF16, swizzled store -------
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, const float* bias, unsigned char* dst, int row,
                                                int col0)
{
    const uint32_t dbase = smem_addr(dst);
#pragma unroll 1
    for (int blk = 0; blk < 4; ++blk) {
        const int c = col0 + 32 * blk;
        uint32_t v[32];
        tmem_ld32(taddr + (uint32_t)(32 * blk), v);
        tmem_wait_ld();
        uint32_t q[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float x0 = fmaxf(__uint_as_float(v[2 * j]) + bias[c + 2 * j], 0.f);
            const float x1 = fmaxf(__uint_as_float(v[2 * j + 1]) + bias[c + 2 * j + 1], 0.f);
            q[j] = pack_bf16x2(x0, x1);
        }
        const int unit0 = (c & 63) >> 3;
        const uint32_t rbase = dbase + (uint32_t)((c >> 6) * kChunkBytes + row * 128);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            st_shared_v4(rbase + ((uint32_t)((unit0 + u) ^ (row & 7)) << 4), q[4 * u], q[4 * u + 1], q[4 * u + 2],
                         q[4 * u + 3]);
    }
}

// ---- sampling of the action levels of chargers c0..c0+3 of one env ------
// Inverse transform of the softmax: level = #{j < L-1 : e_0 + .. + e_j <= u S}
// with e_j = exp(l_j - max l), S = sum e_j, u from the policy Philox word.
__device__ __forceinline__ uint32_t sample4(const uint32_t (&v)[48], const float* b3, int c0, int n_ports,
                                           int n_levels, uint4 words, float* logits_out)
{
    uint32_t packed = 0;
#pragma unroll
    for (int ci = 0; ci < 4; ++ci) {
        const int c = c0 + ci;
        if (c >= n_ports) break;
        float l[kGroup];
        float m = -INFINITY;
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
            l[j] = __uint_as_float(v[kGroup * ci + j]) + b3[kGroup * c + j];
            if (j < n_levels) m = fmaxf(m, l[j]);
        }
        float e[kGroup], S = 0.f;
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
            e[j] = j < n_levels ? __expf(l[j] - m) : 0.f;
            S += e[j];
        }
        const float T = unit_of(word_of(words, (uint32_t)ci)) * S;
        float cum = 0.f;
        int level = 0;
#pragma unroll
        for (int j = 0; j < kGroup - 1; ++j) {
            cum += e[j];
            level += (j < n_levels - 1 && cum <= T) ? 1 : 0;
        }
        packed |= (uint32_t)level << (8 * ci);
        if (logits_out)
            for (int j = 0; j < n_levels; ++j) logits_out[(long long)ci * n_levels + j] = l[j];
    }
    return packed;
}

__device__ void epilogue(const PolicyArgs& a, unsigned char* act0, unsigned char* act1, Bars& B, const float* bias_s,
                         uint32_t tmem, int n_tiles)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ew = warp - 2;                 // 0..7
    const int q = warp & 3;                  // TMEM lane quadrant
    const int h = ew >> 2;                   // column half
    const int row = 32 * q + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
    const uint32_t a0 = smem_addr(act0);
    const int D = a.obs_dim;
    const int pairs = ((D + 15) & ~15) >> 1; // K padded to the MMA's 16
    int i = 0;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
        // (1) observations -> BF16 A operand of layer 1 (rows ew, ew + 8, ...)
        for (int r = ew; r < kM; r += kEpiWarps) {
            const long long e = (long long)tile * kM + r;
            const float* src = a.obs + e * D;
            for (int pr = lane; pr < pairs; pr += 32) {
                const int k = 2 * pr;
                float2 x = make_float2(0.f, 0.f);
                if (e < a.E && k < D) x = *reinterpret_cast<const float2*>(src + k);
                st_shared_u32(a0 + sw128_offset(r, k, kChunkBytes), pack_bf16x2(x.x, x.y));
            }
        }
        fence_proxy_async();
        fence_before();
        mbar_arrive(&B.xrdy);

        // per-env sampling inputs, fetched early
        const long long env = (long long)tile * kM + row;
        const bool live = env < a.E;
        uint32_t g = 0, k0 = 0, k1 = 0;
        if (live) {
            const int slot = a.user_to_slot[env];
            g = a.gstep[slot];
            k0 = a.key0[slot];
            k1 = a.key1[slot];
        }

        // (2) layers 1 and 2: this half's 128 columns
        bool ok = true;
        for (int L = 0; L < 2; ++L) {
            if (!mbar_wait(&B.accb[h], (2 * i + L) & 1)) { ok = false; break; }
            fence_after();
            hidden_epilogue(tl + (uint32_t)(128 * h), bias_s + 256 * L, L == 0 ? act1 : act0, row, 128 * h);
            fence_proxy_async();
            fence_before();
            mbar_arrive(&B.hrdy[h]);
        }
        if (ok && !mbar_wait(&B.acc3, i & 1)) ok = false;
        if (!ok) {
            raise(a.err);
            return;
        }
        fence_after();

        // (3) layer 3: chargers 16h .. 16h + 15 of this env, four at a time
        const float* b3 = bias_s + 512;
        uint32_t packed[4] = {0, 0, 0, 0};
#pragma unroll 1
        for (int blk = 0; blk < 4; ++blk) {
            const int c0 = 16 * h + 4 * blk;
            if (c0 >= a.n_ports) break;
            uint32_t v[48];
            tmem_ld32(tl + (uint32_t)(kGroup * c0), *reinterpret_cast<uint32_t(*)[32]>(v));
            tmem_ld16(tl + (uint32_t)(kGroup * c0 + 32), v + 32);
            tmem_wait_ld();
            if (!live) continue;
            const uint4 words = philox4x32_10(make_uint4((uint32_t)env, g, (uint32_t)(c0 >> 2), kPurposePolicy), k0, k1);
            float* lo = a.logits ? a.logits + (env * a.n_ports + c0) * a.n_levels : nullptr;
            packed[blk] = sample4(v, b3, c0, a.n_ports, a.n_levels, words, lo);
        }
        fence_before();
        if (live) {
            int8_t* dst = a.actions + env * a.n_ports;
            if (a.n_ports == 32) {
                *reinterpret_cast<uint4*>(dst + 16 * h) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            } else {
                for (int c = 16 * h; c < 16 * h + 16 && c < a.n_ports; ++c)
                    dst[c] = (int8_t)((packed[(c - 16 * h) >> 2] >> (8 * (c & 3))) & 0xFF);
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_policy(const __grid_constant__ CUtensorMap wmap, const PolicyArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    unsigned char* act0 = base;
    unsigned char* act1 = base + kActBytes;
    unsigned char* ring = base + 2 * kActBytes;
    __shared__ Bars B;
    __shared__ float bias_s[512 + kPolicyMaxOut];
    const int warp = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < 512 + a.n_out_pad; j += blockDim.x) bias_s[j] = a.bias[j];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&B.full[s], 1);
            mbar_init(&B.empty[s], 1);
        }
        mbar_init(&B.accb[0], 1);
        mbar_init(&B.accb[1], 1);
        mbar_init(&B.acc3, 1);
        mbar_init(&B.fin, 1);
        mbar_init(&B.xrdy, kEpiWarps * 32);
        mbar_init(&B.hrdy[0], kEpiWarps * 16);
        mbar_init(&B.hrdy[1], kEpiWarps * 16);
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(&B.tmem, kTmemCols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = B.tmem;
    const int n_tiles = (a.E + kM - 1) / kM;
    if (warp == 0) {
        if ((threadIdx.x & 31) == 0) produce(&wmap, a, ring, B, n_tiles);
        __syncwarp();
    } else if (warp == 1) {
        if ((threadIdx.x & 31) == 0) issue(a, act0, act1, ring, B, tmem, n_tiles);
        __syncwarp();
    } else {
        epilogue(a, act0, act1, B, bias_s, tmem, n_tiles);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace

int policy_smem_bytes() { return kSmemBytes; }

cudaError_t policy_prepare()
{
    return cudaFuncSetAttribute(k_policy, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

cudaError_t launch_policy(const CUtensorMap& wmap, const PolicyArgs& a, int sm_count, cudaStream_t st)
{
    const int n_tiles = (a.E + kM - 1) / kM;
    const int grid = n_tiles < sm_count ? n_tiles : sm_count;
    if (grid <= 0) return cudaSuccess;
    k_policy<<<grid, kThreads, kSmemBytes, st>>>(wmap, a);
    return cudaGetLastError();
}

}  // namespace chx
