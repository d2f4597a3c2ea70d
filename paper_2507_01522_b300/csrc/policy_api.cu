// policy_api.cu -- C entry points of the on-device policy and of the rollout
// that alternates it with the environment step: fused (one kernel) or split
// (two launches per step, captured once into a CUDA graph).
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/chargax_b300.h"
#include "chx_handle.h"
#include "chx_kernels.h"

using chx::fail;

#define CUDA_TRY(expr)                                          \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return chx::cuda_fail(_e, #expr); \
    } while (0)

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point, so the
// library does not link libcuda directly
EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

void free_policy_graph(chx::PolicyState& P)
{
    if (P.graph_exec) cudaGraphExecDestroy(P.graph_exec);
    if (P.graph) cudaGraphDestroy(P.graph);
    P.graph_exec = nullptr;
    P.graph = nullptr;
    P.key = chx::PolicyGraphKey{};
}

chx::PolicyArgs policy_args(const chx_handle* h, const float* obs, int8_t* actions, float* logits)
{
    const chx::PolicyState& P = h->policy;
    chx::PolicyArgs a{};
    a.obs = obs;
    a.E = h->E;
    a.obs_dim = P.obs_dim;
    a.n_ports = P.n_ports;
    a.n_levels = P.n_levels;
    a.ch1 = P.ch1;
    a.ks1_last = P.ks1_last;
    a.parts3 = P.parts3;
    a.n3_last = P.n3_last;
    a.n_out_pad = P.n_out_pad;
    a.bias = P.d_bias;
    a.user_to_slot = h->d_user_to_slot;
    a.gstep = h->b.gstep;
    a.key0 = h->b.key0;
    a.key1 = h->b.key1;
    a.logits = logits;
    a.actions = actions;
    a.err = h->b.err;
    return a;
}

int enqueue_policy(chx_handle* h, const float* obs, int8_t* actions, float* logits, cudaStream_t st)
{
    CUDA_TRY(chx::launch_policy(h->policy.maps, policy_args(h, obs, actions, logits), h->sm_count, st));
    return CHX_OK;
}

int build_policy_graph(chx_handle* h, const chx::PolicyGraphKey& k)
{
    chx::PolicyState& P = h->policy;
    free_policy_graph(P);
    const long long E = h->E, D = P.obs_dim, NP = (long long)h->E * P.n_ports, NL = NP * P.n_levels;
    cudaStream_t cs = h->cap_stream;
    CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = CHX_OK;
    chx::launch_observe(h->b, h->dp, k.obs, cs);
    if (cudaGetLastError() != cudaSuccess) rc = fail(CHX_ECUDA, "observe launch failed");
    if (!rc) rc = enqueue_policy(h, k.obs, k.actions, k.logits, cs);
    for (int t = 0; t < k.n_steps && !rc; ++t) {
        const bool more = t + 1 < k.n_steps;
        float* next_obs = more ? k.obs + (t + 1) * E * D : nullptr;
        rc = chx::enqueue_fused(h, 1, k.actions + t * NP, 1, k.reward ? k.reward + t * E : nullptr,
                                k.done ? k.done + t * E : nullptr, 1, next_obs, h->warps_per_block, cs);
        if (!rc && more)
            rc = enqueue_policy(h, next_obs, k.actions + (t + 1) * NP, k.logits ? k.logits + (t + 1) * NL : nullptr,
                                cs);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return chx::cuda_fail(e, "cudaStreamEndCapture");
    P.graph = g;
    const cudaError_t ei = cudaGraphInstantiate(&P.graph_exec, g, 0);
    if (ei != cudaSuccess) {
        free_policy_graph(P);
        return chx::cuda_fail(ei, "cudaGraphInstantiate");
    }
    P.key = k;
    return CHX_OK;
}

}  // namespace

namespace chx {

void free_policy(chx_handle* h)
{
    PolicyState& P = h->policy;
    free_policy_graph(P);
    if (P.d_w) cudaFree(P.d_w);
    if (P.d_bias) cudaFree(P.d_bias);
    P.d_w = nullptr;
    P.d_bias = nullptr;
    P.loaded = false;
}

}  // namespace chx

extern "C" int chx_policy_load(chx_handle* h, int32_t hidden, const uint16_t* h_w1, const float* h_b1,
                               const uint16_t* h_w2, const float* h_b2, const uint16_t* h_w3, const float* h_b3)
{
    if (!h || !h_w1 || !h_b1 || !h_w2 || !h_b2 || !h_w3 || !h_b3) return fail(CHX_EINVAL, "null argument");
    if (hidden != chx::kPolicyHidden) return fail(CHX_EINVAL, "the policy's hidden width must be 256");
    if (h->dp.v2g) return fail(CHX_EINVAL, "the on-device policy runs the charge-only mode (v2g = 0)");
    if (h->dp.delta) return fail(CHX_EINVAL, "the on-device policy samples absolute levels (action_delta = 0)");
    if (h->dp.cs_share) return fail(CHX_EINVAL, "the on-device policy runs time-sensitive users only (cs_share_256 = 0)");
    if (h->dp.tree_levels) return fail(CHX_EINVAL, "the on-device policy takes two-level trees (no upper nodes)");
    const long long n = h->user_port_off[1] - h->user_port_off[0];
    for (int e = 1; e < h->E; ++e)
        if (h->user_port_off[e + 1] - h->user_port_off[e] != n)
            return fail(CHX_EINVAL, "the policy needs every station of the batch to have the same charger count");
    if (n < 1 || n > chx::kPolicyMaxPorts) return fail(CHX_EINVAL, "the policy supports 1..32 chargers per station");
    const int L = h->params.n_levels;
    if (L < 2 || L > chx::kPolicyGroup) return fail(CHX_EINVAL, "the policy supports 2..12 action levels");
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return fail(CHX_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");

    const int N = (int)n, D = 8 + 6 * N, H = chx::kPolicyHidden;
    const int n_out_pad = (L * N + 15) & ~15;
    const int rows = 2 * H + n_out_pad;
    std::vector<uint16_t> W((size_t)rows * H, 0);
    std::vector<float> bias((size_t)2 * H + n_out_pad, 0.f);
    for (int r = 0; r < H; ++r) {
        std::memcpy(&W[(size_t)r * H], h_w1 + (size_t)r * D, (size_t)D * sizeof(uint16_t));
        std::memcpy(&W[(size_t)(H + r) * H], h_w2 + (size_t)r * H, (size_t)H * sizeof(uint16_t));
        bias[r] = h_b1[r];
        bias[H + r] = h_b2[r];
    }
    for (int j = 0; j < N * L; ++j) {
        std::memcpy(&W[(size_t)(2 * H + j) * H], h_w3 + (size_t)j * H, (size_t)H * sizeof(uint16_t));
        bias[2 * H + j] = h_b3[j];
    }

    chx::PolicyState& P = h->policy;
    CUDA_TRY(cudaDeviceSynchronize());       // no rollout may be reading the old weights
    if (!P.loaded || P.rows != rows) {
        chx::free_policy(h);
        CUDA_TRY(cudaMalloc(&P.d_w, W.size() * sizeof(uint16_t)));
        CUDA_TRY(cudaMalloc(&P.d_bias, bias.size() * sizeof(float)));
        const cuuint64_t dims[2] = {(cuuint64_t)H, (cuuint64_t)rows};
        const cuuint64_t strides[1] = {(cuuint64_t)H * sizeof(uint16_t)};
        const cuuint32_t estr[2] = {1, 1};
        const int sr = chx::policy_stage_rows();
        const int parts3 = (n_out_pad + sr - 1) / sr, n3_last = n_out_pad - sr * (parts3 - 1);
        struct { CUtensorMap* m; int box_rows; } want[2] = {{&P.maps.main, sr}, {&P.maps.tail, n3_last}};
        for (auto& w : want) {
            const cuuint32_t box[2] = {64, (cuuint32_t)w.box_rows};
            const CUresult r = enc(w.m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, P.d_w, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                chx::free_policy(h);
                return fail(CHX_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
            }
        }
        CUDA_TRY(chx::policy_prepare());
    }
    CUDA_TRY(cudaMemcpy(P.d_w, W.data(), W.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(P.d_bias, bias.data(), bias.size() * sizeof(float), cudaMemcpyHostToDevice));
    P.obs_dim = D;
    P.n_ports = N;
    P.n_levels = L;
    P.n_out_pad = n_out_pad;
    P.rows = rows;
    P.ch1 = (D + 63) / 64;
    P.ks1_last = (D - 64 * (P.ch1 - 1) + 15) / 16;
    P.parts3 = (n_out_pad + chx::policy_stage_rows() - 1) / chx::policy_stage_rows();
    P.n3_last = n_out_pad - chx::policy_stage_rows() * (P.parts3 - 1);
    P.loaded = true;
    return CHX_OK;
}

// the policy kernels move observations, levels and logits in 8- to 32-byte
// vectors: their buffers must start on a 16-byte boundary (NULL passes)
static bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

extern "C" int chx_policy_act(chx_handle* h, const float* d_obs, int8_t* d_actions, float* d_logits, void* stream)
{
    if (!h || !d_obs || !d_actions) return fail(CHX_EINVAL, "null argument");
    if (!h->policy.loaded) return fail(CHX_EINVAL, "no policy loaded");
    if (misaligned(d_obs) || misaligned(d_actions) || misaligned(d_logits))
        return fail(CHX_EINVAL, "observation, level and logit buffers must be 16-byte aligned");
    return enqueue_policy(h, d_obs, d_actions, d_logits, (cudaStream_t)stream);
}

extern "C" int chx_selftest_wait(chx_handle* h, int32_t* h_result)
{
    if (!h || !h_result) return fail(CHX_EINVAL, "null argument");
    int* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, 3 * sizeof(int)));
    int out[3] = {0, 0, 0};
    cudaError_t e = chx::wait_selftest(h->b.err, d, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof out, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return chx::cuda_fail(e, "wait self-test");
    h_result[0] = out[0] && out[1];
    h_result[1] = out[2];
    return CHX_OK;
}

extern "C" int chx_policy_rollout(chx_handle* h, int32_t n_steps, float* d_obs, int8_t* d_actions, float* d_reward,
                                  uint8_t* d_done, float* d_logits, int32_t form, void* stream)
{
    if (!h || !d_actions) return fail(CHX_EINVAL, "null argument");
    if (!h->policy.loaded) return fail(CHX_EINVAL, "no policy loaded");
    if (n_steps < 1) return fail(CHX_EINVAL, "n_steps must be >= 1");
    if (form != CHX_ROLLOUT_FUSED && form != CHX_ROLLOUT_SPLIT) return fail(CHX_EINVAL, "unknown rollout form");
    if (misaligned(d_obs) || misaligned(d_actions) || misaligned(d_logits))
        return fail(CHX_EINVAL, "observation, level and logit buffers must be 16-byte aligned");
    const chx::PolicyState& P = h->policy;
    if (form == CHX_ROLLOUT_FUSED) {
        if (!chx::rollout_fits(P.n_out_pad))
            return fail(CHX_EINVAL, "the fused rollout needs n_ports * n_levels <= 352 (use CHX_ROLLOUT_SPLIT)");
        int cls = 0;
        while ((8 << cls) < P.n_ports) ++cls;
        chx::RolloutArgs r{};
        r.pol = policy_args(h, nullptr, d_actions, d_logits);
        r.b = h->b;
        r.p = h->dp;
        r.T = n_steps;
        r.obs_out = d_obs;
        r.reward = d_reward;
        r.done = d_done;
        r.port_base = h->cls_port_base[cls];
        r.env_base = h->cls_env_base[cls];
        r.C = 8 << cls;
        CUDA_TRY(chx::launch_rollout(P.maps, r, (cudaStream_t)stream));
        return CHX_OK;
    }
    if (!d_obs) return fail(CHX_EINVAL, "the split rollout needs the observation buffer");
    const chx::PolicyGraphKey want{n_steps, d_obs, d_actions, d_reward, d_done, d_logits, h->warps_per_block, true};
    if (!(h->policy.key == want)) {
        const int rc = build_policy_graph(h, want);
        if (rc) return rc;
    }
    CUDA_TRY(cudaGraphLaunch(h->policy.graph_exec, (cudaStream_t)stream));
    return CHX_OK;
}
