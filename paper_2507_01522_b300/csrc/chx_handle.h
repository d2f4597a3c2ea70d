// chx_handle.h -- host-side state of a batch (the opaque chx_handle).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/chargax_b300.h"
#include "chx_device.cuh"
#include "chx_kernels.h"

namespace chx {

using Buffers = std::vector<void*>;

constexpr int kHostChunks = 4;            // launches of a host-call rollout (copies overlap the next)
constexpr int kActChunks = 12;            // launches of a host-actions rollout (copies in and out overlap)
constexpr double kActShrink8 = 0.85;      // size ratio of consecutive launches of an int8 host-actions rollout

struct GraphKey {
    int n_steps = 0;
    float* reward = nullptr;
    uint8_t* done = nullptr;
    float* obs = nullptr;
    int k = 0, w = 0;
    bool valid = false;
    bool operator==(const GraphKey& o) const
    {
        return valid && o.valid && n_steps == o.n_steps && reward == o.reward && done == o.done && obs == o.obs &&
               k == o.k && w == o.w;
    }
};

// the rollout with the on-device policy: graph cache key
struct PolicyGraphKey {
    int n_steps = 0;
    float* obs = nullptr;
    int8_t* actions = nullptr;
    float* reward = nullptr;
    uint8_t* done = nullptr;
    float* logits = nullptr;
    int w = 0;
    bool valid = false;
    bool operator==(const PolicyGraphKey& o) const
    {
        return valid && o.valid && n_steps == o.n_steps && obs == o.obs && actions == o.actions &&
               reward == o.reward && done == o.done && logits == o.logits && w == o.w;
    }
};

// weights and geometry of the loaded policy (see PolicyArgs)
struct PolicyState {
    bool loaded = false;
    int obs_dim = 0, n_ports = 0, n_levels = 0, n_out_pad = 0, rows = 0;
    int ch1 = 0, ks1_last = 0, parts3 = 0, n3_last = 0;
    uint16_t* d_w = nullptr;               // [rows][256] BF16 bits
    float* d_bias = nullptr;               // [512 + n_out_pad]
    WMaps maps{};                          // k_policy and k_rollout (over-aligned; the handle is allocated with new)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    PolicyGraphKey key{};
};

int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

}  // namespace chx

struct chx_handle {
    chx_env_params params{};
    int E = 0;
    long long P = 0;
    int n_days = 0, n_arrival_classes = 0;
    int device = 0, sm_count = 0;
    std::vector<long long> user_port_off;      // [E+1] batch-order charger offsets
    int cls_n_env[chx::kNumClasses] = {};      // padded stations per class
    int cls_n_real[chx::kNumClasses] = {};
    int cls_env_base[chx::kNumClasses] = {};
    long long cls_port_base[chx::kNumClasses] = {};
    int n_slots = 0;
    long long n_port_slots = 0;
    std::vector<int32_t> user_to_slot, slot_user;
    std::vector<long long> slot_port_base;
    chx::DevBatch b{};
    chx::DevParams dp{};
    chx::Buffers bufs;
    int32_t* d_user_to_slot = nullptr;
    int* d_counter = nullptr;
    chx::FusedIO sched{};
    int warps_per_block = 8, steps_per_launch = 32;
    float tuned_ms = 0.f;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t copy_stream = nullptr;    // device-to-host copies of the host-call rollout
    chx::FusedSide side;                   // the 128-charger class's launch beside the others
    cudaEvent_t chunk_done[chx::kHostChunks] = {};
    cudaStream_t in_stream = nullptr;      // host-to-device copies of the host-actions rollout
    cudaEvent_t act_in[chx::kActChunks] = {}, act_done[chx::kActChunks] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    chx::GraphKey graph_key{};
    void* staging[8] = {};
    size_t staging_bytes[8] = {};
    chx::PolicyState policy;
};

namespace chx {
int class_of_ports(int n);
int validate_params(const chx_env_params* p, const chx_exo* x);
int validate_stations(const chx_stations* st, const chx_exo* x, long long max_envs);
DevParams make_params(const chx_env_params& q, int n_days);
// Poisson CDF table of the arrival counts for n_rows_steps means (see poisson_count)
void build_poisson_cdf(const float* lam, size_t n_rows_steps, std::vector<float>& F);
int build_handle(const chx_stations* st, const chx_env_params* prm, const chx_exo* exo, uint64_t seed,
                 int min_pad_envs_per_class, chx_handle** out);
int enqueue_fused(chx_handle* h, int k_steps, const int8_t* actions, long long lda, float* reward, uint8_t* done,
                  long long ld_out, float* obs, int warps, cudaStream_t st, long long ld_step = 1,
                  long long lda_step = 1, int act_bits = 8);
void free_graph(chx_handle* h);
void free_policy(chx_handle* h);
}  // namespace chx
