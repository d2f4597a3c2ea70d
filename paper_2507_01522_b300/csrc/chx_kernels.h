// chx_kernels.h -- host-side launchers of the device kernels.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "chx_device.cuh"

namespace chx {

// Arguments of one fused launch.  Tiles are scheduled largest class first:
// sched_cls[i] is the class of schedule entry i, whose tiles are numbered
// sched_tile_base[i] .. sched_tile_base[i+1]-1.
struct FusedIO {
    int k_steps;
    const int8_t* actions;                 // given level of action slot q at step k: actions[q * lda + k * lda_step]
    long long lda;
    long long lda_step;
    int act_bits;                          // 8: one int8 level per byte; 4: two levels per byte, the index
                                           // above counting nibbles, the even one in the low nibble
    float* reward;
    uint8_t* done;
    long long ld_out;                      // env e, step k at e * ld_out + k * ld_step
    long long ld_step;
    float* obs;
    int n_sched;
    int sched_cls[kNumClasses];
    int sched_tile_base[kNumClasses + 1];
    int total_tiles;
    int* counter;                          // work counter, zero at launch
    // gather mode (NULL = every station of the batch): per class, a list of
    // entries (station slot, action offset, output index, observation offset)
    // padded with a padding slot to whole tiles; class c starts at gather_base[c].
    // An action offset < 0 draws that station's levels with Philox; an
    // observation offset < 0 writes no observation for that station.
    const int4* gather;
    int gather_base[kNumClasses];
    // gather mode with a device-side schedule (NULL = the host schedule
    // above): entries of class c in dcount[c]; tiles run largest class first.
    // dmax_small / dmax_mid / dmax_large bound the tiles of the classes of
    // 8..32, of 64 and of 128 chargers (grid sizes; 0 = no launch for that range)
    const int* dcount;
    int dmax_small, dmax_mid, dmax_large;
};

void launch_step_plain(const DevBatch& b, const DevParams& p, const int8_t* actions, long long lda, float* reward,
                       uint8_t* done, const int* slot_list, int n_list, cudaStream_t st);
// The fused step over io's schedule: the 128-charger class (if any) by one
// persistent kernel, the smaller classes by a second; in the V2G and extended
// forms without upper tree levels the 64-charger class by a third of its own.
// Each grid is sized to the resident blocks on sm_count SMs.  io.counter must
// point to kFusedCounters zeroed ints (one work counter per kernel).
constexpr int kFusedCounters = 3;
// A side stream for the 128-charger class and a 64-charger instance: with
// one, those launches run (in turn) beside the smaller classes' (forked from
// and joined back to st by the two events, which CUDA-graph capture
// supports); without, all the launches run in turn.
struct FusedSide {
    cudaStream_t aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
void launch_step_fused(const DevBatch& b, const DevParams& p, const FusedIO& io, int threads, int sm_count,
                       cudaStream_t st, const FusedSide* side = nullptr);
// both fused kernels can be resident with blocks of `threads` threads
bool fused_block_size_ok(int threads);

// reset the stations whose batch ids are listed (NULL = all)
void launch_reset(const DevBatch& b, const DevParams& p, const int32_t* user_to_slot, const int32_t* env_ids, int n,
                  int n_users, uint64_t seed, cudaStream_t st);
void launch_observe(const DevBatch& b, const DevParams& p, float* obs, cudaStream_t st);
// reset listed slots (station id = slot), one 64-bit seed per entry
void launch_reset_slots(const DevBatch& b, const DevParams& p, const int32_t* slots, const unsigned long long* seeds,
                        int n, cudaStream_t st);
// the same with the entry count *d_n in device memory, `grid` blocks striding over it
void launch_reset_slots_dev(const DevBatch& b, const DevParams& p, const int32_t* slots,
                            const unsigned long long* seeds, const int* d_n, int grid, cudaStream_t st);


// ---- policy (3-layer BF16 MLP on the tensor cores + fused sampling) ------
constexpr int kPolicyHidden = 256;
constexpr int kPolicyMaxPorts = 32;
constexpr int kPolicyGroup = 12;           // most action levels the sampler handles

// Weights: one BF16 matrix [512 + n_out_pad][256], row-major, streamed by
// TMA with 128-byte swizzle.  Rows 0-255 = W1 (columns >= obs_dim zero),
// 256-511 = W2, 512 + c * L + j = level j of charger c (W3; rows up to
// n_out_pad zero).  bias = b1 | b2 | b3 in the same order.  Two maps over
// it, used by k_policy and k_rollout alike: boxes of 64 columns x
// policy_stage_rows() rows, and 64 x n3_last rows for the last part of
// layer 3.
struct WMaps {
    CUtensorMap main, tail;
};
struct PolicyArgs {
    const float* obs;                      // [E][obs_dim] FP32 (k_policy)
    int E, obs_dim, n_ports, n_levels;
    int ch1, ks1_last;                     // layer-1 K chunks of 64, K = 16 steps in the last one
    int parts3, n3_last;                   // layer-3 N parts of policy_stage_rows(), N of the last part
    int n_out_pad;                         // n_ports * n_levels rounded up to 16
    const float* bias;
    const int32_t* user_to_slot;
    const uint32_t *gstep, *key0, *key1;   // per station slot
    float* logits;                         // NULL or [(T)][E][n_ports][n_levels]
    int8_t* actions;                       // [(T)][E][n_ports]
    uint32_t* err;
};

// The fused rollout: T x (MLP pass, sample, environment step) per 128-env
// tile, all stations of one size class (class size C >= n_ports).
struct RolloutArgs {
    PolicyArgs pol;
    DevBatch b;
    DevParams p;
    int T;
    float* obs_out;                        // NULL or [T][E][obs_dim]
    float* reward;                         // NULL or [T][E]
    uint8_t* done;                         // NULL or [T][E]
    long long port_base;                   // charger slot of the class's first station
    int env_base;                          // station slot of the class's first station
    int C;                                 // charger slots per station
};

int policy_smem_bytes();
cudaError_t policy_prepare();              // once per process, before capture
int policy_stage_rows();                   // weight rows (MMA N) of a full layer part
cudaError_t launch_policy(const WMaps& wm, const PolicyArgs& a, int sm_count, cudaStream_t st);
bool rollout_fits(int n_out_pad);          // logits leave TMEM room for the env state
cudaError_t launch_rollout(const WMaps& wm, const RolloutArgs& r, cudaStream_t st);
// one bounded wait on a barrier nothing releases (d_out: 3 ints, device)
cudaError_t wait_selftest(uint32_t* err, int* d_out, cudaStream_t st);

}  // namespace chx
