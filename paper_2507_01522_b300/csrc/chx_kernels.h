// chx_kernels.h -- host-side launchers of the device kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "chx_device.cuh"

namespace chx {

// Arguments of one fused launch.  Tiles are scheduled largest class first:
// sched_cls[i] is the class of schedule entry i, whose tiles are numbered
// sched_tile_base[i] .. sched_tile_base[i+1]-1.
struct FusedIO {
    int k_steps;
    const int8_t* actions;
    long long lda;
    float* reward;
    uint8_t* done;
    long long ld_out;
    float* obs;
    int n_sched;
    int sched_cls[kNumClasses];
    int sched_tile_base[kNumClasses + 1];
    int total_tiles;
    int* counter;                          // work counter, zero at launch
    // gather mode (NULL = every station of the batch): per class, a list of
    // entries (station slot, action offset, output index, observation offset)
    // padded with a padding slot to whole tiles; class c starts at gather_base[c]
    const int4* gather;
    int gather_base[kNumClasses];
};

void launch_step_plain(const DevBatch& b, const DevParams& p, const int8_t* actions, long long lda, float* reward,
                       uint8_t* done, const int* slot_list, int n_list, cudaStream_t st);
// The fused step over io's schedule: the 128-charger class (if any) by one
// persistent kernel, the other classes by a second one, each grid sized to
// the resident blocks on sm_count SMs.  io.counter must point to
// kFusedCounters zeroed ints (one work counter per kernel).
constexpr int kFusedCounters = 2;
void launch_step_fused(const DevBatch& b, const DevParams& p, const FusedIO& io, int threads, int sm_count,
                       cudaStream_t st);
// both fused kernels can be resident with blocks of `threads` threads
bool fused_block_size_ok(int threads);

// reset the stations whose batch ids are listed (NULL = all)
void launch_reset(const DevBatch& b, const DevParams& p, const int32_t* user_to_slot, const int32_t* env_ids, int n,
                  uint64_t seed, cudaStream_t st);
void launch_observe(const DevBatch& b, const DevParams& p, float* obs, cudaStream_t st);
// reset listed slots (station id = slot), one 64-bit seed per entry
void launch_reset_slots(const DevBatch& b, const DevParams& p, const int32_t* slots, const unsigned long long* seeds,
                        int n, cudaStream_t st);

}  // namespace chx
