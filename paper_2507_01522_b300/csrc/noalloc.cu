// noalloc.cu -- a rollout entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc while they run the simulator: code that
// runs under a memory pool or allocator it does not own (a framework that
// forbids foreign device allocations), latency-critical loops that must not
// reach the driver's allocator, or hosts that preallocate all device memory
// up front.  chx_rollout may allocate (it builds and instantiates a CUDA graph
// the first time), and the host-buffer calls allocate staging memory.  This
// file gives those callers chx_rollout_noalloc: the same fused launches, whose
// only scratch -- one work counter per launch -- lives in a file-scope device
// array instead of handle memory, so the call itself allocates nothing.
#include <mutex>
#include <string>

#include "../../include/chargax_b300.h"
#include "chx_handle.h"
#include "chx_kernels.h"

namespace {

constexpr int kMaxDevices = 64;

// The work counters of every launch of a call (kFusedCounters per launch).
// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) int g_noalloc_counters[CHX_NOALLOC_MAX_LAUNCHES * chx::kFusedCounters];

std::mutex g_setup_mutex;
int* g_counters_addr[kMaxDevices] = {};

// Device address of g_noalloc_counters on `device`, looked up once per device
// with that device current.  In host code the array's name is only a host-side
// stand-in, so kernels must be given this address, never the name.  The cached
// address belongs to the device's primary context: it is valid until that
// context is destroyed (cudaDeviceReset), after which this library must not
// be called again in the process.
int counters_on(int device, int** out)
{
    if (device < 0 || device >= kMaxDevices) return chx::fail(CHX_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_counters_addr[device]) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return chx::cuda_fail(e, "cudaGetDevice");
        if (cur != device && (e = cudaSetDevice(device)) != cudaSuccess) return chx::cuda_fail(e, "cudaSetDevice");
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_counters);
        if (cur != device) cudaSetDevice(cur);
        if (e != cudaSuccess) return chx::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_counters)");
        g_counters_addr[device] = static_cast<int*>(p);
    }
    *out = g_counters_addr[device];
    return CHX_OK;
}

}  // namespace

extern "C" int chx_rollout_noalloc(chx_handle* h, int32_t n_steps, float* d_reward, uint8_t* d_done, float* d_obs,
                                   void* stream)
{
    if (!h) return chx::fail(CHX_EINVAL, "null handle");
    if (n_steps < 1) return chx::fail(CHX_EINVAL, "n_steps must be >= 1");
    const int K = h->steps_per_launch;
    const long long launches = ((long long)n_steps + K - 1) / K;
    if (launches > CHX_NOALLOC_MAX_LAUNCHES)
        return chx::fail(CHX_EINVAL, "chx_rollout_noalloc: n_steps = " + std::to_string(n_steps) + " needs " +
                                         std::to_string(launches) + " launches of " + std::to_string(K) +
                                         " steps; the scratch holds at most " +
                                         std::to_string(CHX_NOALLOC_MAX_LAUNCHES));
    int cur = -1;
    cudaError_t ce = cudaGetDevice(&cur);
    if (ce != cudaSuccess) return chx::cuda_fail(ce, "cudaGetDevice");
    if (cur != h->device)
        return chx::fail(CHX_EINVAL, "chx_rollout_noalloc: the current device (" + std::to_string(cur) +
                                         ") is not the handle's device (" + std::to_string(h->device) + ")");
    int* counters = nullptr;
    int rc = counters_on(h->device, &counters);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // the previous call left its counters non-zero: clear the ones this call uses
    cudaError_t e = cudaMemsetAsync(counters, 0, (size_t)launches * chx::kFusedCounters * sizeof(int), st);
    if (e != cudaSuccess) return chx::cuda_fail(e, "cudaMemsetAsync");
    const int threads = h->warps_per_block * 32;
    if (!chx::fused_block_size_ok(threads))
        return chx::fail(CHX_ECUDA, "fused kernel cannot be resident with this block size");
    for (long long i = 0; i < launches; ++i) {
        const int k0 = (int)(i * K);
        const int k = n_steps - k0 < K ? n_steps - k0 : K;
        chx::FusedIO io = h->sched;
        io.k_steps = k;
        io.actions = nullptr;
        io.lda = 0;
        io.lda_step = 0;
        io.reward = d_reward ? d_reward + k0 : nullptr;
        io.done = d_done ? d_done + k0 : nullptr;
        io.ld_out = n_steps;
        io.ld_step = 1;
        io.obs = (i == launches - 1) ? d_obs : nullptr;
        io.counter = counters + i * chx::kFusedCounters;
        // the 128-charger class beside the others, on the handle's own side
        // stream and events (created with the handle, so nothing is allocated)
        chx::launch_step_fused(h->b, h->dp, io, threads, h->sm_count, st, &h->side);
        e = cudaGetLastError();
        if (e != cudaSuccess) return chx::cuda_fail(e, "k_step_fused launch");
    }
    return CHX_OK;
}
