// aux_kernels.cu -- explicit reset and observation kernels.
#include "chx_device.cuh"
#include "chx_kernels.h"

namespace chx {

// Exploring-starts reset (Appendix "Practical Considerations"): one block per
// listed station; threads clear the chargers, thread 0 sets the per-station
// fields and draws the day.
__global__ void k_reset(DevBatch b, DevParams p, const int32_t* __restrict__ user_to_slot,
                        const int32_t* __restrict__ env_ids, int n, int n_users, uint32_t seed_lo, uint32_t seed_hi)
{
    const int j = blockIdx.x;
    if (j >= n) return;
    const int uid = env_ids ? env_ids[j] : j;
    if (uid < 0 || uid >= n_users) {       // caller's list: skip and flag
        if (threadIdx.x == 0) atomicOr(b.err, kErrEnvId);
        return;
    }
    const int s = user_to_slot[uid];
    const int c = class_of_slot(b, s);
    const int C = 8 << c;
    const long long pb = b.cls_port_base[c] + (long long)(s - b.cls_env_base[c]) * C;
    for (int q = threadIdx.x; q < C; q += blockDim.x) {
        const long long i = pb + q;
        b.soc[i] = 0.f; b.erem[i] = 0.f; b.cap[i] = 0.f; b.rbar[i] = 0.f; b.pw[i] = 0.f; b.trem[i] = 0;
        if (p.cs_share) b.due[i] = 0;      // the array exists only with charge-sensitive users
    }
    if (threadIdx.x == 0) {
        b.key0[s] = seed_lo;
        b.key1[s] = seed_hi;
        b.gstep[s] = 0u;
        b.ncar[s] = 0u;
        b.tod[s] = 0;
        b.ep_ret[s] = 0.f;
        if (p.v2g) {  // the battery arrays exist only in V2G mode
            b.bsoc[s] = p.batt_soc0;
            b.bp[s] = 0.f;
        }
        b.day[s] = draw_day((uint32_t)uid, 0u, 1u, seed_lo, seed_hi, p.n_days);
    }
}

void launch_reset(const DevBatch& b, const DevParams& p, const int32_t* user_to_slot, const int32_t* env_ids, int n,
                  int n_users, uint64_t seed, cudaStream_t st)
{
    if (n <= 0) return;
    k_reset<<<n, 128, 0, st>>>(b, p, user_to_slot, env_ids, n, n_users, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Reset of listed station slots with one seed each (the serving pool, where a
// station's id is its slot): same episode start as k_reset.  The count is n,
// or *d_n when d_n is given (the list was built on the device).
__global__ void k_reset_slots(DevBatch b, DevParams p, const int32_t* __restrict__ slots,
                              const unsigned long long* __restrict__ seeds, int n, const int* __restrict__ d_n)
{
    const int cnt = d_n ? *d_n : n;
    for (int j = blockIdx.x; j < cnt; j += gridDim.x)
        reset_one_slot(b, p, slots[j], seeds[j]);
}

void launch_reset_slots(const DevBatch& b, const DevParams& p, const int32_t* slots, const unsigned long long* seeds,
                        int n, cudaStream_t st)
{
    if (n > 0) k_reset_slots<<<n, 128, 0, st>>>(b, p, slots, seeds, n, nullptr);
}

void launch_reset_slots_dev(const DevBatch& b, const DevParams& p, const int32_t* slots,
                            const unsigned long long* seeds, const int* d_n, int grid, cudaStream_t st)
{
    k_reset_slots<<<grid, 128, 0, st>>>(b, p, slots, seeds, 0, d_n);
}

// Observation: one warp per station slot; lanes stride over the chargers.
__global__ void k_observe(DevBatch b, DevParams p, float* __restrict__ obs)
{
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= b.n_slots) return;
    const int uid = b.user_id[s];
    if (uid < 0) return;
    const int c = class_of_slot(b, s);
    const int C = 8 << c;
    const long long pb = b.cls_port_base[c] + (long long)(s - b.cls_env_base[c]) * C;
    const int n = b.n_ports[s];
    float* ob = obs + (long long)p.obs_env * uid + (long long)p.obs_port * b.user_port_off[s];
    int occ = 0;
    for (int q = lane; q < n; q += 32) {
        const long long i = pb + q;
        const int tr = b.trem[i];
        occ += tr > 0;
        obs_port(ob + p.obs_env + p.obs_port * q, tr, p.cs_share ? (int)b.due[i] : 0, b.soc[i], b.erem[i], b.rbar[i],
                 b.pw[i], b.meta[i] & kMetaDC, p);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) occ += __shfl_xor_sync(0xFFFFFFFFu, occ, o);
    if (lane == 0)
        obs_env(ob, b.tod[s], b.day[s], occ, n, p.v2g ? b.bsoc[s] : 0.f, p.v2g ? b.bp[s] : 0.f, b, p);
}

void launch_observe(const DevBatch& b, const DevParams& p, float* obs, cudaStream_t st)
{
    const int warps = 8;
    const int blocks = (b.n_slots + warps - 1) / warps;
    if (blocks > 0) k_observe<<<blocks, warps * 32, 0, st>>>(b, p, obs);
}

}  // namespace chx
