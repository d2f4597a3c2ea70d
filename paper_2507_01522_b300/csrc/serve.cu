// serve.cu -- the serving loop: a pool of device-resident stations stepped by
// requests from many actors with continuous batching, each tick built on the
// device.
//
// * Pool: station slots bucketed by size class (the layout of chx_device.cuh),
//   allocated once; stations are admitted into free slots while the bytes they
//   occupy stay within an HBM budget, and evicted to free them.  A station's
//   id is its slot, which is also its Philox stream id.
// * Requests: chx_srv_submit validates a request in the caller's thread,
//   takes the next ticket and writes the request into a record of pinned,
//   device-mapped host memory (station list, given levels, output buffers);
//   nothing else is done per station on the host.
// * Ticks: one scheduler thread hands the device a window of tickets [lo, hi)
//   -- the requests not yet known to be finished -- and the device does the
//   rest, on one stream, in order:
//     window   the window's end moves past every request published since the
//              launch (a tick queued behind a running one takes what arrived
//              meanwhile);
//     claim    each open request of the window copies its list into a device
//              arena and writes its rank (arrival order) into every station
//              it lists with atomicMin;
//     select   a request whose rank won every one of its stations is taken
//              (the earliest request for each station runs first, later ones
//              wait for a later tick); its stations become gather entries of
//              their size class, or reset entries;
//     prep     each class's entries are padded to whole warp tiles, and the
//              reset entries start new episodes;
//     step     the fused kernel of step_fused.cu runs one step in gather mode
//              over the device-side entry counts;
//     finish   each taken request's rewards, done flags and observations go
//              straight into its pinned buffers, then its completion flag
//              (after a system-wide fence); the window's claims are cleared.
//   Each of the n_streams tick slots is one CUDA graph, captured at start,
//   whose kernels read the window from the slot's pinned argument record; up
//   to n_streams ticks are queued on the device at once, and requests that
//   arrive while a tick runs join the next one to start.
// * Completion: chx_srv_wait / chx_srv_test read the request's completion
//   flag and copy its results to the caller's buffers in the caller's thread.
// * A station's result depends only on its own state and its position inside
//   its station tile, so a request's results are the same whatever else
//   shares its tick.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "../../include/chargax_b300.h"
#include "chx_handle.h"
#include "chx_kernels.h"

using namespace chx;

#define SRV_TRY(expr)                                           \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return chx::cuda_fail(_e, #expr); \
    } while (0)

namespace {

using Clock = std::chrono::steady_clock;
inline int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

constexpr uint64_t kMaxOutstanding = 1u << 16;   // request records (power of two)

// bytes a station of class c occupies in the pool (state + statics)
inline double slot_bytes(int c) { return (double)(8 << c) * 33.0 + 128.0; }

constexpr int kFree = 0, kFilling = 1, kQueued = 2;

// What the device reads of a request: one per record, in pinned host memory
// mapped into the device's address space.
struct DevReq {
    unsigned long long ticket;
    int kind, n;                           // CHX_SRV_STEP / CHX_SRV_RESET, stations listed
    int n_act;                             // chargers of the listed stations
    int has_act;                           // given levels (else Philox)
    int obs_floats;                        // observation floats to return (0 = none)
    int unused;
    long long cum_envs, cum_act, cum_obs;  // totals of every earlier submission
    const int32_t* ids;                    // [n] station slots
    const int8_t* acts;                    // [n_act] given levels
    float* rew;                            // [n] outputs, written by the device
    uint8_t* done;                         // [n]
    float* obs;                            // [obs_floats]
    unsigned long long seed;               // reset: new Philox key
};

// a block of pinned, device-mapped host memory from PinnedPool
template <class T>
struct PinnedBuf {
    T* h = nullptr;                        // host address
    T* d = nullptr;                        // device address
    size_t cap = 0;                        // elements
    int cls = 0;                           // log2 of the block's bytes
};

struct PinnedPool {
    static constexpr size_t kChunk = 64u << 20;
    std::mutex mu;
    std::vector<void*> chunks;
    char *cur_h = nullptr, *cur_d = nullptr;
    size_t left = 0;
    std::vector<std::pair<void*, void*>> free_list[48];
    int get(size_t bytes, void** host, void** dev, int* cls);
    void put(void* host, void* dev, int cls);
    ~PinnedPool();
};

// A request record (host side).  Records live in a fixed table indexed by
// ticket modulo its size; each keeps its pinned buffers for reuse.
struct Request {
    std::atomic<int> state{kFree};
    std::atomic<uint64_t> ticket{0};
    int32_t kind = 0, n = 0;
    int64_t t_submit = 0;
    float* h_reward = nullptr;
    uint8_t* h_done = nullptr;
    float* h_obs = nullptr;
    int64_t obs_floats = 0;
    int64_t cum_envs = 0, cum_act = 0, cum_obs = 0;
    // pinned, device-mapped buffers
    PinnedBuf<int32_t> ids;
    PinnedBuf<int8_t> acts;
    PinnedBuf<float> rew;
    PinnedBuf<uint8_t> done;
    PinnedBuf<float> obs;
};

// A record's descriptor as the claim kernel read it (host memory is read
// once per record and tick), with its arena offsets in that tick.
struct RecMeta {
    long long off, aoff, ooff;             // arena offsets: stations, given levels, observation floats
    unsigned long long seed;
    float* rew;
    uint8_t* done;
    float* obs;
    int n, kind, has_act, obs_floats;
};

// counters of a tick, in device memory (zeroed by the claim kernel)
enum { kCntClass = 0, kCntAdmitted = 5, kCntReset = 6, kCntBlocked = 7, kCntWork = 8, kCnt = 11 };
static_assert(kCntWork + kFusedCounters <= kCnt, "counter layout");

// what a tick reports to the host (pinned, mapped)
struct TickResult {
    int admitted, stepped, resets, blocked;
};

struct TickArgs {
    unsigned long long lo, hi;             // the window's tickets
    long long base_envs, base_act, base_obs;   // totals of the submissions before ticket lo
    int tick;                              // tick number (>= 1)
    int slot;                              // TickResult slot
};

// device-side state of the server
struct DevSrv {
    const DevReq* req;                     // [kMaxOutstanding] mapped
    unsigned long long* done_flag;         // [kMaxOutstanding] mapped: ticket finished
    unsigned long long* executed;          // [kMaxOutstanding]: ticket taken by a tick
    int* claimed_tick;                     // [kMaxOutstanding]: tick whose claim pass the record joined
    RecMeta* meta;                         // [kMaxOutstanding]: the record as that claim pass read it
    unsigned long long* adm;               // [kMaxOutstanding]: tickets taken by the tick
    uint32_t* claim;                       // [n_slots]: lowest rank claiming a station
    int32_t* ids;                          // [A] station lists of the window
    int8_t* acts;                          // [A_act] given levels of the window
    float* rew;                            // [A] step outputs
    uint8_t* done;                         // [A]
    float* obs;                            // [A_obs]
    int4* gather;                          // [kNumClasses][G] entries, G = A + padding
    int32_t* rslot;                        // [A] reset entries
    unsigned long long* rseed;             // [A]
    int* cnt;                              // [kCnt]
    TickResult* result;                    // [n_streams] mapped
    TickArgs* targs;                       // [n_streams] the ticks' arguments (device copy)
    long long A, A_act, A_obs;
    int G, max_tick_envs;
    int pad_slot[kNumClasses];
    unsigned long long mask;
};

__device__ __forceinline__ long long warp_global()
{
    return ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}
__device__ __forceinline__ long long warps_total() { return ((long long)gridDim.x * blockDim.x) >> 5; }

// A request's ticket as published in its pinned record (the submitter
// stores it last, with release order, after every other field)
__device__ __forceinline__ unsigned long long published_ticket(const DevReq* r)
{
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(&r->ticket) : "memory");
    return v;
}

// window: the tick's arguments from the slot's pinned record into device
// memory, the window's end moved past every request published since the
// host launched the tick (so a tick queued behind a running one takes what
// arrived meanwhile), the tick's counters zeroed.  One warp; records are
// read 32 at a time while all 32 are published, at most kWindowRounds times.
// The scheduler does not learn the extended end: it launches a tick for any
// request it sees newly published, and a tick whose window holds only
// requests an earlier tick already took finds them executed and skips them.
constexpr int kWindowRounds = 8;
__global__ void k_tick_window(DevSrv d, const TickArgs* __restrict__ host_args, int slot)
{
    TickArgs a = host_args[slot];
    const int lane = threadIdx.x & 31;
    if (lane < kCnt) d.cnt[lane] = 0;
    unsigned long long hi = a.hi;
    for (int r = 0; r < kWindowRounds; ++r) {
        const unsigned long long t = hi + (unsigned long long)lane;
        const bool ok = t - a.lo < (unsigned long long)(d.mask + 1) &&
                        published_ticket(d.req + (t & d.mask)) == t;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, ok);
        const int run = bal == 0xFFFFFFFFu ? 32 : __ffs(~bal) - 1;   // published prefix
        hi += (unsigned long long)run;
        if (run < 32) break;
    }
    if (lane == 0) {
        a.hi = hi;
        d.targs[slot] = a;
    }
}

// claim: copy each open request's list (and levels) into the arenas and mark
// its stations with its rank.  A request whose arena span does not fit waits
// for a later tick; spans grow with the ticket, so every later one waits too.
// Host memory is read in two dependent rounds per record (descriptor, then
// its list with up to 8 loads in flight per lane).
__global__ void k_tick_claim(DevSrv d, int slot)
{
    const TickArgs a = d.targs[slot];      // the window as k_tick_window extended it
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)(a.hi - a.lo);
    for (long long w = warp_global(); w < nw; w += warps_total()) {
        const unsigned long long t = a.lo + (unsigned long long)w;
        const int rec = (int)(t & d.mask);
        if (d.executed[rec] == t) continue;
        const DevReq q = d.req[rec];
        RecMeta m;
        m.n = q.n;
        m.kind = q.kind;
        m.has_act = q.has_act;
        m.obs_floats = q.obs_floats;
        m.off = q.cum_envs - a.base_envs;
        m.aoff = q.cum_act - a.base_act;
        m.ooff = q.cum_obs - a.base_obs;
        m.seed = q.seed;
        m.rew = q.rew;
        m.done = q.done;
        m.obs = q.obs;
        const int n = m.n;
        if (m.off < 0 || m.off + n > d.A || (m.has_act && m.aoff + q.n_act > d.A_act) ||
            (m.obs_floats && m.ooff + m.obs_floats > d.A_obs))
            continue;
        const uint32_t rank = (uint32_t)w;
        const int32_t* ids = q.ids;
        int sv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) sv[u] = lane + 32 * u < n ? ids[lane + 32 * u] : -1;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (sv[u] >= 0) {
                d.ids[m.off + lane + 32 * u] = sv[u];
                atomicMin(d.claim + sv[u], rank);
            }
        for (int j = 256 + lane; j < n; j += 32) {
            const int s = ids[j];
            d.ids[m.off + j] = s;
            atomicMin(d.claim + s, rank);
        }
        if (m.has_act) {
            const int8_t* acts = q.acts;
            for (int j = lane; j < q.n_act; j += 32) d.acts[m.aoff + j] = acts[j];
        }
        if (lane == 0) {
            d.claimed_tick[rec] = a.tick;
            d.meta[rec] = m;
        }
    }
}

// select: take every request that won all of its stations (its arena span
// bounds the tick's stations: at most A); write its stations' gather or reset
// entries.  Per 256 stations of a request: one round of list loads, one of
// claim (or charger-count) loads, one atomicAdd per size class present.
__global__ void __launch_bounds__(256, 2) k_tick_select(DevSrv d, DevBatch b, int slot)
{
    const TickArgs a = d.targs[slot];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const long long nw = (long long)(a.hi - a.lo);
    for (long long w = warp_global(); w < nw; w += warps_total()) {
        const unsigned long long t = a.lo + (unsigned long long)w;
        const int rec = (int)(t & d.mask);
        if (d.executed[rec] == t) continue;
        if (d.claimed_tick[rec] != a.tick) {                   // its span did not fit this tick's arenas
            if (lane == 0) atomicAdd(d.cnt + kCntBlocked, 1);
            continue;
        }
        const RecMeta m = d.meta[rec];
        const int n = m.n;
        const int32_t* ids = d.ids + m.off;
        const uint32_t rank = (uint32_t)w;
        bool mine = true;
        for (int j0 = 0; j0 < n; j0 += 256) {
            int sv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) sv[u] = j0 + lane + 32 * u < n ? ids[j0 + lane + 32 * u] : -1;
#pragma unroll
            for (int u = 0; u < 8; ++u) mine &= sv[u] < 0 || d.claim[sv[u]] == rank;
        }
        mine = __all_sync(0xFFFFFFFFu, mine);
        if (!mine) {                                            // an earlier request holds one of its stations
            if (lane == 0) atomicAdd(d.cnt + kCntBlocked, 1);
            continue;
        }
        if (lane == 0) {
            d.executed[rec] = t;
            d.adm[atomicAdd(d.cnt + kCntAdmitted, 1)] = t;
        }
        if (m.kind == CHX_SRV_RESET) {
            int rb = 0;
            if (lane == 0) rb = atomicAdd(d.cnt + kCntReset, n);
            rb = __shfl_sync(0xFFFFFFFFu, rb, 0);
            for (int j = lane; j < n; j += 32) {
                d.rslot[rb + j] = ids[j];
                d.rseed[rb + j] = m.seed;
            }
            continue;
        }
        int carry = 0;                                          // chargers of the request's earlier stations
        for (int j0 = 0; j0 < n; j0 += 256) {
            int sv[8], np[8], cl[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) sv[u] = j0 + lane + 32 * u < n ? ids[j0 + lane + 32 * u] : -1;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                np[u] = sv[u] >= 0 ? b.n_ports[sv[u]] : 0;
                cl[u] = sv[u] >= 0 ? class_of_slot(b, sv[u]) : -1;
            }
            // per class: stations of this block of 256, then one atomicAdd
            unsigned bal[8][kNumClasses];
            int tot = 0;                                        // lane c < kNumClasses: stations of class c
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int c = 0; c < kNumClasses; ++c) {
                    bal[u][c] = __ballot_sync(0xFFFFFFFFu, cl[u] == c);
                    if (lane == c) tot += __popc(bal[u][c]);
                }
            int base = 0;
            if (lane < kNumClasses && tot > 0) base = atomicAdd(d.cnt + kCntClass + lane, tot);
            int before[kNumClasses];                            // stations of class c in earlier rows u
#pragma unroll
            for (int c = 0; c < kNumClasses; ++c) before[c] = __shfl_sync(0xFFFFFFFFu, base, c);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                int incl = np[u];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int excl = carry + incl - np[u];
                carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
                int pos = 0;
#pragma unroll
                for (int c = 0; c < kNumClasses; ++c) {
                    if (cl[u] == c) pos = before[c] + __popc(bal[u][c] & lt);
                    before[c] += __popc(bal[u][c]);
                }
                if (sv[u] >= 0) {
                    const int j = j0 + lane + 32 * u;
                    const int act = m.has_act ? (int)(m.aoff + excl) : -1;
                    const int ob = m.obs_floats ? (int)(m.ooff + 8LL * j + 6LL * excl) : -1;
                    d.gather[(long long)cl[u] * d.G + pos] = make_int4(sv[u], act, (int)(m.off + j), ob);
                }
            }
        }
    }
}

// prepare the step: block 0 pads each class's entries to whole warp tiles
// with the class's padding slot and zeroes the fused kernel's work counters;
// every block then starts new episodes for the reset entries
__global__ void k_tick_prep(DevSrv d, DevBatch b, DevParams p)
{
    if (blockIdx.x == 0) {
        const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (c < kNumClasses) {
            const int n = d.cnt[kCntClass + c], epw = tile_epw(c);
            const int padded = (n + epw - 1) / epw * epw;
            for (int i = n + lane; i < padded; i += 32)
                d.gather[(long long)c * d.G + i] = make_int4(d.pad_slot[c], -1, 0, -1);
        }
        if (threadIdx.x < kFusedCounters) d.cnt[kCntWork + threadIdx.x] = 0;
    }
    const int n_reset = d.cnt[kCntReset];
    for (int j = blockIdx.x; j < n_reset; j += gridDim.x) reset_one_slot(b, p, d.rslot[j], d.rseed[j]);
}

// finish: clear the claims of the tick's window; deliver the taken requests'
// outputs into their pinned buffers and raise their completion flags
__global__ void k_tick_finish(DevSrv d, int slot)
{
    const TickArgs a = d.targs[slot];
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)(a.hi - a.lo);
    for (long long w = warp_global(); w < nw; w += warps_total()) {
        const unsigned long long t = a.lo + (unsigned long long)w;
        const int rec = (int)(t & d.mask);
        if (d.claimed_tick[rec] != a.tick) continue;
        const long long off = d.meta[rec].off;
        const int n = d.meta[rec].n;
        for (int j0 = 0; j0 < n; j0 += 256) {
            int sv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) sv[u] = j0 + lane + 32 * u < n ? d.ids[off + j0 + lane + 32 * u] : -1;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (sv[u] >= 0) d.claim[sv[u]] = 0xFFFFFFFFu;
        }
    }
    const int n_adm = d.cnt[kCntAdmitted];
    for (long long k = warp_global(); k < n_adm; k += warps_total()) {
        const unsigned long long t = d.adm[k];
        const int rec = (int)(t & d.mask);
        const RecMeta m = d.meta[rec];
        if (m.kind == CHX_SRV_STEP) {
            for (int j = lane; j < m.n; j += 32) {
                m.rew[j] = d.rew[m.off + j];
                m.done[j] = d.done[m.off + j];
            }
            for (int j = lane; j < m.obs_floats; j += 32) m.obs[j] = d.obs[m.ooff + j];
        }
        __threadfence_system();
        __syncwarp();
        if (lane == 0) *reinterpret_cast<volatile unsigned long long*>(d.done_flag + rec) = t;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        TickResult r;
        r.admitted = d.cnt[kCntAdmitted];
        r.stepped = d.cnt[kCntClass] + d.cnt[kCntClass + 1] + d.cnt[kCntClass + 2] + d.cnt[kCntClass + 3] +
                    d.cnt[kCntClass + 4];
        r.resets = d.cnt[kCntReset];
        r.blocked = d.cnt[kCntBlocked];
        volatile int* dst = reinterpret_cast<volatile int*>(d.result + a.slot);
        dst[0] = r.admitted;
        dst[1] = r.stepped;
        dst[2] = r.resets;
        dst[3] = r.blocked;
    }
}

struct TickSlot {
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;
    cudaGraphExec_t exec = nullptr;        // the slot's tick, captured once
};

inline void cpu_relax()
{
#if defined(__x86_64__) || defined(__i386__)
    __builtin_ia32_pause();
#endif
}

// Per-thread slots of the submission path: each host thread takes one (by a
// thread-local index, shared by every server), so that the per-request
// bookkeeping below touches a cache line that no other thread writes.
constexpr int kThreadSlots = 64;
inline int thread_slot()
{
    static std::atomic<int> next{0};
    thread_local const int i = next.fetch_add(1, std::memory_order_relaxed) % kThreadSlots;
    return i;
}
struct alignas(64) ThreadSlot {
    std::atomic<int> readers{0};           // submissions of the slot's threads inside the admin lock
    std::atomic<int64_t> ns_submit{0}, ns_complete{0};
};

// Admission and eviction against submissions: many readers (submissions, each
// on its own thread slot), rare writers (admit / evict).  A reader announces
// itself on its slot, then checks the writer flag; a writer raises the flag,
// then waits until every slot is empty (both sides sequentially consistent,
// so one of them always sees the other).
struct AdminLock {
    ThreadSlot slot[kThreadSlots];
    alignas(64) std::atomic<int> writer{0};
    std::mutex writers;                    // one writer at a time
    void lock_shared(int i)
    {
        for (;;) {
            slot[i].readers.fetch_add(1, std::memory_order_seq_cst);
            if (!writer.load(std::memory_order_seq_cst)) return;
            slot[i].readers.fetch_sub(1, std::memory_order_seq_cst);
            for (int n = 0; writer.load(std::memory_order_acquire); ++n)
                if (n < 64) cpu_relax();
                else std::this_thread::yield();
        }
    }
    void unlock_shared(int i) { slot[i].readers.fetch_sub(1, std::memory_order_release); }
    void lock()
    {
        writers.lock();
        writer.store(1, std::memory_order_seq_cst);
        for (int i = 0; i < kThreadSlots; ++i)
            for (int n = 0; slot[i].readers.load(std::memory_order_seq_cst) != 0; ++n)
                if (n < 64) cpu_relax();
                else std::this_thread::yield();
    }
    void unlock()
    {
        writer.store(0, std::memory_order_release);
        writers.unlock();
    }
};
struct SharedAdmin {                       // scoped reader
    AdminLock& l;
    int i;
    bool held = true;
    SharedAdmin(AdminLock& l_, int i_) : l(l_), i(i_) { l.lock_shared(i); }
    void unlock()
    {
        if (held) l.unlock_shared(i);
        held = false;
    }
    ~SharedAdmin() { unlock(); }
};

// The ticket counter and the running totals of submitted work, on one cache
// line behind a spin lock: the critical section is a few stores, so a
// waiting thread spins instead of sleeping in the kernel.
struct alignas(64) TicketState {
    std::atomic<int> busy{0};
    uint64_t next_ticket = 1;
    int64_t cum_envs = 0, cum_act = 0, cum_obs = 0;
    void lock()
    {
        for (int n = 0;; ++n) {
            if (!busy.load(std::memory_order_relaxed) && !busy.exchange(1, std::memory_order_acquire)) return;
            if (n < 256) cpu_relax();
            else std::this_thread::yield();
        }
    }
    void unlock() { busy.store(0, std::memory_order_release); }
};

}  // namespace

struct chx_srv {
    chx_srv_cfg cfg{};
    chx_env_params params{};
    DevParams dp{};
    int device = 0, sm_count = 0;
    DevBatch b{};
    Buffers bufs;
    int cap[kNumClasses] = {};
    int pad_slot[kNumClasses] = {};
    std::vector<int> free_slots[kNumClasses];
    // per slot: admitted flag, size class, charger count (written under the
    // exclusive admin lock, read under the shared one)
    struct SlotInfo {
        uint8_t admitted, cls;
        uint16_t nports;
    };
    std::vector<SlotInfo> slot;
    double used_bytes = 0.0;
    int n_resident = 0;
    cudaStream_t admin = nullptr;          // admission uploads
    cudaStream_t st = nullptr;             // the ticks, in order
    FusedSide side;                        // the 128-charger class's step beside the smaller classes'
    AdminLock admin_mu;                    // admit / evict exclusive, submit shared

    // requests
    PinnedPool pool;                       // the records' buffers
    std::vector<Request> table;
    DevReq* h_req = nullptr;               // [kMaxOutstanding] pinned, mapped
    unsigned long long* h_done_flag = nullptr;   // [kMaxOutstanding] pinned, mapped
    TickResult* h_result = nullptr;        // [n_streams] pinned, mapped
    TickArgs* h_args = nullptr;            // [n_streams] pinned, mapped: each tick slot's arguments
    TickArgs* d_args = nullptr;            // their device address
    TicketState tk;                        // tickets and running totals
    std::atomic<bool> sleeping{false};     // the scheduler blocks on `wake`

    // ticks
    DevSrv d{};
    std::vector<TickSlot> tslots;
    std::thread sched_thread;
    std::mutex wake_mu;
    std::condition_variable wake;
    std::atomic<bool> stopping{false};
    std::atomic<bool> failed{false};
    std::atomic<int> fail_code{0};         // the CUDA error that stopped the ticks
    std::atomic<int> fail_where{0};        // 1 launch, 2 event query, 3 elapsed time
    int max_tick_envs = 0;
    int64_t max_tick_obs = 0;
    int threads = 256;

    // statistics
    std::mutex stat_mu;
    uint64_t n_ticks = 0, n_requests = 0, n_env_steps = 0, n_resets = 0;
    double busy_ms = 0.0;
    int64_t t_start = 0;
    std::atomic<int64_t> ns_scan{0}, ns_launch{0}, n_scans{0};   // the scheduler's (submit and collect time: per thread slot)
};

namespace {

int alloc_pool(chx_srv* s)
{
    DevBatch& b = s->b;
    long long port_base = 0;
    int env_base = 0;
    for (int c = 0; c < kNumClasses; ++c) {
        const int n = s->cap[c] + 1;          // + one padding slot
        b.cls_n_env[c] = n;
        b.cls_env_base[c] = env_base;
        b.cls_port_base[c] = port_base;
        s->pad_slot[c] = env_base + s->cap[c];
        env_base += n;
        port_base += (long long)n * (8 << c);
    }
    b.n_slots = env_base;
    const size_t PS = (size_t)port_base, NS = (size_t)env_base;
    auto al = [&](void** p, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) return fail(CHX_ENOMEM, "pool allocation of " + std::to_string(bytes) + " bytes failed");
        s->bufs.push_back(*p);
        e = cudaMemset(*p, 0, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
        return CHX_OK;
    };
    int rc = 0;
#define PA(ptr, n) \
    if ((rc = al((void**)&(ptr), (n) * sizeof(*(ptr))))) return rc;
    PA(b.soc, PS) PA(b.erem, PS) PA(b.cap, PS) PA(b.rbar, PS) PA(b.pw, PS) PA(b.trem, PS) PA(b.meta, PS)
    PA(b.gcap, PS) PA(b.ginv_eta, PS) PA(b.user_id, NS) PA(b.user_port_off, NS) PA(b.n_ports, NS)
    PA(b.arrival_class, NS) PA(b.grid_cap, NS) PA(b.grid_inv_eta, NS) PA(b.tod, NS) PA(b.day, NS) PA(b.gstep, NS)
    PA(b.key0, NS) PA(b.key1, NS) PA(b.ncar, NS) PA(b.ep_ret, NS) PA(b.last_ret, NS) PA(b.n_episodes, NS) PA(b.st_arrived, NS)
    PA(b.st_rejected, NS) PA(b.st_missing, NS) PA(b.st_charged, NS) PA(b.err, 1)
#undef PA
    std::vector<int32_t> minus1(NS, -1);
    SRV_TRY(cudaMemcpy(b.user_id, minus1.data(), NS * sizeof(int32_t), cudaMemcpyHostToDevice));
    s->slot.assign(NS, chx_srv::SlotInfo{0, 0, 0});
    for (int c = 0; c < kNumClasses; ++c)
        for (int i = 0; i < b.cls_n_env[c]; ++i) s->slot[b.cls_env_base[c] + i].cls = (uint8_t)c;
    for (int c = 0; c < kNumClasses; ++c) {
        s->free_slots[c].clear();
        for (int i = s->cap[c] - 1; i >= 0; --i) s->free_slots[c].push_back(b.cls_env_base[c] + i);
    }
    return CHX_OK;
}

inline int class_of_slot_host(const chx_srv* s, int slot) { return s->slot[slot].cls; }

// device-side state of the ticks: arenas for a window of (n_streams + 1)
// ticks' requests, the claim array, the per-class entry lists
int alloc_ticks(chx_srv* s)
{
    DevSrv& d = s->d;
    const int ns = s->cfg.n_streams;
    d.max_tick_envs = s->max_tick_envs;
    d.A = (long long)(ns + 1) * s->max_tick_envs;
    d.G = (int)d.A + 8;
    d.A_act = d.A * CHX_MAX_PORTS;
    d.A_obs = std::max<long long>(1, (long long)(ns + 1) * s->max_tick_obs);
    d.mask = kMaxOutstanding - 1;
    for (int c = 0; c < kNumClasses; ++c) d.pad_slot[c] = s->pad_slot[c];
    auto al = [&](void** p, size_t bytes, int fill) -> int {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) return fail(CHX_ENOMEM, "serving allocation of " + std::to_string(bytes) + " bytes failed");
        s->bufs.push_back(*p);
        if ((e = cudaMemset(*p, fill, std::max<size_t>(bytes, 16))) != cudaSuccess) return cuda_fail(e, "cudaMemset");
        return CHX_OK;
    };
    const size_t R = kMaxOutstanding;
    int rc = 0;
    if ((rc = al((void**)&d.executed, R * 8, 0)) || (rc = al((void**)&d.claimed_tick, R * 4, 0)) ||
        (rc = al((void**)&d.meta, R * sizeof(RecMeta), 0)) ||
        (rc = al((void**)&d.adm, R * 8, 0)) || (rc = al((void**)&d.claim, (size_t)s->b.n_slots * 4, 0xFF)) ||
        (rc = al((void**)&d.ids, (size_t)d.A * 4, 0)) || (rc = al((void**)&d.acts, (size_t)d.A_act, 0)) ||
        (rc = al((void**)&d.rew, (size_t)d.A * 4, 0)) || (rc = al((void**)&d.done, (size_t)d.A, 0)) ||
        (rc = al((void**)&d.obs, (size_t)d.A_obs * 4, 0)) ||
        (rc = al((void**)&d.gather, (size_t)kNumClasses * d.G * sizeof(int4), 0)) ||
        (rc = al((void**)&d.rslot, (size_t)d.A * 4, 0)) || (rc = al((void**)&d.rseed, (size_t)d.A * 8, 0)) ||
        (rc = al((void**)&d.cnt, kCnt * 4, 0)) || (rc = al((void**)&d.targs, (size_t)ns * sizeof(TickArgs), 0)))
        return rc;
    SRV_TRY(cudaHostAlloc(&s->h_req, R * sizeof(DevReq), cudaHostAllocMapped | cudaHostAllocPortable));
    SRV_TRY(cudaHostAlloc(&s->h_done_flag, R * 8, cudaHostAllocMapped | cudaHostAllocPortable));
    SRV_TRY(cudaHostAlloc(&s->h_result, (size_t)ns * sizeof(TickResult), cudaHostAllocMapped | cudaHostAllocPortable));
    SRV_TRY(cudaHostAlloc(&s->h_args, (size_t)ns * sizeof(TickArgs), cudaHostAllocMapped | cudaHostAllocPortable));
    std::memset(s->h_args, 0, (size_t)ns * sizeof(TickArgs));
    std::memset(s->h_req, 0, R * sizeof(DevReq));
    std::memset(s->h_done_flag, 0, R * 8);
    std::memset(s->h_result, 0, (size_t)ns * sizeof(TickResult));
    void* p = nullptr;
    SRV_TRY(cudaHostGetDevicePointer(&p, s->h_req, 0));
    d.req = static_cast<const DevReq*>(p);
    SRV_TRY(cudaHostGetDevicePointer(&p, s->h_done_flag, 0));
    d.done_flag = static_cast<unsigned long long*>(p);
    SRV_TRY(cudaHostGetDevicePointer(&p, s->h_result, 0));
    d.result = static_cast<TickResult*>(p);
    SRV_TRY(cudaHostGetDevicePointer(&p, s->h_args, 0));
    s->d_args = static_cast<TickArgs*>(p);
    s->tslots.resize(ns);
    for (auto& t : s->tslots) {
        SRV_TRY(cudaEventCreate(&t.ev_start));
        SRV_TRY(cudaEventCreate(&t.ev_end));
    }
    return CHX_OK;
}

// Pinned, device-mapped memory for the request records' buffers: blocks of
// 2^k bytes carved from 64 MB chunks, with a free list per size, so that a
// submission never waits for the driver's allocator (which serialises every
// thread) once the chunks exist.
int PinnedPool::get(size_t bytes, void** host, void** dev, int* cls)
{
    int k = 6;
    while (((size_t)1 << k) < bytes) ++k;
    std::lock_guard<std::mutex> g(mu);
    if (!free_list[k].empty()) {
        *host = free_list[k].back().first;
        *dev = free_list[k].back().second;
        free_list[k].pop_back();
        *cls = k;
        return CHX_OK;
    }
    const size_t sz = (size_t)1 << k;
    if (left < sz) {
        const size_t chunk = std::max<size_t>(kChunk, sz);
        void *h = nullptr, *d = nullptr;
        if (cudaHostAlloc(&h, chunk, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
            return fail(CHX_ENOMEM, "pinned request memory allocation failed");
        if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
            cudaFreeHost(h);
            return fail(CHX_ECUDA, "no device address for pinned request memory");
        }
        chunks.push_back(h);
        cur_h = static_cast<char*>(h);
        cur_d = static_cast<char*>(d);
        left = chunk;
    }
    *host = cur_h;
    *dev = cur_d;
    cur_h += sz;
    cur_d += sz;
    left -= sz;
    *cls = k;
    return CHX_OK;
}

void PinnedPool::put(void* host, void* dev, int cls)
{
    std::lock_guard<std::mutex> g(mu);
    free_list[cls].push_back({host, dev});
}

PinnedPool::~PinnedPool()
{
    for (void* h : chunks) cudaFreeHost(h);
}

// a record's buffer of at least `need` elements (grown, never shrunk)
template <class T>
int grow_pinned(PinnedPool& pool, PinnedBuf<T>& b, size_t need)
{
    if (need <= b.cap && b.h) return CHX_OK;
    void *h = nullptr, *d = nullptr;
    int cls = 0;
    const int rc = pool.get(std::max<size_t>(need, 16) * sizeof(T), &h, &d, &cls);
    if (rc) return rc;
    if (b.h) pool.put(b.h, b.d, b.cls);
    b.h = static_cast<T*>(h);
    b.d = static_cast<T*>(d);
    b.cls = cls;
    b.cap = ((size_t)1 << cls) / sizeof(T);
    return CHX_OK;
}

// The tick of slot `slot`, captured once as a CUDA graph: claim, select,
// prep, the fused step (the 128-charger class on a side branch), finish.
// Grids are fixed (grid-stride loops over the window; the fused kernels'
// resident grids, whose warps stop at the device-side tile count), and the
// window comes from the slot's pinned argument record, so one graph launch
// runs any tick.
int capture_tick(chx_srv* s, int slot)
{
    cudaStream_t cs = nullptr;
    SRV_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const int g = 2 * s->sm_count;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        k_tick_window<<<1, 32, 0, cs>>>(s->d, s->d_args, slot);
        k_tick_claim<<<g, 256, 0, cs>>>(s->d, slot);
        k_tick_select<<<g, 256, 0, cs>>>(s->d, s->b, slot);
        k_tick_prep<<<g, 32 * kNumClasses, 0, cs>>>(s->d, s->b, s->dp);
        FusedIO io{};
        io.k_steps = 1;
        io.actions = s->d.acts;            // entries with an action offset < 0 draw Philox levels
        io.lda = 1;
        io.lda_step = 1;
        io.reward = s->d.rew;
        io.done = s->d.done;
        io.ld_out = 1;
        io.ld_step = 1;
        io.obs = s->max_tick_obs > 0 ? s->d.obs : nullptr;
        io.counter = s->d.cnt + kCntWork;
        io.gather = s->d.gather;
        for (int c = 0; c < kNumClasses; ++c) io.gather_base[c] = c * s->d.G;
        io.dcount = s->d.cnt + kCntClass;
        io.dmax_small = 1 << 28;           // every resident block
        io.dmax_mid = s->cap[3] > 0 ? 1 << 28 : 0;
        io.dmax_large = s->cap[4] > 0 ? 1 << 28 : 0;
        launch_step_fused(s->b, s->dp, io, s->threads, s->sm_count, cs, &s->side);
        k_tick_finish<<<g, 256, 0, cs>>>(s->d, slot);
        e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->tslots[slot].exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "tick graph capture");
    return CHX_OK;
}

// One tick over the window [lo, hi): its arguments into the slot's record,
// then the slot's graph.
int launch_tick(chx_srv* s, uint64_t lo, uint64_t hi, int tick, int slot)
{
    const Request& q0 = s->table[lo & (kMaxOutstanding - 1)];
    TickArgs& a = s->h_args[slot];
    a.lo = lo;
    a.hi = hi;
    a.base_envs = q0.cum_envs;
    a.base_act = q0.cum_act;
    a.base_obs = q0.cum_obs;
    a.tick = tick;
    a.slot = slot;
    std::atomic_thread_fence(std::memory_order_release);
    TickSlot& ts = s->tslots[slot];
    SRV_TRY(cudaEventRecord(ts.ev_start, s->st));
    SRV_TRY(cudaGraphLaunch(ts.exec, s->st));
    SRV_TRY(cudaEventRecord(ts.ev_end, s->st));
    return CHX_OK;
}

// The scheduler: grows the window with the published tickets, launches a tick
// when there are new requests (or requests a finished tick left waiting and
// nothing is queued on the device), keeps up to n_streams ticks queued,
// collects their reports.  Per request it does O(1) work.
void scheduler(chx_srv* s)
{
    cudaSetDevice(s->device);
    const uint64_t mask = kMaxOutstanding - 1;
    const int ns = (int)s->tslots.size();
    uint64_t pub = 1, lo = 1, last_hi = 1;
    int tick = 0;
    std::deque<int> inflight;              // tick slots in launch order
    std::vector<char> slot_busy(ns, 0);
    bool retry = false;
    int idle = 0;
    volatile unsigned long long* flag = s->h_done_flag;
    // Ticket t is published once its record carries t and is no longer being
    // filled, or carries a later ticket.  A tick's window kernel may take and
    // finish a request as soon as its descriptor is published, so its caller
    // may have released it (state free) or even reused the record before
    // this thread looks.  The ticket is read before the state: the record
    // goes filling -> queued -> free under one ticket, so a ticket t read
    // with any state but filling was published.
    auto published = [&](uint64_t t) {
        const Request& q = s->table[t & mask];
        const uint64_t qt = q.ticket.load(std::memory_order_acquire);
        if (qt != t) return qt > t;
        return q.state.load(std::memory_order_seq_cst) != kFilling;
    };
    for (;;) {
        const int64_t t0 = now_ns();
        while (published(pub)) ++pub;      // published requests extend the window
        while (!inflight.empty()) {        // finished ticks
            const int sl = inflight.front();
            TickSlot& ts = s->tslots[sl];
            const cudaError_t e = cudaEventQuery(ts.ev_end);
            if (e == cudaErrorNotReady) break;
            float ms = 0.f;
            const cudaError_t et = e == cudaSuccess ? cudaEventElapsedTime(&ms, ts.ev_start, ts.ev_end) : e;
            if (et != cudaSuccess) {
                s->fail_code.store((int)et);
                s->fail_where.store(e != cudaSuccess ? 2 : 3);
                s->failed.store(true);
                ms = 0.f;
            }
            const volatile int* src = reinterpret_cast<const volatile int*>(s->h_result + sl);
            const TickResult r{src[0], src[1], src[2], src[3]};
            {
                std::lock_guard<std::mutex> g(s->stat_mu);
                if (r.admitted > 0) s->n_ticks += 1;
                s->n_requests += (uint64_t)r.admitted;
                s->n_env_steps += (uint64_t)r.stepped;
                s->n_resets += (uint64_t)r.resets;
                s->busy_ms += ms;
            }
            if (r.blocked > 0) retry = true;
            slot_busy[sl] = 0;
            inflight.pop_front();
        }
        while (lo < pub) {                 // the window starts at the oldest unfinished request
            const Request& q = s->table[lo & mask];
            if (q.ticket.load(std::memory_order_acquire) == lo && q.state.load(std::memory_order_acquire) != kFree &&
                flag[lo & mask] != lo)
                break;
            ++lo;
        }
        if (s->stopping.load() && inflight.empty()) return;
        const bool fresh = pub > last_hi;
        if (!s->stopping.load() && !s->failed.load() && lo < pub && (int)inflight.size() < ns &&
            (fresh || (retry && inflight.empty()))) {
            int sl = 0;
            while (slot_busy[sl]) ++sl;
            ++tick;
            s->ns_scan += now_ns() - t0;
            const int64_t t1 = now_ns();
            // at most one ticket per record in a window: an index whose
            // record a later ticket reuses is then one that was executed and
            // still marked so (the later ticket lies past every earlier window)
            const uint64_t hi = std::min(pub, lo + kMaxOutstanding);
            if (launch_tick(s, lo, hi, tick, sl) != CHX_OK) {
                s->fail_code.store((int)cudaGetLastError());
                s->fail_where.store(1);
                s->failed.store(true);
            }
            s->ns_launch += now_ns() - t1;
            s->n_scans += 1;
            slot_busy[sl] = 1;
            inflight.push_back(sl);
            last_hi = hi;                  // requests past a clamped window stay fresh
            retry = false;
            idle = 0;
            continue;
        }
        s->ns_scan += now_ns() - t0;
        // nothing to launch: spin briefly (ticks finish within tens of
        // microseconds), then block until a submission or a timeout
        if (++idle < 2000 || !inflight.empty()) {
            cpu_relax();
            if (idle > 200) std::this_thread::yield();
            continue;
        }
        {
            std::unique_lock<std::mutex> lk(s->wake_mu);
            s->sleeping.store(true, std::memory_order_seq_cst);
            s->wake.wait_for(lk, std::chrono::microseconds(200),
                             [&] { return published(pub) || s->stopping.load(); });
            s->sleeping.store(false, std::memory_order_relaxed);
        }
        idle = 0;
    }
}

// Copy a finished request's results to the caller's buffers and release it.
int collect(chx_srv* s, Request& q, int64_t* latency_ns)
{
    const int64_t t0 = now_ns();
    if (latency_ns) *latency_ns = t0 - q.t_submit;
    if (q.kind == CHX_SRV_STEP) {
        if (q.h_reward) std::memcpy(q.h_reward, q.rew.h, (size_t)q.n * sizeof(float));
        if (q.h_done) std::memcpy(q.h_done, q.done.h, (size_t)q.n);
        if (q.h_obs) std::memcpy(q.h_obs, q.obs.h, (size_t)q.obs_floats * sizeof(float));
    }
    q.state.store(kFree, std::memory_order_release);
    s->admin_mu.slot[thread_slot()].ns_complete.fetch_add(now_ns() - t0, std::memory_order_relaxed);
    return CHX_OK;
}

// Write admitted stations' statics into their slots: one warp per station.
__global__ void k_admit_scatter(DevBatch b, int n, const int32_t* __restrict__ slots,
                                const int32_t* __restrict__ nports, const int32_t* __restrict__ arr,
                                const float* __restrict__ gcap_root, const float* __restrict__ ginv_root,
                                const long long* __restrict__ poff, const uint32_t* __restrict__ meta,
                                const float* __restrict__ gcap, const float* __restrict__ ginv)
{
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const int s = slots[j];
    const int c = class_of_slot(b, s);
    const int C = 8 << c;
    const long long pb = b.cls_port_base[c] + (long long)(s - b.cls_env_base[c]) * C;
    for (int q = lane; q < C; q += 32) {
        b.meta[pb + q] = meta[poff[j] + q];
        b.gcap[pb + q] = gcap[poff[j] + q];
        b.ginv_eta[pb + q] = ginv[poff[j] + q];
    }
    if (lane == 0) {
        b.user_id[s] = s;
        b.user_port_off[s] = 0;
        b.n_ports[s] = nports[j];
        b.arrival_class[s] = arr[j];
        b.grid_cap[s] = gcap_root[j];
        b.grid_inv_eta[s] = ginv_root[j];
    }
}

}  // namespace

// ===========================================================================
// C interface
// ===========================================================================

extern "C" int chx_srv_start(const chx_srv_cfg* cfg, chx_srv** out)
{
    if (!cfg || !out) return fail(CHX_EINVAL, "null argument");
    *out = nullptr;
    if (cfg->params.v2g) return fail(CHX_EINVAL, "the serving loop runs the charge-only mode (v2g = 0)");
    if (cfg->params.action_delta) return fail(CHX_EINVAL, "the serving loop takes absolute levels (action_delta = 0)");
    if (cfg->params.cs_share_256) return fail(CHX_EINVAL, "the serving loop runs time-sensitive users only (cs_share_256 = 0)");
    int rc = validate_params(&cfg->params, &cfg->exo);
    if (rc) return rc;
    if (cfg->max_tick_envs < 1 || cfg->max_tick_envs > (1 << 20)) return fail(CHX_EINVAL, "max_tick_envs out of range");
    if (cfg->n_streams < 1 || cfg->n_streams > 8) return fail(CHX_EINVAL, "n_streams must be in 1..8");
    if (cfg->max_tick_obs_floats < 0 || (long long)(cfg->n_streams + 1) * cfg->max_tick_obs_floats > INT32_MAX)
        return fail(CHX_EINVAL, "max_tick_obs_floats x (n_streams + 1) must stay below 2^31");
    long long total = 0;
    for (int c = 0; c < kNumClasses; ++c) {
        if (cfg->class_capacity[c] < 0) return fail(CHX_EINVAL, "class_capacity must be >= 0");
        total += cfg->class_capacity[c];
    }
    if (total < 1 || total > (1LL << 24)) return fail(CHX_EINVAL, "pool capacity out of range");
    auto* s = new chx_srv();
    s->cfg = *cfg;
    s->params = cfg->params;
    s->dp = make_params(cfg->params, cfg->exo.n_days);
    s->max_tick_envs = cfg->max_tick_envs;
    s->max_tick_obs = cfg->max_tick_obs_floats;
    s->table = std::vector<Request>(kMaxOutstanding);
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
        delete s;
        return fail(CHX_ECUDA, "no CUDA device");
    }
    for (int c = 0; c < kNumClasses; ++c) s->cap[c] = cfg->class_capacity[c];
    if ((rc = alloc_pool(s))) {
        chx_srv_stop(s);
        return rc;
    }
    const size_t nprice = (size_t)cfg->exo.n_days * cfg->params.ep_len;
    const size_t nlam = (size_t)cfg->exo.n_arrival_classes * cfg->params.ep_len;
    float *price = nullptr, *cdf = nullptr;
    if (cudaMalloc(&price, nprice * 4) != cudaSuccess || cudaMalloc(&cdf, nlam * kCdfLen * 4) != cudaSuccess) {
        cudaFree(price);
        chx_srv_stop(s);
        return fail(CHX_ENOMEM, "exogenous table allocation failed");
    }
    s->bufs.push_back(price);
    s->bufs.push_back(cdf);
    std::vector<float> F;
    build_poisson_cdf(cfg->exo.h_arrival_rate, nlam, F);
    if (cudaMemcpy(price, cfg->exo.h_price, nprice * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(cdf, F.data(), F.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        chx_srv_stop(s);
        return fail(CHX_ECUDA, "exogenous table upload failed");
    }
    s->b.price = price;
    s->b.cdf = cdf;
    s->threads = 256;
    if (!fused_block_size_ok(s->threads)) {
        chx_srv_stop(s);
        return fail(CHX_ECUDA, "fused kernel cannot be resident");
    }
    if ((rc = alloc_ticks(s))) {
        chx_srv_stop(s);
        return rc;
    }
    if (cudaStreamCreateWithFlags(&s->admin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->side.aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->side.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->side.join, cudaEventDisableTiming) != cudaSuccess) {
        chx_srv_stop(s);
        return fail(CHX_ECUDA, "stream creation failed");
    }
    for (int sl = 0; sl < cfg->n_streams; ++sl)
        if ((rc = capture_tick(s, sl))) {
            chx_srv_stop(s);
            return rc;
        }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        chx_srv_stop(s);
        return fail(CHX_ECUDA, "server set-up failed on the device");
    }
    s->t_start = now_ns();
    s->sched_thread = std::thread(scheduler, s);
    *out = s;
    return CHX_OK;
}

extern "C" int chx_srv_stop(chx_srv* s)
{
    if (!s) return CHX_OK;
    s->stopping.store(true);
    {
        std::lock_guard<std::mutex> lk(s->wake_mu);
        s->wake.notify_all();
    }
    if (s->sched_thread.joinable()) s->sched_thread.join();
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->admin) cudaStreamSynchronize(s->admin);
    for (auto& t : s->tslots) {
        if (t.exec) cudaGraphExecDestroy(t.exec);
        if (t.ev_start) cudaEventDestroy(t.ev_start);
        if (t.ev_end) cudaEventDestroy(t.ev_end);
    }
    if (s->h_args) cudaFreeHost(s->h_args);
    if (s->h_req) cudaFreeHost(s->h_req);
    if (s->h_done_flag) cudaFreeHost(s->h_done_flag);
    if (s->h_result) cudaFreeHost(s->h_result);
    for (void* p : s->bufs) cudaFree(p);
    if (s->admin) cudaStreamDestroy(s->admin);
    if (s->st) cudaStreamDestroy(s->st);
    if (s->side.aux) cudaStreamSynchronize(s->side.aux), cudaStreamDestroy(s->side.aux);
    if (s->side.fork) cudaEventDestroy(s->side.fork);
    if (s->side.join) cudaEventDestroy(s->side.join);
    delete s;
    return CHX_OK;
}

extern "C" int chx_srv_admit(chx_srv* s, const chx_stations* st, uint64_t seed, int32_t* h_ids)
{
    if (!s || !st || !h_ids) return fail(CHX_EINVAL, "null argument");
    if (st->h_n_upper) return fail(CHX_EINVAL, "the serving loop takes two-level trees (h_n_upper = NULL)");
    int rc = validate_stations(st, &s->cfg.exo, 1LL << 24);
    if (rc) return rc;
    std::unique_lock<AdminLock> lk(s->admin_mu);
    // all or nothing: class capacity and HBM budget
    int need[kNumClasses] = {};
    double bytes = 0.0;
    for (int e = 0; e < st->n_envs; ++e) {
        const int c = class_of_ports(st->h_n_ports[e]);
        need[c] += 1;
        bytes += slot_bytes(c);
    }
    for (int c = 0; c < kNumClasses; ++c)
        if (need[c] > (int)s->free_slots[c].size())
            return fail(CHX_ENOMEM, "no free slot for a station of the " + std::to_string(8 << c) + "-charger class");
    if (s->used_bytes + bytes > s->cfg.hbm_budget_bytes)
        return fail(CHX_ENOMEM, "admission would exceed the HBM budget");
    // host images of the new stations (per-charger statics packed by class
    // size), uploaded at once and scattered into their slots by a kernel
    DevBatch& b = s->b;
    const int n_new = st->n_envs;
    std::vector<int32_t> slots(n_new), nports(n_new), arr(n_new);
    std::vector<float> g_cap(n_new), g_inv(n_new);
    std::vector<long long> poff(n_new + 1, 0);
    for (int e = 0; e < n_new; ++e) poff[e + 1] = poff[e] + (8 << class_of_ports(st->h_n_ports[e]));
    std::vector<uint32_t> meta(poff[n_new], 0u);
    std::vector<float> gcap(poff[n_new], 0.f), ginv(poff[n_new], 0.f);
    long long po = 0, go = 0;
    for (int e = 0; e < n_new; ++e) {
        const int n = st->h_n_ports[e];
        const int c = class_of_ports(n);
        slots[e] = s->free_slots[c].back();
        s->free_slots[c].pop_back();
        nports[e] = n;
        arr[e] = st->h_arrival_class[e];
        const double eta0 = st->h_grid_eta ? st->h_grid_eta[e] : 1.0;
        g_cap[e] = (float)(eta0 * (double)st->h_grid_limit_kw[e]);
        g_inv[e] = (float)(1.0 / eta0);
        int q = 0;
        for (int k = 0; k < st->h_n_groups[e]; ++k) {
            const long long gi = go + k;
            const int gs = st->h_group_size[gi];
            const double eta = st->h_group_eta ? st->h_group_eta[gi] : 1.0;
            for (int r = 0; r < gs; ++r, ++q) {
                uint32_t m = kMetaValid | (uint32_t)k << kMetaGroupShift;
                if (st->h_port_type[po + q]) m |= kMetaDC;
                if (r == 0) m |= kMetaHead;
                if (r == gs - 1) m |= kMetaTail;
                meta[poff[e] + q] = m;
                gcap[poff[e] + q] = (float)(eta * (double)st->h_group_limit_kw[gi]);
                ginv[poff[e] + q] = (float)(1.0 / eta);
            }
        }
        s->slot[slots[e]].admitted = 1;
        s->slot[slots[e]].nports = (uint16_t)n;
        s->used_bytes += slot_bytes(c);
        s->n_resident += 1;
        po += n;
        go += st->h_n_groups[e];
    }
    std::vector<unsigned long long> seeds(n_new, (unsigned long long)seed);
    void* tmp[10] = {};
    const void* src[10] = {slots.data(), nports.data(), arr.data(), g_cap.data(), g_inv.data(),
                           poff.data(),  meta.data(),   gcap.data(), ginv.data(), seeds.data()};
    const size_t sz[10] = {n_new * 4u, n_new * 4u, n_new * 4u, n_new * 4u, n_new * 4u,
                           (n_new + 1) * 8u, meta.size() * 4, gcap.size() * 4, ginv.size() * 4, n_new * 8u};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 10 && e == cudaSuccess; ++i) {
        e = cudaMalloc(&tmp[i], std::max<size_t>(sz[i], 16));
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp[i], src[i], sz[i], cudaMemcpyHostToDevice, s->admin);
    }
    if (e == cudaSuccess) {
        k_admit_scatter<<<(n_new + 3) / 4, 128, 0, s->admin>>>(
            b, n_new, (const int32_t*)tmp[0], (const int32_t*)tmp[1], (const int32_t*)tmp[2], (const float*)tmp[3],
            (const float*)tmp[4], (const long long*)tmp[5], (const uint32_t*)tmp[6], (const float*)tmp[7],
            (const float*)tmp[8]);
        launch_reset_slots(b, s->dp, (const int32_t*)tmp[0], (const unsigned long long*)tmp[9], n_new, s->admin);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->admin);
    }
    for (void* t : tmp) cudaFree(t);
    if (e != cudaSuccess) return cuda_fail(e, "station admission");
    std::memcpy(h_ids, slots.data(), n_new * sizeof(int32_t));
    return CHX_OK;
}

extern "C" int chx_srv_evict(chx_srv* s, const int32_t* h_ids, int32_t n)
{
    if (!s || (!h_ids && n > 0) || n < 0) return fail(CHX_EINVAL, "bad argument");
    std::unique_lock<AdminLock> lk(s->admin_mu);
    for (int j = 0; j < n; ++j) {
        const int e = h_ids[j];
        if (e < 0 || e >= s->b.n_slots || !s->slot[e].admitted) return fail(CHX_EINVAL, "station id not admitted");
    }
    // no ticket that lists one of them may be unreleased (queued, in flight or
    // finished and not yet collected); submissions hold the shared lock, so
    // none is being filled now
    {
        std::vector<uint8_t> gone((size_t)s->b.n_slots, 0);
        for (int j = 0; j < n; ++j) gone[h_ids[j]] = 1;
        for (const Request& q : s->table)
            if (q.state.load(std::memory_order_acquire) == kQueued)
                for (int j = 0; j < q.n; ++j)
                    if (gone[q.ids.h[j]]) return fail(CHX_EINVAL, "station is listed by a ticket not yet released");
    }
    DevBatch& b = s->b;
    const int32_t minus1 = -1;
    for (int j = 0; j < n; ++j) {
        const int e = h_ids[j];
        const int c = class_of_slot_host(s, e);
        const int C = 8 << c;
        const long long pb = b.cls_port_base[c] + (long long)(e - b.cls_env_base[c]) * C;
        SRV_TRY(cudaMemsetAsync(b.meta + pb, 0, C * 4, s->admin));
        SRV_TRY(cudaMemsetAsync(b.trem + pb, 0, C, s->admin));
        SRV_TRY(cudaMemcpyAsync(b.user_id + e, &minus1, 4, cudaMemcpyHostToDevice, s->admin));
        SRV_TRY(cudaStreamSynchronize(s->admin));
        s->slot[e].admitted = 0;
        s->slot[e].nports = 0;
        s->free_slots[c].push_back(e);
        s->used_bytes -= slot_bytes(c);
        s->n_resident -= 1;
    }
    return CHX_OK;
}

extern "C" int chx_srv_submit(chx_srv* s, const chx_srv_req* r, uint64_t* ticket)
{
    if (!s || !r || !ticket) return fail(CHX_EINVAL, "null argument");
    const int64_t t_in = now_ns();
    if (r->kind != CHX_SRV_STEP && r->kind != CHX_SRV_RESET) return fail(CHX_EINVAL, "unknown request kind");
    if (r->n_envs < 1 || r->n_envs > s->max_tick_envs || !r->h_env_ids)
        return fail(CHX_EINVAL, "n_envs must be in 1..max_tick_envs");
    const int n = r->n_envs;
    const bool step = r->kind == CHX_SRV_STEP;
    // duplicate check: a per-thread open-addressing set of at least 2n slots
    thread_local std::vector<int32_t> set;
    size_t cap = 64;
    while (cap < 2 * (size_t)n) cap *= 2;
    if (set.size() < cap) set.resize(cap);
    std::fill(set.begin(), set.begin() + cap, -1);
    const int ts = thread_slot();
    SharedAdmin lk(s->admin_mu, ts);
    if (s->stopping.load()) return fail(CHX_EINVAL, "server is stopping");
    int64_t n_act = 0;
    for (int j = 0; j < n; ++j) {
        const int32_t e = r->h_env_ids[j];
        if (e < 0 || e >= s->b.n_slots) return fail(CHX_EINVAL, "station id out of range");
        const chx_srv::SlotInfo si = s->slot[e];
        if (!si.admitted) return fail(CHX_EINVAL, "station id not admitted");
        size_t h = ((uint32_t)e * 2654435761u) & (cap - 1);
        while (set[h] >= 0 && set[h] != e) h = (h + 1) & (cap - 1);
        if (set[h] == e) return fail(CHX_EINVAL, "station listed twice in one request");
        set[h] = e;
        n_act += si.nports;
    }
    const bool given = step && r->h_actions;
    if (given)
        for (int64_t i = 0; i < n_act; ++i)
            if (r->h_actions[i] < 0 || r->h_actions[i] >= s->params.n_levels)
                return fail(CHX_EINVAL, "action level out of range");
    const int64_t obs_floats = (step && r->h_obs) ? 8LL * n + 6LL * n_act : 0;
    if (obs_floats > s->max_tick_obs) return fail(CHX_EINVAL, "observation larger than max_tick_obs_floats");
    // a record and a ticket; the record's buffers grow here (rarely, inside
    // the lock, so that a ticket is never taken without being published)
    Request* q = nullptr;
    uint64_t tk = 0;
    {
        // The next ticket's record is still held while the request
        // kMaxOutstanding tickets older is unreleased: refuse at once (a
        // submission that waited here would stop its thread from releasing
        // the tickets it holds itself, and threads could wait on each other)
        TicketState& T = s->tk;
        T.lock();
        tk = T.next_ticket;
        q = &s->table[tk & (kMaxOutstanding - 1)];
        int expect = kFree;
        if (!q->state.compare_exchange_strong(expect, kFilling, std::memory_order_acq_rel)) {
            T.unlock();
            return fail(CHX_ENOMEM, "too many outstanding requests: release tickets with chx_srv_wait or chx_srv_test");
        }
        int rc = grow_pinned(s->pool, q->ids, (size_t)n);
        if (!rc && step) rc = grow_pinned(s->pool, q->rew, (size_t)n);
        if (!rc && step) rc = grow_pinned(s->pool, q->done, (size_t)n);
        if (!rc && given) rc = grow_pinned(s->pool, q->acts, (size_t)n_act);
        if (!rc && obs_floats) rc = grow_pinned(s->pool, q->obs, (size_t)obs_floats);
        if (rc) {
            q->state.store(kFree, std::memory_order_release);
            T.unlock();
            return rc;
        }
        ++T.next_ticket;
        q->cum_envs = T.cum_envs;
        q->cum_act = T.cum_act;
        q->cum_obs = T.cum_obs;
        T.cum_envs += n;
        if (given) T.cum_act += n_act;
        T.cum_obs += obs_floats;
        T.unlock();
    }
    std::memcpy(q->ids.h, r->h_env_ids, (size_t)n * sizeof(int32_t));
    if (given) std::memcpy(q->acts.h, r->h_actions, (size_t)n_act);
    DevReq& dr = s->h_req[tk & (kMaxOutstanding - 1)];
    dr.kind = r->kind;
    dr.n = n;
    dr.n_act = (int)n_act;
    dr.has_act = given ? 1 : 0;
    dr.obs_floats = (int)obs_floats;
    dr.cum_envs = q->cum_envs;
    dr.cum_act = q->cum_act;
    dr.cum_obs = q->cum_obs;
    dr.ids = q->ids.d;
    dr.acts = given ? q->acts.d : nullptr;
    dr.rew = step ? q->rew.d : nullptr;
    dr.done = step ? q->done.d : nullptr;
    dr.obs = obs_floats ? q->obs.d : nullptr;
    dr.seed = (unsigned long long)r->seed;
    // the device takes a record as published when it reads this ticket
    __atomic_store_n(&dr.ticket, (unsigned long long)tk, __ATOMIC_RELEASE);
    q->kind = r->kind;
    q->n = n;
    q->h_reward = step ? r->h_reward : nullptr;
    q->h_done = step ? r->h_done : nullptr;
    q->h_obs = obs_floats ? r->h_obs : nullptr;
    q->obs_floats = obs_floats;
    q->t_submit = now_ns();
    q->ticket.store(tk, std::memory_order_relaxed);
    // published; then, if the scheduler has gone to sleep, wake it (it raises
    // `sleeping` before it looks for published records, both sequentially
    // consistent, so either it sees this record or this thread sees the flag)
    q->state.store(kQueued, std::memory_order_seq_cst);
    lk.unlock();
    *ticket = tk;
    if (s->sleeping.load(std::memory_order_seq_cst)) {
        std::lock_guard<std::mutex> g(s->wake_mu);
        s->wake.notify_one();
    }
    s->admin_mu.slot[ts].ns_submit.fetch_add(now_ns() - t_in, std::memory_order_relaxed);
    return CHX_OK;
}

namespace {
int failed_status(const chx_srv* s)
{
    static const char* where[] = {"", "a tick launch", "a tick's completion", "a tick's timing"};
    const int w = s->fail_where.load();
    return fail(CHX_ECUDA, std::string("the server's device work failed at ") + where[w >= 0 && w <= 3 ? w : 0] +
                               ": " + cudaGetErrorString((cudaError_t)s->fail_code.load()));
}

inline bool finished(const chx_srv* s, uint64_t ticket)
{
    return reinterpret_cast<volatile const unsigned long long*>(s->h_done_flag)[ticket & (kMaxOutstanding - 1)] ==
           ticket;
}
}  // namespace

extern "C" int chx_srv_wait(chx_srv* s, uint64_t ticket, int64_t timeout_us, int64_t* latency_ns)
{
    if (!s) return fail(CHX_EINVAL, "null server");
    Request& q = s->table[ticket & (kMaxOutstanding - 1)];
    if (q.ticket.load(std::memory_order_acquire) != ticket || q.state.load(std::memory_order_acquire) != kQueued)
        return fail(CHX_EINVAL, "unknown ticket");
    if (!finished(s, ticket)) {
        const int64_t deadline = now_ns() + 1000 * std::max<int64_t>(timeout_us, 0);
        for (int spins = 0; !finished(s, ticket); ++spins) {
            if (s->failed.load()) return failed_status(s);
            if (now_ns() >= deadline) return fail(CHX_ETIMEOUT, "request not finished within the timeout");
            if (spins < 64) cpu_relax();
            else if (spins < 4096) std::this_thread::yield();
            else std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    return collect(s, q, latency_ns);
}

extern "C" int chx_srv_test(chx_srv* s, uint64_t ticket, int32_t* h_done, int64_t* latency_ns)
{
    if (!s || !h_done) return fail(CHX_EINVAL, "null argument");
    Request& q = s->table[ticket & (kMaxOutstanding - 1)];
    if (q.ticket.load(std::memory_order_acquire) != ticket || q.state.load(std::memory_order_acquire) != kQueued)
        return fail(CHX_EINVAL, "unknown ticket");
    *h_done = 0;
    if (!finished(s, ticket)) {
        if (s->failed.load()) return failed_status(s);
        return CHX_OK;
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    *h_done = 1;
    return collect(s, q, latency_ns);
}

extern "C" int chx_srv_stats(chx_srv* s, chx_srv_stats_t* out)
{
    if (!s || !out) return fail(CHX_EINVAL, "null argument");
    {
        std::lock_guard<std::mutex> lk(s->stat_mu);
        out->n_ticks = (int64_t)s->n_ticks;
        out->n_requests = (int64_t)s->n_requests;
        out->env_steps = (int64_t)s->n_env_steps;
        out->env_resets = (int64_t)s->n_resets;
        out->device_busy_ms = s->busy_ms;
    }
    {
        SharedAdmin lk(s->admin_mu, thread_slot());
        out->resident = s->n_resident;
        out->used_bytes = s->used_bytes;
    }
    out->budget_bytes = s->cfg.hbm_budget_bytes;
    out->elapsed_ms = (double)(now_ns() - s->t_start) * 1e-6;
    int64_t ns_submit = 0, ns_complete = 0;
    for (const ThreadSlot& t : s->admin_mu.slot) {
        ns_submit += t.ns_submit.load(std::memory_order_relaxed);
        ns_complete += t.ns_complete.load(std::memory_order_relaxed);
    }
    out->host_submit_ms = ns_submit * 1e-6;
    out->host_scan_ms = s->ns_scan.load() * 1e-6;
    out->host_pack_ms = 0.0;
    out->host_launch_ms = s->ns_launch.load() * 1e-6;
    out->host_complete_ms = ns_complete * 1e-6;
    out->n_scans = s->n_scans.load();
    return CHX_OK;
}

// ---------------------------------------------------------------------------
// simulated actors: closed loop, exponential think time between an actor's
// requests, latency measured from submission to completion by the server
// ---------------------------------------------------------------------------

extern "C" int chx_srv_simulate(chx_srv* s, const chx_srv_sim_cfg* c, const int32_t* h_station_ids,
                                chx_srv_sim_result* res)
{
    if (!s || !c || !h_station_ids || !res) return fail(CHX_EINVAL, "null argument");
    if (c->n_actors < 1 || c->envs_per_actor < 1 || c->n_threads < 1 || c->n_threads > 256 ||
        !(c->duration_s > 0.0) || c->warmup_s < 0.0)
        return fail(CHX_EINVAL, "bad simulation configuration");
    const int A = c->n_actors, per = c->envs_per_actor;
    std::atomic<int> err{0};
    std::mutex err_mu;
    std::string err_msg;                   // the first failing call's message
    auto record = [&](const char* call) {
        std::lock_guard<std::mutex> g(err_mu);
        if (err_msg.empty()) err_msg = std::string(call) + ": " + chx_last_error();
        err = 1;
    };
    std::vector<std::vector<int64_t>> lat(c->n_threads);
    std::vector<int64_t> steps(c->n_threads, 0), nreq(c->n_threads, 0);
    const int64_t t0 = now_ns();
    const int64_t t_warm = t0 + (int64_t)(c->warmup_s * 1e9);
    const int64_t t_end = t_warm + (int64_t)(c->duration_s * 1e9);
    chx_srv_stats_t st0{}, st1{};
    std::atomic<bool> warm_seen{false};
    std::mutex warm_mu;
    auto worker = [&](int w) {
        std::mt19937_64 rng(c->seed * 7919ULL + (uint64_t)w);
        std::exponential_distribution<double> think(c->mean_think_us > 0 ? 1.0 / c->mean_think_us : 1e9);
        struct Actor {
            int id;
            int64_t next;
            uint64_t ticket;
            bool busy;
            int64_t count;
            int32_t kind;
            std::vector<float> rew;
            std::vector<uint8_t> done;
        };
        std::vector<Actor> actors;
        for (int a = w; a < A; a += c->n_threads)
            actors.push_back(Actor{a, t0 + (int64_t)(think(rng) * 1e3), 0, false, 0, 0, std::vector<float>(per),
                                   std::vector<uint8_t>(per)});
        bool stop = false;
        while (!stop && !err.load()) {
            const int64_t tn = now_ns();
            if (tn >= t_warm && !warm_seen.exchange(true)) {
                std::lock_guard<std::mutex> g(warm_mu);
                chx_srv_stats(s, &st0);
            }
            stop = tn >= t_end;
            bool idle = true;
            for (auto& x : actors) {
                if (x.busy) {
                    int32_t d = 0;
                    int64_t l = 0;
                    if (chx_srv_test(s, x.ticket, &d, &l)) {
                        record("chx_srv_test");
                        return;
                    }
                    if (d) {
                        x.busy = false;
                        const int64_t tc = now_ns();
                        if (tc - l >= t_warm && tc <= t_end) {
                            lat[w].push_back(l);
                            nreq[w] += 1;
                            if (x.kind == CHX_SRV_STEP) steps[w] += per;
                        }
                        x.count += 1;
                        x.next = tc + (int64_t)(think(rng) * 1e3);
                        idle = false;
                    }
                } else if (!stop && tn >= x.next) {
                    chx_srv_req r{};
                    x.kind = (c->reset_every > 0 && x.count > 0 && x.count % c->reset_every == 0) ? CHX_SRV_RESET
                                                                                                  : CHX_SRV_STEP;
                    r.kind = x.kind;
                    r.n_envs = per;
                    r.h_env_ids = h_station_ids + (int64_t)x.id * per;
                    r.h_reward = x.rew.data();
                    r.h_done = x.done.data();
                    r.seed = c->seed + (uint64_t)x.count;
                    const int rc = chx_srv_submit(s, &r, &x.ticket);
                    if (rc == CHX_ENOMEM) continue;   // every record held: try again on the next pass
                    if (rc) {
                        record("chx_srv_submit");
                        return;
                    }
                    x.busy = true;
                    idle = false;
                }
            }
            if (idle) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        for (auto& x : actors)            // drain
            if (x.busy) chx_srv_wait(s, x.ticket, 30000000, nullptr);
    };
    std::vector<std::thread> th;
    for (int w = 0; w < c->n_threads; ++w) th.emplace_back(worker, w);
    for (auto& t : th) t.join();
    chx_srv_stats(s, &st1);
    if (err.load()) return fail(CHX_EINVAL, "a simulated actor's call failed: " + err_msg);
    std::vector<int64_t> all;
    int64_t total_steps = 0, total_req = 0;
    for (int w = 0; w < c->n_threads; ++w) {
        all.insert(all.end(), lat[w].begin(), lat[w].end());
        total_steps += steps[w];
        total_req += nreq[w];
    }
    std::sort(all.begin(), all.end());
    auto pct = [&](double q) -> double {
        if (all.empty()) return 0.0;
        const size_t i = (size_t)std::min<double>((double)all.size() - 1, std::floor(q * (double)all.size()));
        return (double)all[i] * 1e-3;
    };
    double sum = 0.0;
    for (int64_t v : all) sum += (double)v;
    res->n_requests = total_req;
    res->env_steps = total_steps;
    res->seconds = c->duration_s;
    res->env_steps_per_s = (double)total_steps / c->duration_s;
    res->p50_us = pct(0.50);
    res->p90_us = pct(0.90);
    res->p99_us = pct(0.99);
    res->max_us = all.empty() ? 0.0 : (double)all.back() * 1e-3;
    res->mean_us = all.empty() ? 0.0 : sum / (double)all.size() * 1e-3;
    const int64_t dticks = st1.n_ticks - st0.n_ticks;
    res->mean_tick_envs = dticks > 0 ? (double)(st1.env_steps - st0.env_steps) / (double)dticks : 0.0;
    res->device_busy_frac =
        (st1.device_busy_ms - st0.device_busy_ms) / std::max(1e-9, st1.elapsed_ms - st0.elapsed_ms);
    return CHX_OK;
}
