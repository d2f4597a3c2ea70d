// serve.cu -- the serving loop: a pool of device-resident stations stepped by
// requests from many actors with continuous batching.
//
// * Pool: station slots bucketed by size class (the layout of chx_device.cuh),
//   allocated once; stations are admitted into free slots while the bytes they
//   occupy stay within an HBM budget, and evicted to free them.  A station's
//   id is its slot, which is also its Philox stream id.
// * Requests (step or reset of a list of stations) are queued by
//   chx_srv_submit.  A scheduler thread packs pending requests into a tick --
//   every request whose stations are not in flight, in arrival order, up to a
//   tick size -- and launches it on one of several streams: up to n_streams
//   ticks run on the device at once while the next one is being packed, so a
//   request that arrives while others are on the GPU joins the next tick as
//   soon as its stations are free.  A completion thread waits for each tick,
//   copies results to the requesters' buffers and completes their tickets.
// * A tick's step is the warp-cooperative kernel of step_fused.cu in gather
//   mode (one step, tiles formed from the tick's stations of one class).  Its
//   reductions depend only on a charger's position inside its station, so a
//   request's results are the same whatever else shares its tick.
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

constexpr int kFree = 0, kQueued = 1, kDone = 2;

// A request record.  Records live in a fixed table indexed by ticket modulo
// its size, so their addresses never change and a ticket's state can be read
// without the server lock.
struct Request {
    std::atomic<int> state{kFree};
    std::atomic<uint64_t> ticket{0};
    int32_t kind = 0;
    std::vector<int32_t> envs;
    std::vector<int8_t> actions;          // empty = Philox levels
    std::vector<int32_t> act_off;         // [n+1]: charger offsets of the listed stations
    float* h_reward = nullptr;
    uint8_t* h_done = nullptr;
    float* h_obs = nullptr;
    uint64_t seed = 0;
    int64_t obs_floats = 0;
    int64_t t_submit = 0, t_done = 0;
    bool failed = false;
};

constexpr size_t kUpHead = 16;             // work counters at the head of a tick's upload
static_assert(kFusedCounters * sizeof(int) <= kUpHead, "counters fit the upload head");

struct Tick {
    cudaStream_t st = nullptr;
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;
    // pinned host and device buffers, one copy each way per tick:
    // up   = [zeroed work counters (kUpHead bytes)][entries][actions]
    // down = [rewards][done flags][observations, 16-byte aligned]
    unsigned char *h_up = nullptr, *d_up = nullptr;
    unsigned char *h_down = nullptr, *d_down = nullptr;
    int4 *h_entries = nullptr, *d_entries = nullptr;   // up + kUpHead
    int* d_counter = nullptr;                          // d_up
    float* h_rew = nullptr;                            // this tick's outputs inside h_down
    uint8_t* h_done = nullptr;
    float* h_obs = nullptr;
    int32_t *h_rslots = nullptr, *d_rslots = nullptr;
    unsigned long long *h_rseeds = nullptr, *d_rseeds = nullptr;
    std::vector<uint32_t> recs;             // request records in this tick
    std::vector<int64_t> rew_off, obs_off;  // per record: where its outputs start in the tick buffers
    bool busy = false;
    bool failed = false;
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
    // per slot, one 8-byte record so that a request touches one cache line
    // per station: admitted flag, size class, charger count, queued or
    // in-flight requests (the last three under the server lock)
    struct SlotInfo {
        uint8_t admitted, cls;
        uint16_t nports;
        int32_t refs;
    };
    std::vector<SlotInfo> slot;
    // stations of ticks on the device; set only by the scheduler (which reads
    // it without the lock: a stale 1 merely delays a request to the next scan)
    // and cleared by the completer
    std::unique_ptr<std::atomic<uint8_t>[]> in_flight;
    std::vector<uint32_t> scan_mark;       // submit: duplicate check (under the lock)
    uint32_t scan_gen = 0;
    std::vector<uint32_t> sched_mark;      // scheduler: stations claimed by waiting requests
    uint32_t sched_gen = 0;
    double used_bytes = 0.0;
    int n_resident = 0;
    cudaStream_t admin = nullptr;

    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_complete;
    std::deque<uint32_t> pending;          // queued request records, arrival order
    std::vector<Request> table;
    uint64_t req_mask = 0;
    uint64_t next_ticket = 1;
    uint64_t events = 0;                   // submissions + completions (wakes a blocked scheduler)
    std::vector<Tick> ticks;
    std::deque<int> launched;              // tick indices in launch order
    std::thread sched_thread, done_thread;
    bool stopping = false;
    int max_tick_envs = 0;
    int64_t max_tick_obs = 0;
    int64_t max_tick_act = 0;
    // statistics
    uint64_t n_ticks = 0, n_requests = 0, n_env_steps = 0, n_resets = 0;
    double busy_ms = 0.0;
    int64_t t_start = 0;
    std::atomic<int64_t> ns_submit{0}, ns_scan{0}, ns_pack{0}, ns_launch{0}, ns_complete{0}, n_scans{0};
    int threads = 256;
};

namespace {

uint32_t next_scan(chx_srv* s)
{
    ++s->scan_gen;
    if (s->scan_gen == 0) {
        std::fill(s->scan_mark.begin(), s->scan_mark.end(), 0u);
        s->scan_gen = 1;
    }
    return s->scan_gen;
}

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
    s->slot.assign(NS, chx_srv::SlotInfo{0, 0, 0, 0});
    for (int c = 0; c < kNumClasses; ++c)
        for (int i = 0; i < b.cls_n_env[c]; ++i) s->slot[b.cls_env_base[c] + i].cls = (uint8_t)c;
    s->in_flight.reset(new std::atomic<uint8_t>[NS]());
    s->scan_mark.assign(NS, 0);
    s->sched_mark.assign(NS, 0);
    for (int c = 0; c < kNumClasses; ++c) {
        s->free_slots[c].clear();
        for (int i = s->cap[c] - 1; i >= 0; --i) s->free_slots[c].push_back(b.cls_env_base[c] + i);
    }
    return CHX_OK;
}

int alloc_tick(chx_srv* s, Tick& t)
{
    const size_t ne = (size_t)s->max_tick_envs + 4 * kNumClasses;
    const size_t na = (size_t)std::max<int64_t>(s->max_tick_act, 1);
    const size_t no = (size_t)std::max<int64_t>(s->max_tick_obs, 1);
    SRV_TRY(cudaStreamCreateWithFlags(&t.st, cudaStreamNonBlocking));
    SRV_TRY(cudaEventCreate(&t.ev_start));
    SRV_TRY(cudaEventCreate(&t.ev_end));
    const size_t up = kUpHead + ne * sizeof(int4) + na;
    const size_t down = ((ne * 5 + 15) & ~size_t(15)) + no * sizeof(float);
    SRV_TRY(cudaHostAlloc(&t.h_up, up, cudaHostAllocDefault));
    SRV_TRY(cudaHostAlloc(&t.h_down, down, cudaHostAllocDefault));
    SRV_TRY(cudaHostAlloc(&t.h_rslots, ne * sizeof(int32_t), cudaHostAllocDefault));
    SRV_TRY(cudaHostAlloc(&t.h_rseeds, ne * sizeof(unsigned long long), cudaHostAllocDefault));
    SRV_TRY(cudaMalloc(&t.d_up, up));
    SRV_TRY(cudaMalloc(&t.d_down, down));
    SRV_TRY(cudaMalloc(&t.d_rslots, ne * sizeof(int32_t)));
    SRV_TRY(cudaMalloc(&t.d_rseeds, ne * sizeof(unsigned long long)));
    std::memset(t.h_up, 0, kUpHead);       // the counters every tick uploads as zero
    t.h_entries = reinterpret_cast<int4*>(t.h_up + kUpHead);
    t.d_entries = reinterpret_cast<int4*>(t.d_up + kUpHead);
    t.d_counter = reinterpret_cast<int*>(t.d_up);
    return CHX_OK;
}

void free_tick(Tick& t)
{
    if (t.st) cudaStreamSynchronize(t.st);
    cudaFreeHost(t.h_up); cudaFreeHost(t.h_down); cudaFreeHost(t.h_rslots); cudaFreeHost(t.h_rseeds);
    cudaFree(t.d_up); cudaFree(t.d_down); cudaFree(t.d_rslots); cudaFree(t.d_rseeds);
    if (t.ev_start) cudaEventDestroy(t.ev_start);
    if (t.ev_end) cudaEventDestroy(t.ev_end);
    if (t.st) cudaStreamDestroy(t.st);
    t = Tick{};
}

inline int class_of_slot_host(const chx_srv* s, int slot) { return s->slot[slot].cls; }

// Pack and launch one tick on ticks[ti] with the requests the scheduler chose.
// Runs without the server lock (the requests and their stations are reserved).
int launch_tick(chx_srv* s, int ti, const std::vector<Request*>& rq)
{
    Tick& t = s->ticks[ti];
    const int64_t t_p0 = now_ns();
    // pass 1: stations per class, output and observation offsets per request
    int count[kNumClasses] = {};
    int n_reset = 0;
    int64_t act_used = 0, rew_used = 0, obs_used = 0;
    t.rew_off.assign(rq.size(), 0);
    t.obs_off.assign(rq.size(), 0);
    for (size_t r = 0; r < rq.size(); ++r) {
        Request& q = *rq[r];
        if (q.kind == CHX_SRV_RESET) {
            for (int32_t e : q.envs) {
                t.h_rslots[n_reset] = e;
                t.h_rseeds[n_reset] = (unsigned long long)q.seed;
                ++n_reset;
            }
            continue;
        }
        t.rew_off[r] = rew_used;
        t.obs_off[r] = obs_used;
        for (int32_t e : q.envs) count[s->slot[e].cls] += 1;
        rew_used += (int64_t)q.envs.size();
        if (q.h_obs) obs_used += q.obs_floats;
    }
    // schedule: largest class first, each class padded to whole tiles
    FusedIO io{};
    int cursor[kNumClasses] = {};
    int n_entries = 0, tb = 0;
    io.n_sched = 0;
    for (int c = kNumClasses - 1; c >= 0; --c) {
        if (count[c] == 0) continue;
        const int epw = tile_epw(c);
        const int padded = (count[c] + epw - 1) / epw * epw;
        io.gather_base[c] = n_entries;
        cursor[c] = n_entries;
        for (int i = count[c]; i < padded; ++i) t.h_entries[n_entries + i] = make_int4(s->pad_slot[c], 0, 0, 0);
        n_entries += padded;
        io.sched_cls[io.n_sched] = c;
        io.sched_tile_base[io.n_sched] = tb;
        io.n_sched++;
        tb += padded / epw;
    }
    io.sched_tile_base[io.n_sched] = tb;
    io.total_tiles = tb;
    // actions right after the used entries (one upload); outputs packed
    int8_t* h_act = reinterpret_cast<int8_t*>(t.h_up + kUpHead + (size_t)n_entries * sizeof(int4));
    int8_t* d_act = reinterpret_cast<int8_t*>(t.d_up + kUpHead + (size_t)n_entries * sizeof(int4));
    const size_t done_at = (size_t)rew_used * sizeof(float);
    const size_t obs_at = ((size_t)rew_used * 5 + 15) & ~size_t(15);
    t.h_rew = reinterpret_cast<float*>(t.h_down);
    t.h_done = t.h_down + done_at;
    t.h_obs = reinterpret_cast<float*>(t.h_down + obs_at);
    // pass 2: entries straight into the pinned buffer, actions concatenated
    for (size_t r = 0; r < rq.size(); ++r) {
        Request& q = *rq[r];
        if (q.kind == CHX_SRV_RESET) continue;
        int64_t act_base = -1;
        if (!q.actions.empty()) {
            std::memcpy(h_act + act_used, q.actions.data(), q.actions.size());
            act_base = act_used;
            act_used += (int64_t)q.actions.size();
        }
        int64_t obs_pos = t.obs_off[r];
        const int out0 = (int)t.rew_off[r];
        for (size_t j = 0; j < q.envs.size(); ++j) {
            const int slot = q.envs[j];
            const int c = s->slot[slot].cls;
            const int ao = act_base >= 0 ? (int)(act_base + q.act_off[j]) : 0;
            t.h_entries[cursor[c]++] = make_int4(slot, ao, out0 + (int)j, (int)obs_pos);
            if (q.h_obs) obs_pos += 8 + 6 * (int64_t)(q.act_off[j + 1] - q.act_off[j]);
        }
    }
    io.k_steps = 1;
    // a tick is either all Philox actions or all given actions (the scheduler
    // never mixes them), so io.actions applies to every entry
    io.actions = act_used > 0 ? d_act : nullptr;
    io.lda = 1;
    io.lda_step = 1;
    io.reward = reinterpret_cast<float*>(t.d_down);
    io.done = t.d_down + done_at;
    io.ld_out = 1;
    io.ld_step = 1;
    io.obs = obs_used > 0 ? reinterpret_cast<float*>(t.d_down + obs_at) : nullptr;
    io.counter = t.d_counter;
    io.gather = t.d_entries;
    s->ns_pack += now_ns() - t_p0;
    cudaStream_t st = t.st;
    SRV_TRY(cudaEventRecord(t.ev_start, st));
    if (n_reset > 0) {
        SRV_TRY(cudaMemcpyAsync(t.d_rslots, t.h_rslots, n_reset * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        SRV_TRY(cudaMemcpyAsync(t.d_rseeds, t.h_rseeds, n_reset * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                                st));
        launch_reset_slots(s->b, s->dp, t.d_rslots, t.d_rseeds, n_reset, st);
        SRV_TRY(cudaGetLastError());
    }
    if (tb > 0) {
        SRV_TRY(cudaMemcpyAsync(t.d_up, t.h_up, kUpHead + (size_t)n_entries * sizeof(int4) + (size_t)act_used,
                                cudaMemcpyHostToDevice, st));
        launch_step_fused(s->b, s->dp, io, s->threads, s->sm_count, st);
        SRV_TRY(cudaGetLastError());
        const size_t down = obs_used > 0 ? obs_at + (size_t)obs_used * sizeof(float) : done_at + (size_t)rew_used;
        SRV_TRY(cudaMemcpyAsync(t.h_down, t.d_down, down, cudaMemcpyDeviceToHost, st));
    }
    SRV_TRY(cudaEventRecord(t.ev_end, st));
    return CHX_OK;
}

void scheduler(chx_srv* s)
{
    cudaSetDevice(s->device);
    std::vector<Request*> rq;
    std::deque<uint32_t> work, rest;
    uint64_t seen = ~0ULL;                 // events counter when nothing could be scheduled
    for (;;) {
        int ti = -1;
        uint64_t events_at_take = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_sched.wait(lk, [&] {
                if (s->stopping) return true;
                if (s->pending.empty() || s->events == seen) return false;
                for (auto& t : s->ticks)
                    if (!t.busy) return true;
                return false;
            });
            if (s->stopping) return;
            for (size_t i = 0; i < s->ticks.size(); ++i)
                if (!s->ticks[i].busy) {
                    ti = (int)i;
                    break;
                }
            s->ticks[ti].busy = true;
            work.swap(s->pending);         // take the queue; submissions continue meanwhile
            events_at_take = s->events;
        }
        // pack in arrival order outside the lock; a request waits if one of its
        // stations is in flight or claimed by an earlier waiting request
        const int64_t t_scan0 = now_ns();
        Tick& t = s->ticks[ti];
        if (++s->sched_gen == 0) {
            std::fill(s->sched_mark.begin(), s->sched_mark.end(), 0u);
            s->sched_gen = 1;
        }
        const uint32_t gen = s->sched_gen;
        rq.clear();
        t.recs.clear();
        rest.clear();
        int envs = 0;
        int64_t act = 0, obs = 0;
        int with_actions = -1;             // a tick is all-Philox or all-given actions
        bool full = false;
        for (uint32_t ri : work) {
            Request& q = s->table[ri];
            if (full) {
                rest.push_back(ri);
                continue;
            }
            bool blocked = false;
            for (int32_t e : q.envs)
                if (s->in_flight[e].load(std::memory_order_relaxed) || s->sched_mark[e] == gen) {
                    blocked = true;
                    break;
                }
            const int wa = q.kind == CHX_SRV_STEP ? (q.actions.empty() ? 0 : 1) : -1;
            const bool fits = envs + (int)q.envs.size() <= s->max_tick_envs &&
                              act + (int64_t)q.actions.size() <= s->max_tick_act &&
                              obs + q.obs_floats <= s->max_tick_obs &&
                              (wa < 0 || with_actions < 0 || wa == with_actions);
            if (blocked || !fits) {
                for (int32_t e : q.envs) s->sched_mark[e] = gen;
                rest.push_back(ri);
                full = !fits && envs >= s->max_tick_envs;
                continue;
            }
            if (wa >= 0) with_actions = wa;
            for (int32_t e : q.envs) s->in_flight[e].store(1, std::memory_order_relaxed);
            envs += (int)q.envs.size();
            act += (int64_t)q.actions.size();
            obs += q.obs_floats;
            rq.push_back(&q);
            t.recs.push_back(ri);
        }
        work.clear();
        s->ns_scan += now_ns() - t_scan0;
        s->n_scans += 1;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (!rest.empty()) {           // waiting requests stay ahead of newer ones
                rest.insert(rest.end(), s->pending.begin(), s->pending.end());
                s->pending.swap(rest);
            }
            if (rq.empty()) {              // everything waits on in-flight stations
                t.busy = false;
                seen = events_at_take;
                continue;
            }
            seen = ~0ULL;
        }
        const int64_t t_l0 = now_ns();
        t.failed = launch_tick(s, ti, rq) != CHX_OK;
        s->ns_launch += now_ns() - t_l0;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->launched.push_back(ti);
        }
        s->cv_complete.notify_one();
    }
}

void completer(chx_srv* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        int ti;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_complete.wait(lk, [&] { return s->stopping || !s->launched.empty(); });
            if (s->launched.empty()) return;   // stopping and drained
            ti = s->launched.front();
            s->launched.pop_front();
        }
        Tick& t = s->ticks[ti];
        float ms = 0.f;
        if (t.failed || cudaEventSynchronize(t.ev_end) != cudaSuccess ||
            cudaEventElapsedTime(&ms, t.ev_start, t.ev_end) != cudaSuccess) {
            t.failed = true;
            ms = 0.f;
        }
        const int64_t t_c0 = now_ns();
        // copy results to the requesters without the lock (records stay put and
        // are not released before they are marked done below)
        for (size_t r = 0; r < t.recs.size(); ++r) {
            Request* q = &s->table[t.recs[r]];
            if (q->kind != CHX_SRV_STEP || t.failed) continue;
            const size_t n = q->envs.size();
            if (q->h_reward) std::memcpy(q->h_reward, t.h_rew + t.rew_off[r], n * sizeof(float));
            if (q->h_done) std::memcpy(q->h_done, t.h_done + t.rew_off[r], n);
            if (q->h_obs) std::memcpy(q->h_obs, t.h_obs + t.obs_off[r], (size_t)q->obs_floats * sizeof(float));
        }
        const int64_t tn = now_ns();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (uint32_t ri : t.recs) {
                Request& q = s->table[ri];
                for (int32_t e : q.envs) {
                    s->in_flight[e].store(0, std::memory_order_relaxed);
                    s->slot[e].refs -= 1;
                }
                q.failed = t.failed;
                q.t_done = tn;
                q.state.store(kDone, std::memory_order_release);
                s->n_requests += 1;
                if (q.kind == CHX_SRV_STEP)
                    s->n_env_steps += q.envs.size();
                else
                    s->n_resets += q.envs.size();
            }
            s->n_ticks += 1;
            s->busy_ms += ms;
            s->events += 1;
            t.busy = false;
            t.recs.clear();
        }
        s->ns_complete += now_ns() - t_c0;
        s->cv_done.notify_all();
        s->cv_sched.notify_one();
    }
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
    if (cfg->max_tick_obs_floats < 0) return fail(CHX_EINVAL, "max_tick_obs_floats must be >= 0");
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
    s->max_tick_act = (int64_t)cfg->max_tick_envs * CHX_MAX_PORTS;
    s->max_tick_obs = cfg->max_tick_obs_floats;
    s->table = std::vector<Request>(kMaxOutstanding);
    s->req_mask = kMaxOutstanding - 1;
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
    s->ticks.resize(cfg->n_streams);
    for (auto& t : s->ticks)
        if ((rc = alloc_tick(s, t))) {
            chx_srv_stop(s);
            return rc;
        }
    if (cudaStreamCreateWithFlags(&s->admin, cudaStreamNonBlocking) != cudaSuccess) {
        chx_srv_stop(s);
        return fail(CHX_ECUDA, "stream creation failed");
    }
    s->t_start = now_ns();
    s->sched_thread = std::thread(scheduler, s);
    s->done_thread = std::thread(completer, s);
    *out = s;
    return CHX_OK;
}

extern "C" int chx_srv_stop(chx_srv* s)
{
    if (!s) return CHX_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_sched.notify_all();
    s->cv_complete.notify_all();
    if (s->sched_thread.joinable()) s->sched_thread.join();
    if (s->done_thread.joinable()) s->done_thread.join();
    cudaDeviceSynchronize();
    for (auto& t : s->ticks) free_tick(t);
    for (void* p : s->bufs) cudaFree(p);
    if (s->admin) cudaStreamDestroy(s->admin);
    delete s;
    return CHX_OK;
}

extern "C" int chx_srv_admit(chx_srv* s, const chx_stations* st, uint64_t seed, int32_t* h_ids)
{
    if (!s || !st || !h_ids) return fail(CHX_EINVAL, "null argument");
    if (st->h_n_upper) return fail(CHX_EINVAL, "the serving loop takes two-level trees (h_n_upper = NULL)");
    int rc = validate_stations(st, &s->cfg.exo, 1LL << 24);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(s->mu);
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
    std::lock_guard<std::mutex> lk(s->mu);
    for (int j = 0; j < n; ++j) {
        const int e = h_ids[j];
        if (e < 0 || e >= s->b.n_slots || !s->slot[e].admitted) return fail(CHX_EINVAL, "station id not admitted");
        if (s->slot[e].refs > 0) return fail(CHX_EINVAL, "station has queued or in-flight requests");
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
    if (r->kind != CHX_SRV_STEP && r->kind != CHX_SRV_RESET) return fail(CHX_EINVAL, "unknown request kind");
    if (r->n_envs < 1 || r->n_envs > s->max_tick_envs || !r->h_env_ids)
        return fail(CHX_EINVAL, "n_envs must be in 1..max_tick_envs");
    // copy the request's inputs before taking the lock
    thread_local std::vector<int32_t> envs;
    thread_local std::vector<int8_t> actions;
    envs.assign(r->h_env_ids, r->h_env_ids + r->n_envs);
    for (int32_t e : envs)
        if (e < 0 || e >= s->b.n_slots) return fail(CHX_EINVAL, "station id out of range");
    std::unique_lock<std::mutex> lk(s->mu);
    const int64_t t_in = now_ns();
    if (s->stopping) return fail(CHX_EINVAL, "server is stopping");
    const uint64_t tk = s->next_ticket;
    const uint32_t ri = (uint32_t)(tk & s->req_mask);
    Request& q = s->table[ri];
    if (q.state.load(std::memory_order_acquire) != kFree)
        return fail(CHX_ENOMEM, "too many outstanding requests: release tickets with chx_srv_wait or chx_srv_test");
    // check the stations (admitted, listed once) and their charger offsets
    const uint32_t gen = next_scan(s);
    q.act_off.resize(envs.size() + 1);
    q.act_off[0] = 0;
    for (size_t j = 0; j < envs.size(); ++j) {
        const int32_t e = envs[j];
        const chx_srv::SlotInfo& si = s->slot[e];
        if (!si.admitted) return fail(CHX_EINVAL, "station id not admitted");
        if (s->scan_mark[e] == gen) return fail(CHX_EINVAL, "station listed twice in one request");
        s->scan_mark[e] = gen;
        q.act_off[j + 1] = q.act_off[j] + si.nports;
    }
    int64_t obs_floats = 0;
    actions.clear();
    if (r->kind == CHX_SRV_STEP) {
        if (r->h_actions) {
            actions.assign(r->h_actions, r->h_actions + q.act_off.back());
            for (int8_t a : actions)
                if (a < 0 || a >= s->params.n_levels) return fail(CHX_EINVAL, "action level out of range");
        }
        if (r->h_obs) obs_floats = 8LL * (int64_t)envs.size() + 6LL * q.act_off.back();
        if (obs_floats > s->max_tick_obs) return fail(CHX_EINVAL, "observation larger than max_tick_obs_floats");
    }
    // the record is free: fill it, publish it last
    q.kind = r->kind;
    q.envs.swap(envs);
    q.actions.swap(actions);
    q.h_reward = r->h_reward;
    q.h_done = r->h_done;
    q.h_obs = r->kind == CHX_SRV_STEP ? r->h_obs : nullptr;
    q.seed = r->seed;
    q.failed = false;
    q.obs_floats = obs_floats;
    for (int32_t e : q.envs) s->slot[e].refs += 1;
    q.t_submit = now_ns();
    q.ticket.store(tk, std::memory_order_relaxed);
    q.state.store(kQueued, std::memory_order_release);
    s->next_ticket++;
    s->pending.push_back(ri);
    s->events += 1;
    *ticket = tk;
    s->ns_submit += now_ns() - t_in;
    lk.unlock();
    s->cv_sched.notify_one();
    return CHX_OK;
}

namespace {
// release a completed record; returns its status
int release(Request& q, int64_t* latency_ns)
{
    if (latency_ns) *latency_ns = q.t_done - q.t_submit;
    const bool failed = q.failed;
    q.state.store(kFree, std::memory_order_release);
    return failed ? fail(CHX_ECUDA, "the tick carrying this request failed on the device") : CHX_OK;
}
}  // namespace

extern "C" int chx_srv_wait(chx_srv* s, uint64_t ticket, int64_t timeout_us, int64_t* latency_ns)
{
    if (!s) return fail(CHX_EINVAL, "null server");
    Request& q = s->table[ticket & s->req_mask];
    if (q.ticket.load(std::memory_order_acquire) != ticket || q.state.load(std::memory_order_acquire) == kFree)
        return fail(CHX_EINVAL, "unknown ticket");
    if (q.state.load(std::memory_order_acquire) != kDone) {
        std::unique_lock<std::mutex> lk(s->mu);
        const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
        if (!s->cv_done.wait_until(lk, deadline, [&] { return q.state.load(std::memory_order_acquire) == kDone; }))
            return fail(CHX_ETIMEOUT, "request not finished within the timeout");
    }
    return release(q, latency_ns);
}

extern "C" int chx_srv_test(chx_srv* s, uint64_t ticket, int32_t* h_done, int64_t* latency_ns)
{
    if (!s || !h_done) return fail(CHX_EINVAL, "null argument");
    Request& q = s->table[ticket & s->req_mask];
    if (q.ticket.load(std::memory_order_acquire) != ticket) return fail(CHX_EINVAL, "unknown ticket");
    const int st = q.state.load(std::memory_order_acquire);
    if (st == kFree) return fail(CHX_EINVAL, "unknown ticket");
    *h_done = st == kDone ? 1 : 0;
    return st == kDone ? release(q, latency_ns) : CHX_OK;
}

extern "C" int chx_srv_stats(chx_srv* s, chx_srv_stats_t* out)
{
    if (!s || !out) return fail(CHX_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->n_ticks = (int64_t)s->n_ticks;
    out->n_requests = (int64_t)s->n_requests;
    out->env_steps = (int64_t)s->n_env_steps;
    out->env_resets = (int64_t)s->n_resets;
    out->resident = s->n_resident;
    out->used_bytes = s->used_bytes;
    out->budget_bytes = s->cfg.hbm_budget_bytes;
    out->device_busy_ms = s->busy_ms;
    out->elapsed_ms = (double)(now_ns() - s->t_start) * 1e-6;
    out->host_submit_ms = s->ns_submit.load() * 1e-6;
    out->host_scan_ms = s->ns_scan.load() * 1e-6;
    out->host_pack_ms = s->ns_pack.load() * 1e-6;
    out->host_launch_ms = s->ns_launch.load() * 1e-6;
    out->host_complete_ms = s->ns_complete.load() * 1e-6;
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
                        err = 1;
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
                    if (chx_srv_submit(s, &r, &x.ticket)) {
                        err = 2;
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
    if (err.load()) return fail(CHX_EINVAL, "a simulated actor's call failed");
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
