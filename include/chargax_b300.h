/*
 * chargax_b300.h -- C interface of the B300 (sm_103a) EV charging-station
 * simulator: a batch of independent stations stepped on one GPU.
 *
 * The operations follow the environment of "Chargax: A JAX Accelerated EV
 * Charging Simulator" (arXiv 2507.01522):
 *   - station layout: a tree whose root is the grid connection, inner nodes
 *     are groups (splitters/cables) with a power limit I_H and efficiency
 *     eta_H, and leaves are the chargers (Sec. "EV Station Layout");
 *     root -> groups -> chargers by default, with up to three levels of
 *     upper nodes between the root and the groups (Fig. c trees, see
 *     chx_stations.h_n_upper): trees of depth up to five;
 *   - transition, Appendix A.2, in order: apply actions (per-charger clip),
 *     architecture constraint Eq. (ArchConst) by proportional rescaling,
 *     charge stationed cars with the SoC taper of Appendix A.1, time advance,
 *     departure of time-sensitive users, Poisson arrivals parked first come
 *     first served;
 *   - reward, Appendix A.3: profit minus alpha-weighted penalties
 *     (missing energy at departure, rejected cars, constraint violation);
 *   - exploring-starts reset (Appendix "Practical Considerations"): an
 *     empty station at step-of-day 0 and a random day of the price bank.
 *
 * Conventions
 *   - Every function returns CHX_OK (0) or a negative status; no exception
 *     crosses the interface.  chx_last_error() gives the message of the last
 *     failure on the calling thread.
 *   - Pointer names: d_* are device pointers (memory of the handle's GPU),
 *     h_* are host pointers.  Unprefixed array pointers follow the rule
 *     stated at the function.
 *   - "Batch order": envs are numbered 0..n_envs-1 as passed to chx_create;
 *     per-charger arrays are CSR by station (charger q of env e is element
 *     port_off[e] + q, port_off = exclusive prefix sum of n_ports).
 *   - Calls that take a stream are asynchronous on it (cudaStream_t passed as
 *     void*; NULL = legacy default stream).  Buffers must stay valid until the
 *     stream reaches the call.  A handle must not be used from two threads at
 *     once.
 *   - Units: power kW, energy kWh, time in steps of dt_h hours, prices EUR/kWh.
 */
#ifndef CHARGAX_B300_H
#define CHARGAX_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define CHX_OK 0
#define CHX_EINVAL (-1)   /* bad argument or configuration                    */
#define CHX_ENOMEM (-2)   /* device or host allocation failed / over budget   */
#define CHX_ECUDA (-3)    /* a CUDA call failed                               */
#define CHX_ETIMEOUT (-4) /* a wait ran out of time                           */
#define CHX_EFAULT (-5)   /* a kernel flagged bad input (e.g. action level out of range) */

#define CHX_MAX_PORTS 128   /* chargers per station                          */
#define CHX_MAX_UPPER_DEPTH 3   /* levels of tree nodes above the groups     */
#define CHX_MAX_GROUPS 32   /* group nodes per station                       */
#define CHX_MAX_STAY 255    /* longest stay in steps                         */

/* ---- configuration ----------------------------------------------------- */

/* Scalar environment parameters (Table "ppo-config" and the car/user
 * profile distributions of Appendix A.1).  Charger type 0 = AC, 1 = DC. */
typedef struct chx_env_params {
    int32_t ep_len;          /* steps per episode (288 = 24 h of 5 min)        */
    int32_t n_levels;        /* action levels: k in 0..n_levels-1 requests
                                k/(n_levels-1) of the charger maximum          */
    float dt_h;              /* step length in hours                          */
    float tau;               /* SoC where the taper starts, (0,1)             */
    float p_sell;            /* price charged to customers                    */
    float c_fixed;           /* fixed cost per step                           */
    float alpha_sat;         /* weight of missing kWh at departure            */
    float alpha_decl;        /* weight of rejected cars                       */
    float alpha_con;         /* weight of the constraint-violation penalty    */
    float soc_target;        /* SoC users want: Delta E = (target - SoC0) C   */
    float p_max_kw[2];       /* charger maximum power per type                */
    float eta_port[2];       /* charger efficiency per type, (0,1]            */
    float cap_kwh[2];        /* car capacity ~ U(lo, hi)                      */
    float soc0[2];           /* arrival SoC ~ U(lo, hi)                       */
    int32_t stay_steps[2];   /* stay ~ U{lo..hi} steps, 1 <= lo <= hi <= 255  */
    float rbar_kw[2][2];     /* car maximum rate ~ U(lo, hi) per charger type */
    /* Vehicle-to-grid mode (App. A.1 "Endogenous state space", A.2 "Apply
     * Actions", A.3): v2g = 1 makes the action levels signed -- level k in
     * 0..n_levels-1 (n_levels odd) requests (k - h)/h of the charger maximum,
     * h = (n_levels-1)/2, negative = discharge along the charging curve
     * flipped at SoC = 0.5 -- and adds one station battery per station
     * (capacity, maximum rate, taper point, SoC at each episode start) with
     * its own action level after the chargers', at the root of the station's
     * tree.  Energy sold back to the grid earns sell_grid_ratio x the buy
     * price; discharged energy (cars and battery) costs alpha_degrad per
     * kWh.  v2g = 0 ignores the remaining fields. */
    int32_t v2g;
    float sell_grid_ratio;
    float alpha_degrad;
    float batt_cap_kwh;
    float batt_rate_kw;
    float batt_tau;
    float batt_soc0;
    /* Action form (A.2 "Apply Actions"): action_delta = 0 takes the level as
     * an absolute request (above); action_delta = 1 takes it as an increment
     * of the charger's last applied power, the Delta-current form: level k
     * (n_levels odd, h = (n_levels-1)/2) requests last + (k - h)/h x the
     * charger maximum, clipped as above (at 0 from below without V2G).  In
     * this form a departing car's charger drops to 0 power, so the next car
     * starts from 0.  The battery's level is an increment of its last power
     * alike. */
    int32_t action_delta;
    /* Discharge maximum I_max<- per charger type, > 0 (V2G mode; the
     * discharge branch of the clip caps at it instead of p_max_kw). */
    float p_max_dis_kw[2];
    /* Charge-sensitive users (A.1 User Profiles, u = 1; A.2 "Departure of
     * Cars"; A.3 c_Sat,1): an arriving car's user is charge-sensitive iff
     * the low byte of the first word of its profile draw is below
     * cs_share_256 (0 = none, 256 = all).  Such a car occupies its charger
     * with trem = CHX_TREM_CS and counts its steps to the desired departure
     * (Delta t_remain, negative once overdue) in a separate per-charger
     * array (chx_get_due); it leaves once its demand is met, i.e. at most
     * eps_cap x its car's capacity remains (the target SoC reached within
     * eps_cap), costing alpha_sat1 x (steps overdue - beta_early x steps
     * early).  cs_share_256 > 0 needs stay_steps[1] <= 254, and adds a 7th
     * per-charger observation feature (u).  0 ignores the other fields. */
    int32_t cs_share_256;
    float alpha_sat1;
    float beta_early;
    float eps_cap;
} chx_env_params;

#define CHX_TREM_CS 255     /* trem of a charger holding a charge-sensitive car */

/* A batch of stations, CSR.  Groups of a station are contiguous charger
 * ranges listed in charger order.  All pointers are host pointers, read only
 * during chx_create. */
typedef struct chx_stations {
    int32_t n_envs;
    const int32_t* h_n_ports;        /* [n_envs], 1..CHX_MAX_PORTS            */
    const uint8_t* h_port_type;      /* [sum n_ports], 0 AC / 1 DC            */
    const int32_t* h_n_groups;       /* [n_envs], 1..min(n_ports, 32)         */
    const int32_t* h_group_size;     /* [sum n_groups], >= 1, sums to n_ports */
    const float* h_group_limit_kw;   /* [sum n_groups] I_H of the group, > 0  */
    const float* h_group_eta;        /* [sum n_groups] eta_H in (0,1], or NULL = 1 */
    const float* h_grid_limit_kw;    /* [n_envs] root limit, > 0              */
    const float* h_grid_eta;         /* [n_envs] or NULL = 1                  */
    const int32_t* h_arrival_class;  /* [n_envs] row of the arrival table     */
    /* Deeper trees (Fig. charge-tree c), optional; NULL h_n_upper: every
     * group hangs from the root.  Station e has h_n_upper[e] nodes above its
     * groups (listed per station, in station order); parents are
     * station-local upper-node indices, -1 = the root.  Eq. (ArchConst)
     * holds at every node, (1/eta_H) sum <= I_H, enforced bottom-up by
     * proportional rescaling (deeper nodes first).  Every upper node has at
     * least one group below it, the groups below a node are consecutive,
     * and upper nodes lie at most CHX_MAX_UPPER_DEPTH levels deep
     * (CHX_EINVAL otherwise). */
    const int32_t* h_n_upper;        /* [n_envs] 0..CHX_MAX_GROUPS            */
    const int32_t* h_group_parent;   /* [sum n_groups] parent of each group   */
    const int32_t* h_upper_parent;   /* [sum n_upper] parent of each node     */
    const float* h_upper_limit_kw;   /* [sum n_upper] I_H > 0                 */
    const float* h_upper_eta;        /* [sum n_upper] in (0,1], or NULL = 1   */
} chx_stations;

/* Exogenous tables (host pointers, copied to the device by chx_create). */
typedef struct chx_exo {
    int32_t n_days;                  /* rows of the price bank, >= 1          */
    const float* h_price;            /* [n_days][ep_len] buy price            */
    int32_t n_arrival_classes;       /* rows of the arrival table, >= 1       */
    const float* h_arrival_rate;     /* [n_classes][ep_len] mean cars/step, 0..64 */
} chx_exo;

typedef struct chx_handle chx_handle;

/* ---- lifetime ---------------------------------------------------------- */

/* Create a batch on the current CUDA device and reset every env with `seed`
 * (per-env Philox key = seed; stream id = env index).  The library allocates
 * and owns all env state on the device.  Blocks until the state is ready.
 * Errors: CHX_EINVAL for a configuration outside the documented ranges,
 * CHX_ENOMEM, CHX_ECUDA. */
int chx_create(const chx_stations* st, const chx_env_params* params, const chx_exo* exo,
               uint64_t seed, chx_handle** out);
int chx_destroy(chx_handle* h);

/* Message of the last failed call on this thread (static storage). */
const char* chx_last_error(void);

int chx_n_envs(const chx_handle* h, int32_t* out);
int chx_n_ports_total(const chx_handle* h, int64_t* out);
/* h_offsets[n_envs+1]: charger offsets in batch order. */
int chx_port_offsets(const chx_handle* h, int64_t* h_offsets);
/* Floats of one observation of the whole batch: 8 per env (10 in V2G mode)
 * + 6 per charger. */
int chx_obs_size(const chx_handle* h, int64_t* out);

/* ---- reset, Appendix "Practical Considerations" ---------------------------
 * Start a new episode for the listed envs (d_env_ids: device int32 [n] in
 * batch numbering; NULL = all envs): Philox key := seed, global step := 0,
 * every charger empty, step of day 0, day drawn from the price bank.
 * Statistics are kept.  CHX_EINVAL for n < 0; n = 0 with a list does
 * nothing.  A listed id outside 0..n_envs-1 is skipped (the others are
 * reset) and makes the next chx_check return CHX_EFAULT. */
int chx_reset(chx_handle* h, const int32_t* d_env_ids, int32_t n, uint64_t seed, void* stream);

/* ---- one step, plain form ------------------------------------------------
 * One transition of every env, one kernel launch, one thread per env, state
 * read from and written back to device memory.
 *   d_actions: device int8, level of charger (port_off[e]+q) at element
 *              (port_off[e]+q)*lda; NULL = uniform levels drawn in the kernel
 *              with Philox (counter: env, step/8, charger, 2; 16-bit half of a
 *              word).  Levels outside 0..n_levels-1 are clamped and flag
 *              CHX_EFAULT at the next chx_check.  V2G mode: every env has
 *              n_ports + 1 actions, its chargers' then its battery's, so
 *              charger q of env e is element (port_off[e]+e+q)*lda and the
 *              battery element (port_off[e+1]+e)*lda; a drawn battery level
 *              uses charger index n_ports in the Philox counter.
 *   d_reward:  device float [n_envs]; d_done: device uint8 [n_envs] (1 when
 *              the episode ended in this step; the env is already reset).
 * Either output may be NULL. */
int chx_step(chx_handle* h, const int8_t* d_actions, int64_t lda, float* d_reward, uint8_t* d_done,
             void* stream);

/* ---- K steps, fused form -------------------------------------------------
 * k_steps transitions of every env in ONE launch of a persistent kernel:
 * each warp owns a tile of stations of one size class, keeps their state in
 * registers across the k steps and reduces over chargers with warp shuffles.
 * Events (arrivals, departures, episode ends) are identical to k calls of
 * chx_step with the same actions; floating-point results agree to rounding
 * (the sums over chargers associate differently).
 *   d_actions: NULL (Philox levels) or device int8 with the level of charger
 *              i at step k at element i*lda + k (lda >= k_steps).
 *   d_reward / d_done: element e*ld_out + k for env e, step k (ld_out >=
 *              k_steps); either may be NULL.
 *   d_obs:     NULL or device float [chx_obs_size]: the observation after the
 *              last step.
 * Launch shape (warps per block) comes from chx_autotune, or a default. */
int chx_step_n(chx_handle* h, int32_t k_steps, const int8_t* d_actions, int64_t lda,
               float* d_reward, uint8_t* d_done, int64_t ld_out, float* d_obs, void* stream);

/* ---- rollout -------------------------------------------------------------
 * n_steps transitions with Philox actions as a CUDA graph of fused launches
 * (steps per launch and warps per block (1..8) from chx_autotune; captured on the
 * first call and re-used while n_steps and the output pointers are the same).
 * Outputs as chx_step_n with ld_out = n_steps; d_obs after the last step. */
int chx_rollout(chx_handle* h, int32_t n_steps, float* d_reward, uint8_t* d_done, float* d_obs,
                void* stream);

/* chx_rollout with HOST outputs, step-major: h_reward[k*n_envs + e] and
 * h_done[k*n_envs + e] for step k of env e ([n_steps][n_envs], a rollout
 * buffer's layout), h_obs as chx_rollout (any may be NULL; pinned memory
 * gives full copy bandwidth).  The steps run in up to 4 launches of
 * shrinking size (5:4:2:1 shares) whose outputs are copied while the next
 * launch computes; the call returns when everything is on the host. */
int chx_rollout_host(chx_handle* h, int32_t n_steps, float* h_reward, uint8_t* h_done, float* h_obs,
                     void* stream);

/* chx_rollout_host with the levels of every step given by the host: the Gym
 * loop of an actor that chose its actions on the host (Appendix "Practical
 * Considerations": one action per charger, plus the battery's in V2G mode).
 * h_actions is step-major, h_actions[k * n_act + q] for action slot q of
 * step k, n_act = total chargers (+ n_envs in V2G mode), each station's
 * slots in batch order (its chargers, then its battery); levels outside
 * 0..n_levels-1 are clamped and flagged (chx_check).  Outputs as
 * chx_rollout_host.  The steps run in up to 12 fused launches, each 0.85 of
 * the size of the one before (the copy in bounds the call, so the launches
 * left after it are short): the levels of launch c are copied in while
 * launch c - 1 computes and
 * its rewards and done flags are copied out while launch c + 1 computes
 * (pinned host memory gives full copy bandwidth); the observation follows
 * the last launch.  The call returns when everything is on the host.
 * h_actions NULL: CHX_EINVAL. */
int chx_rollout_host_actions(chx_handle* h, int32_t n_steps, const int8_t* h_actions, float* h_reward,
                             uint8_t* h_done, float* h_obs, void* stream);
/* chx_rollout_host_actions with the levels packed two per byte (the copy in
 * is half as large, and it is the part that bounds the call): step k's levels
 * take ceil(n_act / 2) bytes starting at byte k * ceil(n_act / 2); slot q is
 * the low nibble of byte q / 2 for even q, the high nibble for odd q.  Needs
 * n_levels <= 16 (else CHX_EINVAL); nibbles of n_levels or more are clamped
 * and flagged (chx_check).  The launches are of near-equal size (this copy
 * in takes about as long as the compute).  Results equal
 * chx_rollout_host_actions' on the same levels. */
int chx_rollout_host_levels4(chx_handle* h, int32_t n_steps, const uint8_t* h_levels4, float* h_reward,
                             uint8_t* h_done, float* h_obs, void* stream);

/* One plain step with HOST buffers: actions are copied in (h_actions NULL =
 * Philox levels), reward/done/observation copied out; returns when done. */
int chx_step_host(chx_handle* h, const int8_t* h_actions, float* h_reward, uint8_t* h_done,
                  float* h_obs, void* stream);

/* ---- rollout without allocation --------------------------------------------
 * (No counterpart in the paper: an interface for callers that cannot allocate
 * device memory while they step the simulator -- code running under a memory
 * pool it does not own, latency-critical loops that must not enter the
 * driver's allocator, or hosts that reserve all device memory up front.)
 * Same transitions and outputs as chx_rollout (Philox actions, fused launches
 * of the handle's steps per launch and warps per block), launched directly
 * without a CUDA graph.  The call allocates nothing: its only scratch, the
 * work counters of each launch (three per launch), lives in a 12 KB static
 * device array that every GPU loading this library keeps until the process
 * exits.  n_steps may need at most that many launches
 * (ceil(n_steps / steps per launch)); more returns CHX_EINVAL.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it; make that first call before any
 *     stream capture.  The cached address is valid until the device's
 *     context is reset (cudaDeviceReset); do not call the library after that.
 *   - The handle's device must be the current device (else CHX_EINVAL).
 *   - The 128-charger class runs beside the smaller classes on the handle's
 *     side stream, as in chx_rollout (that stream and its two events are
 *     created with the handle, not by this call).
 *   - All calls share the array.  Each call clears the counters it uses on
 *     `stream` first; calls that overlap on the GPU (other streams, other
 *     handles on the same device) race on the counters and must be ordered
 *     by the caller. */
#define CHX_NOALLOC_MAX_LAUNCHES 1024
int chx_rollout_noalloc(chx_handle* h, int32_t n_steps, float* d_reward, uint8_t* d_done, float* d_obs,
                        void* stream);

/* Choose steps per launch and warps per block for chx_rollout by timing
 * candidate shapes on a copy of the state (the state is restored).  Blocks.
 * h_steps_per_launch / h_warps_per_block receive the choice (may be NULL). */
int chx_autotune(chx_handle* h, int32_t n_steps, int32_t* h_steps_per_launch, int32_t* h_warps_per_block);
/* Set the launch shape by hand (0 keeps the current value). */
int chx_set_launch(chx_handle* h, int32_t steps_per_launch, int32_t warps_per_block);

/* ---- observation -----------------------------------------------------------
 * d_obs: device float [chx_obs_size].  Env e's block starts at float
 * 8*e + 6*port_off[e]: [sin, cos of time of day, buy price now, p_sell,
 * occupied fraction, day/n_days, step/ep_len, weekday flag] (V2G mode: then
 * battery SoC and battery power / batt_rate_kw; the station block is 10
 * floats and starts at 10*e + 6*port_off[e]), then per charger
 * [occupied, SoC, remaining stay/stay_hi, r_hat/P_max, last power/P_max,
 * remaining demand/cap_hi]. */
int chx_observe(chx_handle* h, float* d_obs, void* stream);

/* ---- state, checkpoint, statistics ------------------------------------------
 * Host arrays in batch order (all blocking).  Per charger [P]: SoC, remaining
 * demand kWh, capacity kWh, car maximum rate kW, last applied power kW,
 * remaining stay (0 = empty).  Per env [E]: step of day, day, global step,
 * cars admitted since the last reset (indexes the cars' Philox draws),
 * Philox key words, running episode return.  NULL skips a field on get and
 * keeps it on set. */
int chx_get_state(chx_handle* h, float* h_soc, float* h_erem, float* h_cap, float* h_rbar, float* h_p,
                  uint8_t* h_trem, int32_t* h_tod, int32_t* h_day, uint32_t* h_gstep, uint32_t* h_ncar,
                  uint32_t* h_key0, uint32_t* h_key1, float* h_ep_ret);
int chx_set_state(chx_handle* h, const float* h_soc, const float* h_erem, const float* h_cap,
                  const float* h_rbar, const float* h_p, const uint8_t* h_trem, const int32_t* h_tod,
                  const int32_t* h_day, const uint32_t* h_gstep, const uint32_t* h_ncar,
                  const uint32_t* h_key0, const uint32_t* h_key1, const float* h_ep_ret);

/* Station battery per env [E] (V2G mode; zeros otherwise): SoC and last
 * applied power kW.  chx_set_battery: CHX_EINVAL for a SoC outside [0,1];
 * NULL keeps a field.  Blocking. */
int chx_get_battery(chx_handle* h, float* h_soc, float* h_p);
int chx_set_battery(chx_handle* h, const float* h_soc, const float* h_p);

/* Delta t_remain of charge-sensitive cars (A.1 User Profiles, u = 1): per
 * charger in batch order (the order of chx_get_state), int16 steps to the
 * desired departure, negative once overdue; meaningful where trem is
 * CHX_TREM_CS, 0 elsewhere.  Host arrays of [total chargers]; NULL skips.
 * Both synchronise the device.  Without charge-sensitive users the values
 * are unused. */
int chx_get_due(chx_handle* h, int16_t* h_due);
int chx_set_due(chx_handle* h, const int16_t* h_due);

/* Per-env running statistics [E]: cars admitted, cars rejected, kWh missing
 * at departure, kWh charged, finished episodes, return of the last episode. */
int chx_stats(chx_handle* h, uint32_t* h_arrived, uint32_t* h_rejected, float* h_missing_kwh,
              float* h_charged_kwh, uint32_t* h_episodes, float* h_last_return);

/* Checkpoint: the full env state (state + statistics) as a byte blob.
 * chx_save with h_buf NULL writes the needed size to *size. */
int chx_save(chx_handle* h, void* h_buf, size_t* size);
int chx_load(chx_handle* h, const void* h_buf, size_t size);

/* ---- on-device policy and policy rollout -------------------------------------
 * The agent of the paper's experiments (Sec. 5 and Table "PPO hyper-
 * parameters": a PPO actor over the Gym-style observation) as a 3-layer MLP
 * run on the tensor cores:
 *   h1 = relu(W1 bf16(obs) + b1), h2 = relu(W2 bf16(h1) + b2),
 *   logits = W3 bf16(h2) + b3,
 * BF16 operands (bf16() = round to nearest even), FP32 accumulation.  Each
 * charger's level is sampled from the softmax of its n_levels logits by
 * inverse transform: with u = (w >> 8) * 2^-24 from Philox word w at counter
 * (env, global step of the env, charger / 4, 4), word charger % 4, under the
 * env's key, the level is the number of j < n_levels - 1 whose cumulative
 * sum e_0 + .. + e_j is <= u * sum(e), e_j = exp(l_j - max l).
 *
 * chx_policy_load: host weights, BF16 bit patterns, row-major:
 *   h_w1 [hidden][D], h_w2 [hidden][hidden], h_w3 [N * n_levels][hidden]
 *   (row c * n_levels + j = level j of charger c), biases FP32 h_b1 [hidden],
 *   h_b2 [hidden], h_b3 [N * n_levels].  D = 8 + 6 N, the observation size of
 *   one env.  Requirements (else CHX_EINVAL): hidden = 256; every station of
 *   the batch has the same charger count N, 1 <= N <= 32; 2 <= n_levels <= 12.
 *   The weights are copied to the device (the call synchronises the device
 *   first); loading again with the same N updates them in place, so captured
 *   rollouts stay valid.
 * chx_policy_act: actions for every env from observations d_obs [E][D] FP32
 *   (the layout of chx_observe) into d_actions [E][N] int8; d_logits (NULL
 *   or [E][N][n_levels] FP32) receives the logits.  Uses each env's current
 *   global step and key; changes no env state.
 * chx_policy_rollout: n_steps steps of "act, then step" from the current
 *   state, written to caller buffers (device):
 *   d_obs [n_steps][E][D]      observation the step's action was chosen from
 *                              (may be NULL in the fused form)
 *   d_actions [n_steps][E][N]  sampled levels
 *   d_reward [n_steps][E], d_done [n_steps][E] (each NULL to skip)
 *   d_logits NULL or [n_steps][E][N][n_levels].
 *   d_obs, d_actions and d_logits (also in chx_policy_act) must start on a
 *   16-byte boundary, else CHX_EINVAL.
 *   form CHX_ROLLOUT_FUSED: one kernel launch; each CTA keeps 128 envs on
 *   its SM for all n_steps (state in tensor memory, weights streamed from
 *   L2), needs N * n_levels <= 352 (else CHX_EINVAL).  CHX_ROLLOUT_SPLIT:
 *   per step one policy launch and one environment-step launch, captured
 *   into a CUDA graph on the first call with the same (n_steps, buffers,
 *   launch shape) and replayed afterwards.  Both forms compute the same
 *   function (FP32 sums may round differently) and leave the same state.
 * A tensor-core wait that runs out of time (it should not) makes chx_check
 * return CHX_ETIMEOUT; the results of that call are then invalid. */
/* Diagnostics: one bounded wait, the kind every role of the tensor-core
 * kernels uses, on a barrier nothing releases.  It must give up after its
 * limit (2^31 SM cycles, about a second), set the handle's fault flag (the
 * next chx_check returns CHX_ETIMEOUT) and leave the context usable.
 * h_result[0] = 1 if the wait gave up and raised the flag; h_result[1] =
 * cycles it waited / 2^20. */
int chx_selftest_wait(chx_handle* h, int32_t* h_result);

#define CHX_ROLLOUT_FUSED 0
#define CHX_ROLLOUT_SPLIT 1
int chx_policy_load(chx_handle* h, int32_t hidden, const uint16_t* h_w1, const float* h_b1,
                    const uint16_t* h_w2, const float* h_b2, const uint16_t* h_w3, const float* h_b3);
int chx_policy_act(chx_handle* h, const float* d_obs, int8_t* d_actions, float* d_logits, void* stream);
int chx_policy_rollout(chx_handle* h, int32_t n_steps, float* d_obs, int8_t* d_actions, float* d_reward,
                       uint8_t* d_done, float* d_logits, int32_t form, void* stream);

/* ---- serving loop ------------------------------------------------------------
 * A pool of device-resident stations stepped by requests from many actors with
 * continuous batching (the reset/step interface of the paper's Gym-style
 * environment, App. "Practical Considerations", served to many clients).
 * Stations are admitted into slots of their size class while the bytes they
 * occupy stay within an HBM budget; a station's id is its slot and also its
 * Philox stream id.
 *   - chx_srv_submit checks a request in the caller's thread and writes it,
 *     with its station list and given levels, into a record of pinned host
 *     memory the device reads; it returns a ticket.
 *   - A scheduler thread hands the device the window of tickets not yet
 *     finished; each tick (a CUDA graph, up to n_streams of them queued at
 *     once) takes, in arrival order, every request whose stations no earlier
 *     request of the window lists, steps or resets them (the fused kernel in
 *     gather mode), writes each taken request's results into its record and
 *     then raises the record's completion flag.  A tick's first kernel moves
 *     its window's end past every request published since the launch, so
 *     requests that arrive while a tick runs join the next tick to start;
 *     requests for one station are applied in submission order.
 *   - chx_srv_wait / chx_srv_test read the flag and copy the results to the
 *     caller's buffers (in the caller's thread).
 * A request's results do not depend on what else shares its tick.  All server
 * calls are thread-safe. */
#define CHX_SRV_STEP 0
#define CHX_SRV_RESET 1

typedef struct chx_srv chx_srv;

typedef struct chx_srv_cfg {
    chx_env_params params;
    chx_exo exo;                    /* host tables, copied at start; a station's
                                       arrival class is its row                     */
    int32_t class_capacity[5];      /* station slots of size class 8,16,32,64,128     */
    double hbm_budget_bytes;        /* admission limit on the bytes admitted stations
                                       occupy (33 B per charger slot + 128 B)        */
    int32_t max_tick_envs;          /* most stations in one request; a tick takes at
                                       most (n_streams + 1) x this many               */
    int32_t n_streams;              /* tick slots: ticks queued on the device at once,
                                       1..8                                           */
    int64_t max_tick_obs_floats;    /* observation floats one request can return, 0 =
                                       none; x (n_streams + 1) must stay below 2^31   */
} chx_srv_cfg;

typedef struct chx_srv_req {
    int32_t kind;                   /* CHX_SRV_STEP or CHX_SRV_RESET                  */
    int32_t n_envs;                 /* 1..max_tick_envs, no station twice             */
    const int32_t* h_env_ids;       /* station ids from chx_srv_admit (copied)        */
    const int8_t* h_actions;        /* step: levels of the listed stations' chargers,
                                       concatenated in list order (copied); NULL =
                                       Philox levels as in chx_step                  */
    float* h_reward;                /* step: [n_envs], written before completion      */
    uint8_t* h_done;                /* step: [n_envs]                                 */
    float* h_obs;                   /* step: observation after the step, 8 + 6 n floats
                                       per listed station in list order, or NULL     */
    uint64_t seed;                  /* reset: new Philox key of the listed stations   */
} chx_srv_req;

typedef struct chx_srv_stats_t {
    int64_t n_ticks, n_requests, env_steps, env_resets;
    int32_t resident;               /* admitted stations                              */
    double used_bytes, budget_bytes;
    double device_busy_ms, elapsed_ms;
    /* host time spent (ms) in: submissions, the scheduler's bookkeeping
     * (window, completed ticks; its idle spinning included), packing (0: the
     * device builds each tick), launching ticks, copying results to the
     * callers (in chx_srv_wait / chx_srv_test); ticks launched */
    double host_submit_ms, host_scan_ms, host_pack_ms, host_launch_ms, host_complete_ms;
    int64_t n_scans;
} chx_srv_stats_t;

/* Start a server on the current device: allocate the pool and tick buffers,
 * capture the tick graphs, start the scheduler thread.  CHX_EINVAL,
 * CHX_ENOMEM. */
int chx_srv_start(const chx_srv_cfg* cfg, chx_srv** out);
/* Finish in-flight ticks, stop the threads, free everything. */
int chx_srv_stop(chx_srv* s);
/* Admit a batch of stations (all or none) and start their episodes with
 * `seed`; their ids go to h_ids [n_envs].  CHX_ENOMEM if a class has no free
 * slot or the HBM budget would be exceeded. */
int chx_srv_admit(chx_srv* s, const chx_stations* st, uint64_t seed, int32_t* h_ids);
/* Free the slots of stations that no unreleased ticket lists (queued, in
 * flight, or finished and not yet collected by chx_srv_wait / chx_srv_test);
 * else CHX_EINVAL and nothing is evicted. */
int chx_srv_evict(chx_srv* s, const int32_t* h_ids, int32_t n);
/* Queue a request; *ticket identifies it.  The output buffers must stay valid
 * until the ticket completes.  Ticket t uses request record t mod 65536: while
 * the ticket 65536 before it is not yet released (by chx_srv_wait /
 * chx_srv_test), the call returns CHX_ENOMEM at once with no ticket taken
 * (release tickets, then submit again).  A ticket is waited on or tested by
 * one thread at a time. */
int chx_srv_submit(chx_srv* s, const chx_srv_req* r, uint64_t* ticket);
/* Block until the ticket completes (CHX_ETIMEOUT after timeout_us), copy its
 * results to the request's buffers and release the ticket.  latency_ns (may be
 * NULL) = the moment the completion is seen - submission.  CHX_ECUDA (with the
 * CUDA error) if the server's device work failed; the server then takes no
 * further ticks. */
int chx_srv_wait(chx_srv* s, uint64_t ticket, int64_t timeout_us, int64_t* latency_ns);
/* Non-blocking: if the ticket has completed, its results are copied, the
 * ticket is released and *h_done = 1. */
int chx_srv_test(chx_srv* s, uint64_t ticket, int32_t* h_done, int64_t* latency_ns);
int chx_srv_stats(chx_srv* s, chx_srv_stats_t* out);

/* Simulated actors for measurement: actor a owns the stations
 * h_station_ids[a*envs_per_actor ...]; it submits a step of its stations
 * (every reset_every-th request a reset instead, 0 = never), waits for it,
 * thinks for an exponential time of mean mean_think_us and repeats, for
 * warmup_s + duration_s seconds, driven by n_threads host threads.  Latency
 * percentiles and throughput cover requests completed after the warm-up. */
typedef struct chx_srv_sim_cfg {
    int32_t n_actors, envs_per_actor, n_threads, reset_every;
    double mean_think_us, warmup_s, duration_s;
    uint64_t seed;
} chx_srv_sim_cfg;
typedef struct chx_srv_sim_result {
    int64_t n_requests, env_steps;
    double seconds, env_steps_per_s;
    double p50_us, p90_us, p99_us, max_us, mean_us;
    double mean_tick_envs, device_busy_frac;
} chx_srv_sim_result;
int chx_srv_simulate(chx_srv* s, const chx_srv_sim_cfg* c, const int32_t* h_station_ids, chx_srv_sim_result* res);

/* Synchronise the handle's work on `stream` and report (then clear) the
 * device-side fault flags: CHX_ETIMEOUT if a policy kernel's wait ran out,
 * else CHX_EFAULT if a kernel saw bad input. */
int chx_check(chx_handle* h, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CHARGAX_B300_H */
