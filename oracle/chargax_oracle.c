/*
 * chargax_oracle.c -- CPU oracle for the EV charging-station step.
 *
 * TEST INFRASTRUCTURE.  This file exists to check the CUDA library: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may build, load
 * or call it.  It shares no code, header, table or constant generator with the
 * CUDA path.  It is deliberately plain: one thread, FP64 state and arithmetic,
 * loops over envs and ports in the order the paper gives (Appendix A.2 "Apply
 * Actions" -> "Charge Stationed Cars" -> "Departure of Cars" -> "Arrival of new
 * Cars", then the reward of Appendix A.3).
 *
 * Two places are NOT FP64, on purpose:
 *  - the Poisson count of arriving cars is an integer decided by floating
 *    point; it is taken in FP32 (the paper's JAX default precision, which is
 *    also the kernel's) with a fixed operation order, so both sides agree
 *    bit for bit (see orc_poisson);
 *  - inputs arrive as float32 arrays (prices, arrival rates, limits) and are
 *    widened to double.
 *
 * Randomness: Philox4x32-10 written from its published definition (Salmon,
 * Moraes, Dror, Shaw: "Parallel Random Numbers: As Easy as 1, 2, 3", SC 2011),
 * keyed per env; counters (stream, step, slot, purpose).
 *
 * Parity status of each function is recorded next to it ("pinned by ...").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_KMAX 127          /* largest Poisson count the sampler returns     */
#define ORC_PURPOSE_ARRIVAL 0u
#define ORC_PURPOSE_CAR 1u
#define ORC_PURPOSE_ACTION 2u
#define ORC_PURPOSE_DAY 3u
#define ORC_PURPOSE_POLICY 4u
#define ORC_TREM_CS 255       /* trem of a port holding a charge-sensitive car */

typedef struct orc_params {
    int32_t ep_len;        /* steps per episode (24 h / dt)                     */
    int32_t n_levels;      /* discrete action levels k = 0..n_levels-1          */
    double dt_h;           /* step length in hours                              */
    double tau;            /* bulk/absorption breakpoint of the taper           */
    double p_sell;         /* price charged to customers, EUR/kWh               */
    double c_fixed;        /* fixed running cost per step, EUR                  */
    double alpha_sat, alpha_decl, alpha_con;
    double soc_target;     /* SoC a user wants at departure                     */
    double p_max_kw[2];    /* per charger type: 0 = AC, 1 = DC                  */
    double eta_port[2];
    double cap_kwh[2];     /* U(lo, hi) battery capacity                        */
    double soc0[2];        /* U(lo, hi) arrival SoC                             */
    int32_t stay_steps[2]; /* inclusive integer range of the stay, in steps     */
    double rbar_kw[2][2];  /* [type][lo, hi] car maximum rate per charger type  */
    /* vehicle-to-grid mode: signed levels, station battery, sell-back price,
     * degradation penalty (see orc_step) */
    int32_t v2g;
    double sell_grid_ratio;
    double alpha_degrad;
    double batt_cap_kwh, batt_rate_kw, batt_tau, batt_soc0;
    /* Delta-current action form (A.2 "Apply Actions"): the level is an
     * increment of the charger's (battery's) last applied power */
    int32_t action_delta;
    double p_max_dis_kw[2]; /* discharge maximum I_max<- per charger type (V2G) */
    /* charge-sensitive users (u = 1, A.1 User Profiles): a car's user is
     * charge-sensitive iff the low byte of its first profile word is below
     * cs_share_256; such a user leaves once its Delta E_remain is 0, read
     * as at most eps_cap of its car's capacity (the target SoC reached
     * within eps_cap); it costs alpha_sat1 * c_Sat,1 with early-leave
     * weight beta_early */
    int32_t cs_share_256;
    double alpha_sat1, beta_early, eps_cap;
} orc_params;

typedef struct orc {
    orc_params p;
    int32_t E, n_days, n_classes;
    int64_t P, G;
    int64_t *port_off, *group_off;
    int32_t *n_ports, *n_groups, *group_size, *arrival_class;
    uint8_t *port_type;
    int32_t *port_group;                   /* global group index of each port   */
    double *group_limit, *group_eta, *grid_limit, *grid_eta;
    /* deeper architecture trees (Fig. charge-tree c): nodes above the
     * groups; parents are global indices, -1 = the root */
    int64_t U, *upper_off;
    int32_t *group_parent, *upper_parent;
    double *upper_limit, *upper_eta;
    float *price, *lam;                    /* [D][T], [C][T] as given           */
    /* per-port state (car-state + port state, Appendix A.1) */
    double *soc, *erem, *cap, *rbar, *pw;
    int32_t *trem;                         /* remaining steps, 0 = empty port;
                                              ORC_TREM_CS: a charge-sensitive car */
    int32_t *due;                          /* Delta t_remain of a charge-sensitive
                                              car (steps to its desired departure,
                                              negative once overdue)              */
    /* per-env state */
    int32_t *tod, *day;
    uint32_t *gstep, *key0, *key1;
    uint32_t *ncar;                        /* cars admitted since the last reset    */
    uint32_t *stream;                      /* Philox stream id (default: index) */
    double *ep_ret, *last_ret;
    uint32_t *n_episodes;
    /* station battery (V2G mode): SoC and last applied power */
    double *bsoc, *bp;
    /* per-env running statistics */
    double *st_arrived, *st_rejected, *st_missing, *st_charged;
    /* per-env record of the last step (for invariant tests) */
    int32_t *inf_M, *inf_admitted, *inf_departed;
    double *inf_csat, *inf_ccon, *inf_enet, *inf_egrid, *inf_price, *inf_req_sum;
    double *inf_eto, *inf_eb, *inf_degrad, *inf_egrid_net;   /* V2G terms of the last step */
    double *inf_csat1;                     /* c_Sat,1 of the last step                        */
    double *inf_cs_margin;                 /* min over charge-sensitive cars tested in the last
                                              step of |Delta E_remain - eps_cap C| / (eps_cap C),
                                              their distance from the departure decision      */
    double *scratch_p;                     /* per-port power within one step    */
    double *scratch_req;                   /* per-port requested power (pre-rescale) */
    uint8_t *scratch_in;                   /* per-port leaf mask of one node         */
    uint8_t *scratch_leave;                /* port's stay ended in this step    */
} orc;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011, Sec. 3.3 and Table 2): ten rounds of  */
/* two 32x32->64 multiplies on counter words 0 and 2, XOR of the high halves */
/* into the other words and the key, with the key bumped by the Weyl        */
/* constants between rounds.  Pinned by the published known-answer values   */
/* (tests/golden/philox4x32_10_kat.txt).                                    */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t a = (uint64_t)M0 * (uint64_t)x0;
        uint64_t b = (uint64_t)M1 * (uint64_t)x2;
        uint32_t a_hi = (uint32_t)(a >> 32), a_lo = (uint32_t)a;
        uint32_t b_hi = (uint32_t)(b >> 32), b_lo = (uint32_t)b;
        uint32_t y0 = b_hi ^ x1 ^ k0;
        uint32_t y1 = b_lo;
        uint32_t y2 = a_hi ^ x3 ^ k1;
        uint32_t y3 = a_lo;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(const orc *o, int32_t e, uint32_t c1, uint32_t c2, uint32_t purpose, uint32_t out[4])
{
    uint32_t ctr[4] = {o->stream[e], c1, c2, purpose};
    uint32_t key[2] = {o->key0[e], o->key1[e]};
    orc_philox(ctr, key, out);
}

/* integer in [0, n): high word of the 64-bit product (exact) */
static uint32_t to_range(uint32_t w, uint32_t n) { return (uint32_t)(((uint64_t)w * n) >> 32); }

/* uniform in [0, 1) from the top 24 bits (exactly representable in FP32) */
static double to_unit(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------ */
/* Arrival count M(t) ~ Poisson(lambda(t)) (Appendix "Practical             */
/* Considerations": bundled scenarios give mean cars per step, the count is */
/* drawn from a Poisson).  Inverse transform: the smallest k whose CDF      */
/* exceeds u.  Because k is an integer chosen by floating point, the        */
/* decision is taken in FP32 with this exact sequence of correctly rounded  */
/* operations (exp in double, rounded once).  Pinned against the exact      */
/* Poisson CDF (tests/test_oracle_pins.py).                                 */
/* ------------------------------------------------------------------------ */
int32_t orc_poisson(float lam, uint32_t w)
{
    float u = (float)(w >> 8) * 5.9604644775390625e-8f;    /* 2^-24 */
    float pk = (float)exp(-(double)lam);
    float cdf = pk;
    int32_t k = 0;
    while (u >= cdf && k < ORC_KMAX) {
        k += 1;
        float num = pk * lam;
        pk = num / (float)k;
        cdf = cdf + pk;
    }
    return k;
}

/* Charging-rate taper r_hat(SoC) (Appendix A.1, Car Profiles): bulk stage at
 * r_bar up to tau, then linear to zero at SoC = 1.  Pinned by the closed-form
 * single-car trajectory test. */
double orc_taper(double soc, double rbar, double tau)
{
    if (soc <= tau) return rbar;
    return (1.0 - soc) * rbar / (1.0 - tau);
}

static void clear_port(orc *o, int64_t i)
{
    o->soc[i] = 0.0; o->erem[i] = 0.0; o->cap[i] = 0.0; o->rbar[i] = 0.0; o->trem[i] = 0; o->due[i] = 0;
}

/* Episode start (Appendix "Practical Considerations", exploring starts): an
 * empty station at step-of-day 0 and a random day of the price bank. */
static void start_episode(orc *o, int32_t e, uint32_t c1, uint32_t c2)
{
    for (int64_t i = o->port_off[e]; i < o->port_off[e + 1]; ++i) { clear_port(o, i); o->pw[i] = 0.0; }
    o->bsoc[e] = o->p.v2g ? o->p.batt_soc0 : 0.0;
    o->bp[e] = 0.0;
    o->tod[e] = 0;
    uint32_t w[4];
    draw(o, e, c1, c2, ORC_PURPOSE_DAY, w);
    o->day[e] = (int32_t)to_range(w[0], (uint32_t)o->n_days);
}

void orc_reset(orc *o, const int32_t *env_ids, int32_t n, uint64_t seed)
{
    int32_t count = env_ids ? n : o->E;
    for (int32_t j = 0; j < count; ++j) {
        int32_t e = env_ids ? env_ids[j] : j;
        o->key0[e] = (uint32_t)seed;
        o->key1[e] = (uint32_t)(seed >> 32);
        o->gstep[e] = 0;
        o->ncar[e] = 0;
        o->ep_ret[e] = 0.0;
        start_episode(o, e, 0u, 1u);
    }
}

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

orc *orc_create(const orc_params *prm, int32_t E,
                const int32_t *n_ports, const uint8_t *port_type,
                const int32_t *n_groups, const int32_t *group_size,
                const float *group_limit, const float *group_eta,
                const float *grid_limit, const float *grid_eta,
                const int32_t *arrival_class,
                int32_t n_days, const float *price,
                int32_t n_classes, const float *lam, uint64_t seed)
{
    orc *o = (orc *)xcalloc(1, sizeof(orc));
    o->p = *prm;
    o->E = E; o->n_days = n_days; o->n_classes = n_classes;
    o->port_off = (int64_t *)xcalloc((size_t)E + 1, sizeof(int64_t));
    o->group_off = (int64_t *)xcalloc((size_t)E + 1, sizeof(int64_t));
    for (int32_t e = 0; e < E; ++e) {
        o->port_off[e + 1] = o->port_off[e] + n_ports[e];
        o->group_off[e + 1] = o->group_off[e] + n_groups[e];
    }
    o->P = o->port_off[E]; o->G = o->group_off[E];
    int64_t P = o->P, G = o->G;
    o->n_ports = (int32_t *)xcalloc((size_t)E, sizeof(int32_t));
    o->n_groups = (int32_t *)xcalloc((size_t)E, sizeof(int32_t));
    o->arrival_class = (int32_t *)xcalloc((size_t)E, sizeof(int32_t));
    o->grid_limit = (double *)xcalloc((size_t)E, sizeof(double));
    o->grid_eta = (double *)xcalloc((size_t)E, sizeof(double));
    o->port_type = (uint8_t *)xcalloc((size_t)P, 1);
    o->port_group = (int32_t *)xcalloc((size_t)P, sizeof(int32_t));
    o->group_size = (int32_t *)xcalloc((size_t)G, sizeof(int32_t));
    o->group_limit = (double *)xcalloc((size_t)G, sizeof(double));
    o->group_eta = (double *)xcalloc((size_t)G, sizeof(double));
    memcpy(o->n_ports, n_ports, sizeof(int32_t) * (size_t)E);
    memcpy(o->n_groups, n_groups, sizeof(int32_t) * (size_t)E);
    memcpy(o->arrival_class, arrival_class, sizeof(int32_t) * (size_t)E);
    memcpy(o->port_type, port_type, (size_t)P);
    memcpy(o->group_size, group_size, sizeof(int32_t) * (size_t)G);
    for (int32_t e = 0; e < E; ++e) {
        o->grid_limit[e] = grid_limit[e];
        o->grid_eta[e] = grid_eta ? grid_eta[e] : 1.0;
        int64_t port = o->port_off[e];
        for (int64_t g = o->group_off[e]; g < o->group_off[e + 1]; ++g)
            for (int32_t k = 0; k < group_size[g]; ++k) o->port_group[port++] = (int32_t)g;
    }
    for (int64_t g = 0; g < G; ++g) {
        o->group_limit[g] = group_limit[g];
        o->group_eta[g] = group_eta ? group_eta[g] : 1.0;
    }
    size_t T = (size_t)prm->ep_len;
    o->price = (float *)xcalloc((size_t)n_days * T, sizeof(float));
    o->lam = (float *)xcalloc((size_t)n_classes * T, sizeof(float));
    memcpy(o->price, price, sizeof(float) * (size_t)n_days * T);
    memcpy(o->lam, lam, sizeof(float) * (size_t)n_classes * T);

    o->soc = (double *)xcalloc((size_t)P, sizeof(double));
    o->erem = (double *)xcalloc((size_t)P, sizeof(double));
    o->cap = (double *)xcalloc((size_t)P, sizeof(double));
    o->rbar = (double *)xcalloc((size_t)P, sizeof(double));
    o->pw = (double *)xcalloc((size_t)P, sizeof(double));
    o->scratch_p = (double *)xcalloc((size_t)P, sizeof(double));
    o->scratch_req = (double *)xcalloc((size_t)P, sizeof(double));
    o->scratch_in = (uint8_t *)xcalloc((size_t)P + 1, 1);
    o->upper_off = (int64_t *)xcalloc((size_t)E + 1, sizeof(int64_t));
    o->group_parent = (int32_t *)xcalloc((size_t)G, sizeof(int32_t));
    for (int64_t g = 0; g < G; ++g) o->group_parent[g] = -1;
    o->scratch_leave = (uint8_t *)xcalloc((size_t)P, 1);
    o->trem = (int32_t *)xcalloc((size_t)P, sizeof(int32_t));
    o->due = (int32_t *)xcalloc((size_t)P, sizeof(int32_t));
    o->tod = (int32_t *)xcalloc((size_t)E, sizeof(int32_t));
    o->day = (int32_t *)xcalloc((size_t)E, sizeof(int32_t));
    o->gstep = (uint32_t *)xcalloc((size_t)E, sizeof(uint32_t));
    o->ncar = (uint32_t *)xcalloc((size_t)E, sizeof(uint32_t));
    o->key0 = (uint32_t *)xcalloc((size_t)E, sizeof(uint32_t));
    o->key1 = (uint32_t *)xcalloc((size_t)E, sizeof(uint32_t));
    o->stream = (uint32_t *)xcalloc((size_t)E, sizeof(uint32_t));
    for (int32_t e = 0; e < E; ++e) o->stream[e] = (uint32_t)e;
    o->ep_ret = (double *)xcalloc((size_t)E, sizeof(double));
    o->last_ret = (double *)xcalloc((size_t)E, sizeof(double));
    o->n_episodes = (uint32_t *)xcalloc((size_t)E, sizeof(uint32_t));
    o->st_arrived = (double *)xcalloc((size_t)E, sizeof(double));
    o->st_rejected = (double *)xcalloc((size_t)E, sizeof(double));
    o->st_missing = (double *)xcalloc((size_t)E, sizeof(double));
    o->st_charged = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_M = (int32_t *)xcalloc((size_t)E, sizeof(int32_t));
    o->inf_admitted = (int32_t *)xcalloc((size_t)E, sizeof(int32_t));
    o->inf_departed = (int32_t *)xcalloc((size_t)E, sizeof(int32_t));
    o->inf_csat = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_ccon = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_enet = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_egrid = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_price = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_req_sum = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_eto = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_eb = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_degrad = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_egrid_net = (double *)xcalloc((size_t)E, sizeof(double));
    o->bsoc = (double *)xcalloc((size_t)E, sizeof(double));
    o->bp = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_csat1 = (double *)xcalloc((size_t)E, sizeof(double));
    o->inf_cs_margin = (double *)xcalloc((size_t)E, sizeof(double));
    orc_reset(o, NULL, 0, seed);
    return o;
}

void orc_destroy(orc *o)
{
    if (!o) return;
    void *ptrs[] = {o->port_off, o->group_off, o->n_ports, o->n_groups, o->arrival_class, o->grid_limit,
                    o->grid_eta, o->port_type, o->port_group, o->group_size, o->group_limit, o->group_eta,
                    o->price, o->lam, o->soc, o->erem, o->cap, o->rbar, o->pw, o->scratch_p, o->scratch_leave, o->trem, o->tod,
                    o->day, o->gstep, o->ncar, o->key0, o->key1, o->stream, o->ep_ret, o->last_ret, o->n_episodes,
                    o->st_arrived, o->st_rejected, o->st_missing, o->st_charged, o->inf_M, o->inf_admitted,
                    o->inf_departed, o->inf_csat, o->inf_ccon, o->inf_enet, o->inf_egrid, o->inf_price,
                    o->inf_req_sum, o->inf_eto, o->inf_eb, o->inf_degrad, o->inf_egrid_net, o->bsoc, o->bp, o->due,
                    o->inf_csat1, o->inf_cs_margin,
                    o->scratch_req, o->scratch_in, o->upper_off, o->group_parent, o->upper_parent, o->upper_limit, o->upper_eta};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    free(o);
}

/* Action level of local port q of env e at global step g when no action
 * array is given (the random policy of the speed benchmark, Table
 * "performance"): one Philox call of counter (e, g/8, q, ACTION) serves 8
 * steps; step g takes the 16-bit half (g mod 2) of word (g/2 mod 4) and maps
 * it to 0..n_levels-1 by the high half of the product with n_levels. */
int32_t orc_random_action(const orc *o, int32_t e, uint32_t g, int32_t q)
{
    uint32_t w[4];
    draw(o, e, g >> 3, (uint32_t)q, ORC_PURPOSE_ACTION, w);
    uint32_t word = w[(g >> 1) & 3u];
    uint32_t half = (g & 1u) ? (word >> 16) : (word & 0xFFFFu);
    return (int32_t)((half * (uint32_t)o->p.n_levels) >> 16);
}

/* Uniforms of the policy's action samples for the next step (the PPO actor
 * of Sec. 5 samples one level per charger): u[e][q] for charger q of env e
 * is word q mod 4 of the Philox block (e, g, q / 4, POLICY), g = the env's
 * global step, mapped to [0, 1) by its top 24 bits.  All envs must have
 * n_ports chargers.  Pinned by the Philox known-answer tests and by the
 * policy pins (closed-form samples, frequencies). */
void orc_policy_uniforms(const orc *o, int32_t n_ports, double *u)
{
    for (int32_t e = 0; e < o->E; ++e)
        for (int32_t q = 0; q < n_ports; q += 4) {
            uint32_t w[4];
            draw(o, e, o->gstep[e], (uint32_t)(q >> 2), ORC_PURPOSE_POLICY, w);
            for (int32_t j = 0; j < 4 && q + j < n_ports; ++j)
                u[(int64_t)e * n_ports + q + j] = to_unit(w[j]);
        }
}

/* Deeper trees (Fig. charge-tree c): n_upper[e] nodes above the groups of
 * env e, listed per env; group_parent[g] and upper_parent[u] are indices
 * into the env's own upper nodes, -1 = the root; each upper node has a
 * limit I_H (kW) and efficiency eta_H.  Without a call every group hangs
 * from the root. */
void orc_set_tree(orc *o, const int32_t *n_upper, const int32_t *group_parent, const int32_t *upper_parent,
                  const float *upper_limit, const float *upper_eta)
{
    for (int32_t e = 0; e < o->E; ++e) o->upper_off[e + 1] = o->upper_off[e] + n_upper[e];
    o->U = o->upper_off[o->E];
    free(o->upper_parent); free(o->upper_limit); free(o->upper_eta);
    o->upper_parent = (int32_t *)xcalloc((size_t)o->U + 1, sizeof(int32_t));
    o->upper_limit = (double *)xcalloc((size_t)o->U + 1, sizeof(double));
    o->upper_eta = (double *)xcalloc((size_t)o->U + 1, sizeof(double));
    for (int32_t e = 0; e < o->E; ++e) {
        int64_t u0 = o->upper_off[e];
        for (int64_t g = o->group_off[e]; g < o->group_off[e + 1]; ++g)
            o->group_parent[g] = group_parent[g] < 0 ? -1 : (int32_t)(u0 + group_parent[g]);
        for (int64_t u = u0; u < o->upper_off[e + 1]; ++u) {
            o->upper_parent[u] = upper_parent[u] < 0 ? -1 : (int32_t)(u0 + upper_parent[u]);
            o->upper_limit[u] = upper_limit[u];
            o->upper_eta[u] = upper_eta[u];
        }
    }
}

/* depth below the root of an upper node (a child of the root has depth 1) */
static int32_t upper_depth(const orc *o, int32_t u)
{
    int32_t d = 0;
    for (int32_t a = u; a >= 0; a = o->upper_parent[a]) d += 1;
    return d;
}

static int32_t group_depth(const orc *o, int64_t g)
{
    int32_t a = o->group_parent[g];
    return 1 + (a < 0 ? 0 : upper_depth(o, a));
}

/* is port i a leaf of upper node u (u an ancestor of the port's group)? */
static int port_under_upper(const orc *o, int64_t i, int32_t u)
{
    for (int32_t a = o->group_parent[o->port_group[i]]; a >= 0; a = o->upper_parent[a])
        if (a == u) return 1;
    return 0;
}

/* One node H of Eq. (ArchConst) over the ports marked in `in`: the penalty
 * on the requested power, then the proportional rescale of the leaves if
 * (1/eta_H) |sum| > I_H. */
static void apply_node(orc *o, int64_t p0, int64_t p1, const uint8_t *in, double limit, double eta, int v2g,
                       double *c_con)
{
    double s = 0.0, sreq = 0.0;
    for (int64_t i = p0; i < p1; ++i)
        if (in[i]) { s += o->scratch_p[i]; sreq += o->scratch_req[i]; }
    double over_req = (v2g ? fabs(sreq) : sreq) / eta - limit;
    if (over_req > *c_con) *c_con = over_req;
    double mag = v2g ? fabs(s) : s;
    if (mag / eta > limit) {
        double scale = eta * limit / mag;
        for (int64_t i = p0; i < p1; ++i)
            if (in[i]) o->scratch_p[i] *= scale;
    }
}

/* ------------------------------------------------------------------------ */
/* One transition of every env, Appendix A.2 then A.3.                      */
/* actions: int8 level per port in batch port order with stride `lda`, or   */
/* NULL for Philox-drawn uniform levels.  reward[E] and done[E] are outputs.*/
/* In V2G mode (p.v2g) each env has one more action, its battery's level,   */
/* after its ports: port i of env e at (i + e) * lda, the battery of env e  */
/* at (port_off[e+1] + e) * lda; a drawn battery level uses local port      */
/* index n_ports.                                                           */
/* ------------------------------------------------------------------------ */

/* Requested power of level k (A.2 "Apply Actions"; discretisation of
 * "Practical Considerations").  Absolute form: k/(L-1) of the maximum, or
 * in V2G mode the signed (k - h)/h of it, h = (L-1)/2.  Delta-current form:
 * the last applied power plus the signed increment (k - h)/h of the
 * maximum, I_drawn(t - dt) + a(t). */
static double request(const orc *o, int32_t k, double pmax, double last)
{
    const int32_t L = o->p.n_levels, h = (L - 1) / 2;
    if (o->p.action_delta) return last + (double)(k - h) / (double)h * pmax;
    if (o->p.v2g) return (double)(k - h) / (double)h * pmax;
    return (double)k / (double)(L - 1) * pmax;
}

/* V2G clip (A.2 "Apply Actions", both branches): charge as in the
 * charge-only mode; discharge limited by the request, the car's discharging
 * rate (the charging curve flipped at SoC = 0.5: r_hat(1 - SoC)), the port's
 * discharge maximum I_max<- and SoC >= 0.  Pinned by the closed-form
 * discharge trajectory and by the reduction to the charge-only mode. */
static double v2g_clip(double preq, double soc, double erem, double cap, double rbar, double tau, double pmax,
                       double pmax_dis, double dt)
{
    if (preq >= 0.0) {
        double P = preq, rhat = orc_taper(soc, rbar, tau);
        double soc_cap = (1.0 - soc) * cap / dt, dem_cap = erem / dt;
        if (rhat < P) P = rhat;
        if (pmax < P) P = pmax;
        if (soc_cap < P) P = soc_cap;
        if (dem_cap < P) P = dem_cap;
        return P < 0.0 ? 0.0 : P;
    }
    double D = -preq, rdis = orc_taper(1.0 - soc, rbar, tau), soc_cap = soc * cap / dt;
    if (rdis < D) D = rdis;
    if (pmax_dis < D) D = pmax_dis;
    if (soc_cap < D) D = soc_cap;
    return D < 0.0 ? 0.0 : -D;
}

void orc_step(orc *o, const int8_t *actions, int64_t lda, double *reward, uint8_t *done)
{
    const orc_params *p = &o->p;
    const double dt = p->dt_h;
    const int v2g = p->v2g != 0;
    for (int32_t e = 0; e < o->E; ++e) {
        const int64_t p0 = o->port_off[e], p1 = o->port_off[e + 1];
        const uint32_t g = o->gstep[e];
        const int32_t t = o->tod[e];

        /* (i) Apply Actions: requested level clipped by the port capacity and
         * by the car's current maximum rate r_hat(SoC); the two extra caps
         * keep SoC <= 1 and the remaining demand >= 0 (SoC in [0,1] and
         * Delta E_remain >= 0 are the state domains of the "State summary").
         * V2G: signed levels (v2g_clip) and the station battery, a leaf of
         * the root with its own level, rate curve and SoC in [0, 1]. */
        double req_sum = 0.0;
        for (int64_t i = p0; i < p1; ++i) {
            double P = 0.0;
            if (o->trem[i] > 0) {
                int32_t k = actions ? (int32_t)actions[(i + (v2g ? e : 0)) * lda]
                                    : orc_random_action(o, e, g, (int32_t)(i - p0));
                int ty = o->port_type[i];
                double pmax = p->p_max_kw[ty];
                double preq = request(o, k, pmax, o->pw[i]);
                if (v2g) {
                    P = v2g_clip(preq, o->soc[i], o->erem[i], o->cap[i], o->rbar[i], p->tau, pmax,
                                 p->p_max_dis_kw[ty], dt);
                } else {
                    double rhat = orc_taper(o->soc[i], o->rbar[i], p->tau);
                    double soc_cap = (1.0 - o->soc[i]) * o->cap[i] / dt;
                    double dem_cap = o->erem[i] / dt;
                    P = preq;
                    if (rhat < P) P = rhat;
                    if (pmax < P) P = pmax;
                    if (soc_cap < P) P = soc_cap;
                    if (dem_cap < P) P = dem_cap;
                    if (P < 0.0) P = 0.0;
                }
            }
            o->scratch_p[i] = P;
            req_sum += P;
        }
        double Pb = 0.0;
        if (v2g) {
            int32_t kb = actions ? (int32_t)actions[(p1 + e) * lda] : orc_random_action(o, e, g, o->n_ports[e]);
            /* the battery never leaves: its remaining demand never binds */
            Pb = v2g_clip(request(o, kb, p->batt_rate_kw, o->bp[e]), o->bsoc[e], 1e300, p->batt_cap_kwh,
                          p->batt_rate_kw, p->batt_tau, p->batt_rate_kw, p->batt_rate_kw, dt);
        }

        /* Architecture constraint, Eq. (ArchConst): for every subtree H,
         * (1/eta_H) * sum of its leaves' power <= I_H.  Violations are
         * resolved by proportional rescaling of the leaves, bottom-up: the
         * nodes in order of decreasing depth (every node after all nodes
         * below it), the root (grid connection) last.  The
         * constraint-violation penalty (Appendix A.3) is measured on the
         * requested (pre-rescale) power.  V2G: the limit binds the net flow
         * in either direction (|sum| / eta_H <= I_H), and the battery is a
         * leaf of the root. */
        double c_con = 0.0;
        for (int64_t i = p0; i < p1; ++i) o->scratch_req[i] = o->scratch_p[i];
        {
            int32_t max_d = 1;
            for (int64_t gi = o->group_off[e]; gi < o->group_off[e + 1]; ++gi) {
                int32_t d = group_depth(o, gi);
                if (d > max_d) max_d = d;
            }
            uint8_t *in = o->scratch_in;
            for (int32_t d = max_d; d >= 1; --d) {
                for (int64_t gi = o->group_off[e]; gi < o->group_off[e + 1]; ++gi) {
                    if (group_depth(o, gi) != d) continue;
                    for (int64_t i = p0; i < p1; ++i) in[i] = o->port_group[i] == gi;
                    apply_node(o, p0, p1, in, o->group_limit[gi], o->group_eta[gi], v2g, &c_con);
                }
                for (int64_t u = o->upper_off[e]; u < o->upper_off[e + 1]; ++u) {
                    if (upper_depth(o, (int32_t)u) != d) continue;
                    for (int64_t i = p0; i < p1; ++i) in[i] = (uint8_t)port_under_upper(o, i, (int32_t)u);
                    apply_node(o, p0, p1, in, o->upper_limit[u], o->upper_eta[u], v2g, &c_con);
                }
            }
        }
        {
            double req_root = req_sum + Pb;
            double root_over = (v2g ? fabs(req_root) : req_root) / o->grid_eta[e] - o->grid_limit[e];
            if (root_over > c_con) c_con = root_over;
            double s = Pb;
            for (int64_t i = p0; i < p1; ++i) s += o->scratch_p[i];
            double mag = v2g ? fabs(s) : s;
            if (mag / o->grid_eta[e] > o->grid_limit[e]) {
                double scale = o->grid_eta[e] * o->grid_limit[e] / mag;
                for (int64_t i = p0; i < p1; ++i) o->scratch_p[i] *= scale;
                Pb *= scale;
            }
        }

        /* (ii) Charge Stationed Cars at constant power over dt; energy bought
         * from the grid includes the port efficiency (Appendix A.3).  V2G:
         * energy pushed into the grid by discharging cars loses the port
         * efficiency on the way (Eq. Profit1), the battery's energy counts at
         * face value, and SoC stays in [0, 1]. */
        double e_net = 0.0, e_grid = 0.0, e_to = 0.0;
        for (int64_t i = p0; i < p1; ++i) {
            double P = o->scratch_p[i];
            o->pw[i] = P;
            if (o->trem[i] > 0) {
                double dE = P * dt;
                double s = o->soc[i] + dE / o->cap[i];
                o->soc[i] = s > 1.0 ? 1.0 : (s < 0.0 ? 0.0 : s);
                double r = o->erem[i] - dE;
                o->erem[i] = r < 0.0 ? 0.0 : r;
                e_net += dE;
                if (dE >= 0.0) e_grid += dE / p->eta_port[o->port_type[i]];
                else e_to += dE * p->eta_port[o->port_type[i]];
            }
        }
        double e_b = 0.0;
        if (v2g) {
            e_b = Pb * dt;
            double s = o->bsoc[e] + e_b / p->batt_cap_kwh;
            o->bsoc[e] = s > 1.0 ? 1.0 : (s < 0.0 ? 0.0 : s);
            o->bp[e] = Pb;
        }

        /* time moves on: every stationed car has one step less to stay; a
         * time-sensitive user (u = 0) leaves when none is left, a
         * charge-sensitive one (u = 1) once its demand is met: Delta
         * E_remain = 0, read as at most eps_cap of the car's capacity (its
         * Delta t_remain may turn negative meanwhile) */
        double cs_margin = 1e300;
        for (int64_t i = p0; i < p1; ++i) {
            o->scratch_leave[i] = 0;
            if (o->trem[i] == ORC_TREM_CS) {
                double thr = p->eps_cap * o->cap[i];
                o->due[i] -= 1;
                o->scratch_leave[i] = (o->erem[i] <= thr);
                if (thr > 0.0) {
                    double m = fabs(o->erem[i] - thr) / thr;
                    if (m < cs_margin) cs_margin = m;
                }
            } else if (o->trem[i] > 0) {
                o->trem[i] -= 1;
                o->scratch_leave[i] = (o->trem[i] == 0);
            }
        }

        /* (iii) Departure of Cars: time-sensitive users (u = 0) leave when no
         * time remains; the satisfaction penalty c_Sat,0 adds their missing
         * energy. */
        double c_sat = 0.0, c_sat1 = 0.0;
        int32_t departed = 0;
        for (int64_t i = p0; i < p1; ++i) {
            if (o->scratch_leave[i]) {
                if (o->trem[i] == ORC_TREM_CS) {
                    /* c_Sat,1 (A.3): steps overdue, minus beta x steps early */
                    int32_t d = o->due[i];
                    c_sat1 += (d < 0 ? (double)-d : 0.0) - p->beta_early * (d > 0 ? (double)d : 0.0);
                } else {
                    c_sat += o->erem[i] > 0.0 ? o->erem[i] : 0.0;
                }
                clear_port(o, i);
                /* Delta form: the charger of a departed car drops to 0, the
                 * base of the next car's first increment (an arriving car's
                 * port state starts at I_drawn = 0) */
                if (p->action_delta) o->pw[i] = 0.0;
                departed += 1;
            }
        }

        /* (iv) Arrival of new Cars: M ~ Poisson(lambda(t)), clipped by the
         * free ports (first come first served); the rest are rejected.  Car j
         * of this step parks at the j-th free port in port order; its car and
         * user profile are the Philox words of the station's car number
         * (cars admitted since the last reset + j). */
        /* one Philox call of counter (e, g/4, 0, ARRIVAL) serves 4 steps:
         * step g uses word g mod 4 */
        uint32_t w[4];
        draw(o, e, g >> 2, 0u, ORC_PURPOSE_ARRIVAL, w);
        float lam = o->lam[(size_t)o->arrival_class[e] * (size_t)p->ep_len + (size_t)t];
        int32_t M = orc_poisson(lam, w[g & 3u]);
        int32_t n_free = 0;
        for (int64_t i = p0; i < p1; ++i) n_free += (o->trem[i] == 0);
        int32_t m = M < n_free ? M : n_free;
        int32_t c_decl = M - m;
        int32_t j = 0;
        for (int64_t i = p0; i < p1 && j < m; ++i) {
            if (o->trem[i] != 0) continue;
            uint32_t c[4];
            draw(o, e, o->ncar[e] + (uint32_t)j, 0u, ORC_PURPOSE_CAR, c);
            int ty = o->port_type[i];
            double C = p->cap_kwh[0] + (p->cap_kwh[1] - p->cap_kwh[0]) * to_unit(c[0]);
            double soc0 = p->soc0[0] + (p->soc0[1] - p->soc0[0]) * to_unit(c[1]);
            uint32_t span = (uint32_t)(p->stay_steps[1] - p->stay_steps[0] + 1);
            int32_t stay = p->stay_steps[0] + (int32_t)to_range(c[2], span);
            double rb = p->rbar_kw[ty][0] + (p->rbar_kw[ty][1] - p->rbar_kw[ty][0]) * to_unit(c[3]);
            double want = p->soc_target - soc0;
            o->cap[i] = C;
            o->soc[i] = soc0;
            o->erem[i] = (want > 0.0 ? want : 0.0) * C;
            o->rbar[i] = rb;
            /* user preference u (A.1 User Profiles): the low byte of the
             * first word, unused by the capacity's 24 bits */
            if ((int32_t)(c[0] & 0xFFu) < p->cs_share_256) {
                o->trem[i] = ORC_TREM_CS;
                o->due[i] = stay;
            } else {
                o->trem[i] = stay;
            }
            j += 1;
        }

        /* Reward (Appendix A.3): profit with the two-case grid price, minus
         * the weighted penalties.  Delta E_grid,net = energy bought for the
         * cars + energy pushed into the grid by discharging cars (<= 0) +
         * the battery's energy; when it is <= 0 the station sells to the
         * grid at p_sell,grid (= sell_grid_ratio x the buy price in V2G
         * mode; without V2G the case cannot occur and p_sell,grid = p_buy).
         * Battery degradation: discharged energy of the battery and of the
         * cars (c_degrad,battery + c_degrad,cars). */
        double price = o->price[(size_t)o->day[e] * (size_t)p->ep_len + (size_t)t];
        double e_grid_net = e_grid + e_to + e_b;
        double profit;
        if (e_grid_net > 0.0) profit = p->p_sell * e_net - price * e_grid_net - p->c_fixed;
        else profit = p->p_sell * e_net - (v2g ? p->sell_grid_ratio : 1.0) * price * e_grid_net - p->c_fixed;
        double c_degrad = (e_b < 0.0 ? -e_b : 0.0) - e_to;
        double r = profit - p->alpha_sat * c_sat - p->alpha_decl * (double)c_decl - p->alpha_con * c_con;
        if (v2g) r -= p->alpha_degrad * c_degrad;
        r -= p->alpha_sat1 * c_sat1;

        o->ncar[e] += (uint32_t)m;
        o->inf_M[e] = M; o->inf_admitted[e] = m; o->inf_departed[e] = departed;
        o->inf_csat[e] = c_sat; o->inf_ccon[e] = c_con; o->inf_enet[e] = e_net;
        o->inf_egrid[e] = e_grid; o->inf_price[e] = price; o->inf_req_sum[e] = req_sum;
        o->inf_eto[e] = e_to; o->inf_eb[e] = e_b; o->inf_degrad[e] = c_degrad; o->inf_egrid_net[e] = e_grid_net;
        o->inf_csat1[e] = c_sat1; o->inf_cs_margin[e] = cs_margin;
        o->st_arrived[e] += m; o->st_rejected[e] += c_decl;
        o->st_missing[e] += c_sat; o->st_charged[e] += e_net;

        o->ep_ret[e] += r;
        reward[e] = r;
        o->tod[e] = t + 1;
        o->gstep[e] = g + 1u;
        done[e] = 0;
        /* episode end: record the return and start a new one at once */
        if (o->tod[e] >= p->ep_len) {
            done[e] = 1;
            o->last_ret[e] = o->ep_ret[e];
            o->ep_ret[e] = 0.0;
            o->n_episodes[e] += 1;
            start_episode(o, e, g, 0u);
        }
    }
}

/* Observation (the state of Appendix "State summary" plus time of day, the
 * episode's day and a weekday flag, as the agent sees them).  Layout per env
 * at float offset F*e + Q*port_off[e]: F env features, then Q per port;
 * F = 8, or 10 in V2G mode (+ battery SoC, battery power / its rate, the
 * battery state s_battery of A.1); Q = 6, or 7 with charge-sensitive users
 * (+ the user preference u; their stay feature is Delta t_remain). */
int32_t orc_obs_env_features(const orc *o) { return o->p.v2g ? 10 : 8; }
int32_t orc_obs_port_features(const orc *o) { return o->p.cs_share_256 > 0 ? 7 : 6; }

void orc_observe(const orc *o, double *obs)
{
    const orc_params *p = &o->p;
    const double two_pi = 6.283185307179586476925;
    const int64_t F = orc_obs_env_features(o), Q = orc_obs_port_features(o);
    for (int32_t e = 0; e < o->E; ++e) {
        double *ob = obs + F * (int64_t)e + Q * o->port_off[e];
        int32_t t = o->tod[e], n = o->n_ports[e], occ = 0;
        for (int64_t i = o->port_off[e]; i < o->port_off[e + 1]; ++i) occ += o->trem[i] > 0;
        ob[0] = sin(two_pi * t / p->ep_len);
        ob[1] = cos(two_pi * t / p->ep_len);
        ob[2] = o->price[(size_t)o->day[e] * (size_t)p->ep_len + (size_t)t];
        ob[3] = p->p_sell;
        ob[4] = (double)occ / n;
        ob[5] = (double)o->day[e] / o->n_days;
        ob[6] = (double)t / p->ep_len;
        ob[7] = (o->day[e] % 7) < 5 ? 1.0 : 0.0;
        if (p->v2g) {
            ob[8] = o->bsoc[e];
            ob[9] = p->batt_rate_kw > 0.0 ? o->bp[e] / p->batt_rate_kw : 0.0;
        }
        for (int32_t q = 0; q < n; ++q) {
            int64_t i = o->port_off[e] + q;
            double *op = ob + F + Q * q;
            double pmax = p->p_max_kw[o->port_type[i]];
            int on = o->trem[i] > 0, cs = o->trem[i] == ORC_TREM_CS;
            op[0] = on ? 1.0 : 0.0;
            op[1] = o->soc[i];
            op[2] = (double)(cs ? o->due[i] : o->trem[i]) / p->stay_steps[1];
            op[3] = on ? orc_taper(o->soc[i], o->rbar[i], p->tau) / pmax : 0.0;
            op[4] = o->pw[i] / pmax;
            op[5] = o->erem[i] / p->cap_kwh[1];
            if (Q == 7) op[6] = cs ? 1.0 : 0.0;
        }
    }
}

/* State access in batch order: per port soc, erem, cap, rbar, p, trem; per
 * env step-of-day, day, global step, car count, key words, running episode
 * return. */
void orc_get_state(const orc *o, double *soc, double *erem, double *cap, double *rbar, double *pw,
                   int32_t *trem, int32_t *tod, int32_t *day, uint32_t *gstep, uint32_t *ncar, uint32_t *key0,
                   uint32_t *key1, double *ep_ret)
{
    size_t P = (size_t)o->P, E = (size_t)o->E;
    memcpy(soc, o->soc, P * sizeof(double)); memcpy(erem, o->erem, P * sizeof(double));
    memcpy(cap, o->cap, P * sizeof(double)); memcpy(rbar, o->rbar, P * sizeof(double));
    memcpy(pw, o->pw, P * sizeof(double)); memcpy(trem, o->trem, P * sizeof(int32_t));
    memcpy(tod, o->tod, E * sizeof(int32_t)); memcpy(day, o->day, E * sizeof(int32_t));
    memcpy(gstep, o->gstep, E * sizeof(uint32_t)); memcpy(key0, o->key0, E * sizeof(uint32_t));
    memcpy(ncar, o->ncar, E * sizeof(uint32_t));
    memcpy(key1, o->key1, E * sizeof(uint32_t)); memcpy(ep_ret, o->ep_ret, E * sizeof(double));
}

void orc_set_state(orc *o, const double *soc, const double *erem, const double *cap, const double *rbar,
                   const double *pw, const int32_t *trem, const int32_t *tod, const int32_t *day,
                   const uint32_t *gstep, const uint32_t *ncar, const uint32_t *key0, const uint32_t *key1,
                   const double *ep_ret)
{
    size_t P = (size_t)o->P, E = (size_t)o->E;
    memcpy(o->soc, soc, P * sizeof(double)); memcpy(o->erem, erem, P * sizeof(double));
    memcpy(o->cap, cap, P * sizeof(double)); memcpy(o->rbar, rbar, P * sizeof(double));
    memcpy(o->pw, pw, P * sizeof(double)); memcpy(o->trem, trem, P * sizeof(int32_t));
    memcpy(o->tod, tod, E * sizeof(int32_t)); memcpy(o->day, day, E * sizeof(int32_t));
    memcpy(o->gstep, gstep, E * sizeof(uint32_t)); memcpy(o->key0, key0, E * sizeof(uint32_t));
    memcpy(o->ncar, ncar, E * sizeof(uint32_t));
    memcpy(o->key1, key1, E * sizeof(uint32_t)); memcpy(o->ep_ret, ep_ret, E * sizeof(double));
}

/* Record of the last step per env: M, admitted, departed, c_sat, c_con,
 * E_net, E_grid, price, and the summed pre-rescale power. */
void orc_get_info(const orc *o, int32_t *M, int32_t *admitted, int32_t *departed, double *csat,
                  double *ccon, double *enet, double *egrid, double *price, double *req_sum)
{
    size_t E = (size_t)o->E;
    memcpy(M, o->inf_M, E * sizeof(int32_t)); memcpy(admitted, o->inf_admitted, E * sizeof(int32_t));
    memcpy(departed, o->inf_departed, E * sizeof(int32_t));
    memcpy(csat, o->inf_csat, E * sizeof(double)); memcpy(ccon, o->inf_ccon, E * sizeof(double));
    memcpy(enet, o->inf_enet, E * sizeof(double)); memcpy(egrid, o->inf_egrid, E * sizeof(double));
    memcpy(price, o->inf_price, E * sizeof(double)); memcpy(req_sum, o->inf_req_sum, E * sizeof(double));
}

/* Running statistics per env: cars admitted, cars rejected, kWh missing at
 * departure, kWh charged, finished episodes, last episode return. */
void orc_get_stats(const orc *o, double *arrived, double *rejected, double *missing, double *charged,
                   uint32_t *n_episodes, double *last_ret)
{
    size_t E = (size_t)o->E;
    memcpy(arrived, o->st_arrived, E * sizeof(double)); memcpy(rejected, o->st_rejected, E * sizeof(double));
    memcpy(missing, o->st_missing, E * sizeof(double)); memcpy(charged, o->st_charged, E * sizeof(double));
    memcpy(n_episodes, o->n_episodes, E * sizeof(uint32_t)); memcpy(last_ret, o->last_ret, E * sizeof(double));
}

/* Give env e the Philox stream id ids[e] (the env's index in a larger batch
 * when this oracle simulates a subset of it), then reset all envs. */
void orc_set_streams(orc *o, const uint32_t *ids, uint64_t seed)
{
    memcpy(o->stream, ids, (size_t)o->E * sizeof(uint32_t));
    orc_reset(o, NULL, 0, seed);
}

/* Station battery state per env (V2G mode): SoC and last applied power. */
void orc_get_battery(const orc *o, double *soc, double *pw)
{
    memcpy(soc, o->bsoc, (size_t)o->E * sizeof(double));
    memcpy(pw, o->bp, (size_t)o->E * sizeof(double));
}
void orc_set_battery(orc *o, const double *soc, const double *pw)
{
    memcpy(o->bsoc, soc, (size_t)o->E * sizeof(double));
    memcpy(o->bp, pw, (size_t)o->E * sizeof(double));
}

/* Delta t_remain of charge-sensitive cars per port (0 elsewhere). */
void orc_get_due(const orc *o, int32_t *due) { memcpy(due, o->due, (size_t)o->P * sizeof(int32_t)); }
void orc_set_due(orc *o, const int32_t *due) { memcpy(o->due, due, (size_t)o->P * sizeof(int32_t)); }

/* c_Sat,1 of the last step per env, and the smallest relative distance
 * |Delta E_remain - eps_cap C| / (eps_cap C) of a tested charge-sensitive
 * car from the departure threshold (1e300 when none was tested). */
void orc_get_info_cs(const orc *o, double *csat1, double *margin)
{
    memcpy(csat1, o->inf_csat1, (size_t)o->E * sizeof(double));
    memcpy(margin, o->inf_cs_margin, (size_t)o->E * sizeof(double));
}

/* V2G terms of the last step per env: energy pushed into the grid by cars
 * (<= 0, after port losses), battery energy, degradation cost basis, and
 * Delta E_grid,net. */
void orc_get_info_v2g(const orc *o, double *e_to, double *e_b, double *degrad, double *e_grid_net)
{
    size_t E = (size_t)o->E;
    memcpy(e_to, o->inf_eto, E * sizeof(double)); memcpy(e_b, o->inf_eb, E * sizeof(double));
    memcpy(degrad, o->inf_degrad, E * sizeof(double)); memcpy(e_grid_net, o->inf_egrid_net, E * sizeof(double));
}

/* the per-step power of each port (after rescaling) of the last step */
void orc_get_power(const orc *o, double *pw) { memcpy(pw, o->pw, (size_t)o->P * sizeof(double)); }
