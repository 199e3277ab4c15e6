/*
 * qs_oracle.c -- plain, slow FP64 CPU oracle of the QuadSwarm forward-dynamics
 * step (Huang et al., "QuadSwarm: A Modular Multi-Quadrotor Simulator for Deep
 * Reinforcement Learning with Direct Thrust Control", arXiv 2306.09537).
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library. The product path (the CUDA
 * library) never calls it, and the two share no source, header, table or
 * constant generator.
 *
 * Scope and order of one control step (paper Sec. III-A .. III-E, IV):
 *   for each substep s (physics at 200 Hz, two per 100 Hz control step, Sec. IV):
 *     per drone: S1 motor command + lag (Sec. III-A "Motor Lag"),
 *                S2 motor noise + thrust (Sec. III-A "Motor Noise"),
 *                S3 wrench from the rotor layout (Sec. III-A dynamics block),
 *                S4 linear dynamics with floor friction (Sec. III-A, III-B "Ground"),
 *                S5 angular (Euler) dynamics (Sec. III-A dynamics block),
 *                S6 semi-implicit Euler + re-orthonormalisation,
 *                S7 floor hit (Sec. III-B "Ground"),
 *                S8 wall / ceiling contact (Sec. III-B "Wall or Ceiling")
 *   S9  pair pass: which pairs of an environment collide (Sec. III-B "Quad-Quad")
 *   S10 collision response (Sec. III-B "Quad-Quad" equation block)
 *   S11 K nearest neighbours (Sec. II-B, III-C)
 *   S12 observation with sensor noise (Sec. III-C)
 *   S13 reward (Sec. III-E) and done (15 s episodes, Sec. IV)
 *
 * Where the paper is silent or garbled this file takes the readings listed in
 * the repository's design notes; each is restated at the point of use.
 *
 * Floating point: everything is double, except the canonical pair key (S9,
 * S11), which is evaluated in binary32 on binary32-rounded positions so that
 * neighbour indices and collision sets are well defined decisions. Build with
 * -ffp-contract=off and without -ffast-math.
 *
 * Two options go beyond the paper: OR_F_EVENT_TIME resolves each detected
 * contact at its crossing time within the substep or step (a variant of the
 * model whose gradients carry the crossing-time terms), and OR_F_ROUND32 /
 * OR_F_ROUND32_SR round the state to binary32 after every substep, an
 * instrument the tests use to measure how strongly a trajectory amplifies
 * perturbations of binary32 size. Neither is on by default.
 *
 * Parity unpinned (no closed form or printed value constrains them): the
 * reward weights' semantics, the friction constant mu, the collision constants
 * and the sensor-noise reading; the tests only check them for self-consistency
 * and against hand-derived single cases.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "qs_oracle.h"

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11): a 4x32-bit counter, a 2x32-bit key, ten rounds   */
/* of two 32x32->64 multiplies with the Weyl key schedule between rounds.     */
/* ------------------------------------------------------------------------- */
static const uint32_t PH_MUL0 = 0xD2511F53u, PH_MUL1 = 0xCD9E8D57u;
static const uint32_t PH_WEYL0 = 0x9E3779B9u, PH_WEYL1 = 0xBB67AE85u;

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PH_WEYL0; k1 += PH_WEYL1; }
        uint64_t prod0 = (uint64_t)PH_MUL0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)PH_MUL1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* n blocks: out[4 i .. 4 i + 3] = or_philox4x32_10(ctr[4 i .. 4 i + 3], key). */
void or_philox4x32_10_n(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, size_t n) {
    for (size_t i = 0; i < n; ++i) or_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* u = (2k+1) / 2^24 with k = the top 23 bits of r: strictly inside (0,1) and
 * exactly representable in binary32 and binary64 alike. */
double or_uniform(uint32_t r) { return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Box-Muller (1958): two independent N(0,1) from two uniforms. */
static void box_muller(double u0, double u1, double* n0, double* n1) {
    double rho = sqrt(-2.0 * log(u0));
    double ang = 2.0 * M_PI * u1;
    *n0 = rho * cos(ang);
    *n1 = rho * sin(ang);
}

/* One Philox block at counter (tick, id, tag<<16 | sub<<8 | blk, 0). */
static void draw_block(const or_env* h, uint32_t tick, uint32_t id, uint32_t tag, uint32_t sub,
                       uint32_t blk, double u[4]) {
    uint32_t ctr[4] = {tick, id, (tag << 16) | (sub << 8) | blk, 0u};
    uint32_t key[2] = {h->key[0], h->key[1]};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) u[i] = or_uniform(r[i]);
}

static void draw_block_key(const uint32_t key_in[2], uint32_t tick, uint32_t id, uint32_t tag,
                           uint32_t sub, uint32_t blk, double u[4]) {
    uint32_t ctr[4] = {tick, id, (tag << 16) | (sub << 8) | blk, 0u};
    uint32_t key[2] = {key_in[0], key_in[1]};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) u[i] = or_uniform(r[i]);
}

/* Six N(0,1) draws (collision / wall perturbation): blocks 0 and 1. */
static void draw_six_normals(const or_env* h, uint32_t tick, uint32_t id, uint32_t tag,
                             uint32_t sub, double n[6]) {
    double u[4], w[4], spare;
    draw_block(h, tick, id, tag, sub, 0, u);
    draw_block(h, tick, id, tag, sub, 1, w);
    box_muller(u[0], u[1], &n[0], &n[1]);
    box_muller(u[2], u[3], &n[2], &n[3]);
    box_muller(w[0], w[1], &n[4], &n[5]);
    (void)spare;
}

/* ------------------------------------------------------------------------- */
/* Small 3x3 helpers (row-major).                                             */
/* ------------------------------------------------------------------------- */
static double det3(const double m[9]) {
    return m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
           m[2] * (m[3] * m[7] - m[4] * m[6]);
}

/* inverse-transpose: (M^{-1})^T = cofactor(M) / det(M) */
static void inv_transpose3(const double m[9], double out[9]) {
    double d = det3(m);
    out[0] = (m[4] * m[8] - m[5] * m[7]) / d;
    out[1] = -(m[3] * m[8] - m[5] * m[6]) / d;
    out[2] = (m[3] * m[7] - m[4] * m[6]) / d;
    out[3] = -(m[1] * m[8] - m[2] * m[7]) / d;
    out[4] = (m[0] * m[8] - m[2] * m[6]) / d;
    out[5] = -(m[0] * m[7] - m[1] * m[6]) / d;
    out[6] = (m[1] * m[5] - m[2] * m[4]) / d;
    out[7] = -(m[0] * m[5] - m[2] * m[3]) / d;
    out[8] = (m[0] * m[4] - m[1] * m[3]) / d;
}

/* Orthogonal polar factor of a nonsingular M with det M > 0: the unique
 * rotation R with M = R H, H symmetric positive definite. Computed by Newton's
 * polar iteration X <- (X + X^{-T}) / 2 (Higham 1986), run until it stops
 * moving in binary64. This is the "nearest rotation" that the re-
 * orthonormalisation of the integrated rotation matrix asks for. */
void or_polar(const double m[9], double r[9]) {
    double x[9], it[9];
    memcpy(x, m, sizeof x);
    for (int iter = 0; iter < 60; ++iter) {
        inv_transpose3(x, it);
        double change = 0.0;
        for (int k = 0; k < 9; ++k) {
            double nx = 0.5 * (x[k] + it[k]);
            double dd = fabs(nx - x[k]);
            if (dd > change) change = dd;
            x[k] = nx;
        }
        if (change < 1e-15) break;
    }
    memcpy(r, x, sizeof x);
}

/* ------------------------------------------------------------------------- */
/* Canonical binary32 pair key (S9, S11): with dx = fl32(x_j - x_i) etc.,     */
/* key = fl32(fl32(fl32(dx*dx) + fl32(dy*dy)) + fl32(dz*dz)). No contraction. */
/* ------------------------------------------------------------------------- */
float or_pair_key(const float xi[3], const float xj[3]) {
    volatile float dx = xj[0] - xi[0];
    volatile float dy = xj[1] - xi[1];
    volatile float dz = xj[2] - xi[2];
    volatile float sx = dx * dx;
    volatile float sy = dy * dy;
    volatile float sz = dz * dz;
    volatile float s = sx + sy;
    volatile float k = s + sz;
    return k;
}

/* Collision threshold fl32(fl32(l_i + l_j)^2) for binary32 arm lengths. */
static float pair_threshold(float li, float lj) {
    volatile float r = li + lj;
    volatile float t = r * r;
    return t;
}

/* ------------------------------------------------------------------------- */
/* Environment creation and defaults.                                         */
/* ------------------------------------------------------------------------- */
void or_default_config(or_config* c) {
    memset(c, 0, sizeof *c);
    c->n_envs = 1;
    c->k_neighbors = 6;
    c->substeps = 2;           /* 200 Hz physics under 100 Hz control (Sec. IV) */
    c->dt = 0.005;
    c->episode_steps = 1500;   /* 15 s at 100 Hz (Sec. IV) */
    c->seed = 1;
    c->flags = OR_F_DR | OR_F_MOTOR_NOISE | OR_F_OBS_NOISE | OR_F_COLLISIONS | OR_F_FLOOR |
               OR_F_WALLS;
    /* Crazyflie 2.x nominal values; the paper states none (proposed readings). */
    c->mass = 0.028;
    c->arm = 0.046;
    c->ixx = 1.657e-5;
    c->iyy = 1.666e-5;
    c->izz = 2.926e-5;
    c->t2w = 2.0;
    c->kappa = 0.006;
    c->tau_m = 0.04;
    c->gravity = 9.81;
    c->mu = 0.3;
    c->alpha_nd = 0.9;
    c->alpha_ns_frac = 0.02;
    c->alpha_c = 0.8;
    c->coll_sigma_v = 0.2;
    c->coll_sigma_w = 0.5;
    c->obs_sigma_x = 5e-3;    /* Sec. III-C */
    c->obs_sigma_v = 1e-2;    /* Sec. III-C */
    c->obs_sigma_w = 1.75e-4; /* Sec. III-C */
    c->room_hx = 5.0;
    c->room_hy = 5.0;
    c->room_h = 10.0;
    c->dr_lo = 0.8;
    c->dr_hi = 1.2;
    c->smooth_beta = 200.0;
    c->smooth_kc = 20.0;
    c->prox_factor = 4.0;
    c->omega_max = 40.0;
    /* downwash: a quarter of g on the lower drone at zero separation, fading
     * linearly to zero 0.5 m below the upper one (the paper gives no constants) */
    c->dw_k1 = 2.4525;
    c->dw_k2 = -2.0;
    c->dw_b1 = 1.0;
    c->dw_height = 0.5;
    c->dw_sigma_a = 0.1;
    c->dw_sigma_w = 1.0;
    /* scenarios (Sec. III-D gives no sizes or rates): goals 0.5 m apart, circle
     * radius at most 4 m, centres 1.5 m clear of the room's faces, shrink to
     * half size and back every 4 s, evader loops at about 0.1 Hz, 3 s Bezier
     * segments */
    c->scenarios = 0;
    c->form_spacing = 0.5;
    c->form_rmax = 4.0;
    c->scn_margin = 1.5;
    c->se_min = 0.5;
    c->se_period = 400.0;
    c->liss_f = 0.1;
    c->bez_seg = 300.0;
    /* goal-reaching weights: position, spin, and each collision indicator */
    c->w[OR_W_POS] = -1.0;
    c->w[OR_W_SPIN] = -0.1;
    c->w[OR_W_HIT_FLOOR] = -1.0;
    c->w[OR_W_HIT_WALL] = -1.0;
    c->w[OR_W_HIT_CEIL] = -1.0;
    c->w[OR_W_HIT_QUAD] = -1.0;
}

or_env* or_create(const or_config* cfg, const int32_t* swarm_sizes) {
    if (!cfg || cfg->n_envs <= 0 || cfg->substeps <= 0 || cfg->substeps > 255) return NULL;
    or_env* h = (or_env*)calloc(1, sizeof(or_env));
    h->cfg = *cfg;
    int E = cfg->n_envs;
    h->env_off = (int32_t*)calloc((size_t)E + 1, sizeof(int32_t));
    for (int e = 0; e < E; ++e) {
        int n = swarm_sizes ? swarm_sizes[e] : 1;
        if (n <= 0) { free(h->env_off); free(h); return NULL; }
        h->env_off[e + 1] = h->env_off[e] + n;
    }
    int D = h->env_off[E];
    h->n_drones = D;
    h->prm = (double*)calloc((size_t)E * OR_NPRM, sizeof(double));
    h->goal = (double*)calloc((size_t)E * 3, sizeof(double));
    h->scn = (double*)calloc((size_t)E * OR_NSCN, sizeof(double));
    h->st = (double*)calloc((size_t)D * OR_NST, sizeof(double));
    h->ep_t = (int32_t*)calloc((size_t)E, sizeof(int32_t));
    h->tick = (uint32_t*)calloc((size_t)E, sizeof(uint32_t));
    h->ev = (uint32_t*)calloc((size_t)D, sizeof(uint32_t));
    int K = cfg->k_neighbors > 0 ? cfg->k_neighbors : 1;
    h->knn = (int32_t*)calloc((size_t)D * K, sizeof(int32_t));
    h->margin = (double*)calloc((size_t)D, sizeof(double));
    h->margin_knn = (double*)calloc((size_t)D, sizeof(double));
    h->cond = (double*)calloc((size_t)D, sizeof(double));
    h->key[0] = (uint32_t)(cfg->seed & 0xffffffffu);
    h->key[1] = (uint32_t)(cfg->seed >> 32);
    for (int d = 0; d < D; ++d) h->margin[d] = h->margin_knn[d] = h->cond[d] = INFINITY;
    return h;
}

void or_destroy(or_env* h) {
    if (!h) return;
    free(h->env_off); free(h->prm); free(h->goal); free(h->scn); free(h->st); free(h->ep_t); free(h->tick);
    free(h->ev); free(h->knn); free(h->margin); free(h->margin_knn); free(h->cond); free(h);
}

int or_n_drones(const or_env* h) { return h->n_drones; }

static double hover_command(const double* prm) { return 1.0 / prm[OR_P_T2W]; }

/* S0: per-environment domain randomisation and goal. Independent U(lo,hi)
 * scale factors on m, Ixx, Iyy, Izz, t2w, tau_m and l (one draw per env, all
 * drones of the env share them); goal uniform in the room. */
static void reset_env_params(or_env* h, const uint32_t key[2], uint32_t tick, uint32_t tag, int e) {
    const or_config* c = &h->cfg;
    double u[12];
    draw_block_key(key, tick, (uint32_t)e, tag, 0, 0, u);
    draw_block_key(key, tick, (uint32_t)e, tag, 0, 1, u + 4);
    draw_block_key(key, tick, (uint32_t)e, tag, 0, 2, u + 8);
    double nominal[OR_NPRM] = {c->mass, c->ixx, c->iyy, c->izz, c->t2w, c->tau_m, c->arm};
    double* p = h->prm + (size_t)e * OR_NPRM;
    for (int k = 0; k < OR_NPRM; ++k) {
        double scale = (c->flags & OR_F_DR) ? c->dr_lo + (c->dr_hi - c->dr_lo) * u[k] : 1.0;
        p[k] = nominal[k] * scale;
    }
    double* g = h->goal + (size_t)e * 3;
    g[0] = -c->room_hx + 2.0 * c->room_hx * u[7];
    g[1] = -c->room_hy + 2.0 * c->room_hy * u[8];
    g[2] = c->room_h * u[9];
}

/* ------------------------------------------------------------------------- */
/* Training scenarios (Sec. III-D): goal formations and their schedules.      */
/* ------------------------------------------------------------------------- */

/* smallest m >= 1 with m^p >= n (p = 2 or 3) */
static int root_ceil(int n, int p) {
    int m = 1;
    while ((p == 2 ? m * m : m * m * m) < n) ++m;
    return m;
}

/* The golden angle (3 - sqrt 5) / 2 turns as a 32-bit fixed-point fraction, so
 * that k times it, taken modulo one turn, is exact integer arithmetic. */
static uint32_t golden_turn_q32(void) { return (uint32_t)floor(4294967296.0 * (3.0 - sqrt(5.0)) / 2.0); }

/* Offset from the formation's centre of goal slot k (0 <= k < n) of a
 * formation of n goals with spacing s.
 *   circle:   n goals evenly on a horizontal circle, each an arc s from the
 *             next (radius s n / 2 pi, at most rmax);
 *   grid:     a horizontal square grid of side m = ceil(sqrt n), filled row by
 *             row, centred on its occupied rows;
 *   sphere:   the Fibonacci lattice: heights z_k = 1 - (2k+1)/n, azimuth
 *             advancing by the golden angle, radius s sqrt(n / 4 pi) (area s^2
 *             per goal);
 *   cylinder: L horizontal rings (L the smallest with 4 L^2 >= n) of
 *             m = ceil(n / L) goals each, radius as for a circle of m goals,
 *             rings s apart and centred on the occupied ones;
 *   cube:     a cubic grid of side m = ceil(cbrt n), filled along x, then y,
 *             then z, centred on its occupied layers. */
void or_formation_offset(int form, int k, int n, double s, double rmax, double out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    if (form == OR_FORM_CIRCLE) {
        double r = fmin(s * n / (2.0 * M_PI), rmax), th = 2.0 * M_PI * k / n;
        out[0] = r * cos(th);
        out[1] = r * sin(th);
    } else if (form == OR_FORM_GRID) {
        int m = root_ceil(n, 2), rows = (n + m - 1) / m;
        out[0] = s * ((k % m) - 0.5 * (m - 1));
        out[1] = s * ((k / m) - 0.5 * (rows - 1));
    } else if (form == OR_FORM_SPHERE) {
        double r = s * sqrt(n / (4.0 * M_PI));
        double z = 1.0 - (2.0 * k + 1.0) / n, rho = sqrt(1.0 - z * z);
        uint32_t turn = (uint32_t)k * golden_turn_q32(); /* modulo 2^32: one turn */
        double phi = 2.0 * M_PI * (turn / 4294967296.0);
        out[0] = r * rho * cos(phi);
        out[1] = r * rho * sin(phi);
        out[2] = r * z;
    } else if (form == OR_FORM_CYLINDER) {
        int L = 1;
        while (4 * L * L < n) ++L;
        int m = (n + L - 1) / L, used = (n + m - 1) / m;
        double r = fmin(s * m / (2.0 * M_PI), rmax), th = 2.0 * M_PI * (k % m) / m;
        out[0] = r * cos(th);
        out[1] = r * sin(th);
        out[2] = s * ((k / m) - 0.5 * (used - 1));
    } else if (form == OR_FORM_CUBE) {
        int m = root_ceil(n, 3), layers = (n + m * m - 1) / (m * m);
        out[0] = s * ((k % m) - 0.5 * (m - 1));
        out[1] = s * (((k / m) % m) - 0.5 * (m - 1));
        out[2] = s * ((k / (m * m)) - 0.5 * (layers - 1));
    }
}

/* floor(top24(r) * n / 2^24): an exact uniform integer choice in [0, n) */
static uint32_t pick(uint32_t r, uint32_t n) { return (uint32_t)(((uint64_t)(r >> 8) * n) >> 24); }

static void raw_block(const uint32_t key_in[2], uint32_t c0, uint32_t c1, uint32_t c2, uint32_t r[4]) {
    uint32_t ctr[4] = {c0, c1, c2, 0u};
    uint32_t key[2] = {key_in[0], key_in[1]};
    or_philox4x32_10(ctr, key, r);
}

/* S0: scenario record of env e, five Philox blocks at (tick, e, tag << 16 |
 * block). The type is uniform over the enabled ones, each formation uniform
 * over the five, the switch step uniform in [T/4, 3T/4] (T the episode
 * length; at least 1), the centres uniform in the room shrunk by the
 * clearance m on every face; a 32-bit seed keys the evader's waypoints and
 * the swap permutation. Lissajous: centre uniform within 1 m (per axis) of the
 * room's middle, amplitude U(0.5, 1) times the half-extent the clearance
 * leaves, frequency U(0.5, 1.5) times the base, phase U(0, 1) turns. With
 * only the single goal enabled the record stays zero and draws nothing. */
static void draw_scenario(or_env* h, const uint32_t key[2], uint32_t tick, uint32_t tag, int e) {
    const or_config* c = &h->cfg;
    double* rec = h->scn + (size_t)e * OR_NSCN;
    for (int k = 0; k < OR_NSCN; ++k) rec[k] = 0.0;
    const uint32_t mask = c->scenarios & ((1u << OR_NSCN_TYPES) - 1u);
    if ((mask & ~1u) == 0) return;
    uint32_t r[5][4];
    for (uint32_t b = 0; b < 5; ++b) raw_block(key, tick, (uint32_t)e, (tag << 16) | b, r[b]);
    uint32_t n_en = 0;
    for (int t = 0; t < OR_NSCN_TYPES; ++t) n_en += (mask >> t) & 1u;
    uint32_t idx = pick(r[0][0], n_en);
    int type = 0;
    for (int t = 0; t < OR_NSCN_TYPES; ++t) {
        if (!((mask >> t) & 1u)) continue;
        if (idx == 0) { type = t; break; }
        --idx;
    }
    rec[OR_R_TYPE] = type;
    rec[OR_R_F0] = pick(r[0][1], OR_NFORM);
    rec[OR_R_F1] = pick(r[0][2], OR_NFORM);
    int lo = c->episode_steps / 4, hi = 3 * c->episode_steps / 4;
    if (lo < 1) lo = 1;
    if (hi < lo) hi = lo;
    rec[OR_R_TSW] = lo + (int)pick(r[0][3], (uint32_t)(hi - lo + 1));
    rec[OR_R_SEED_LO] = r[1][3] & 0xffffu;
    rec[OR_R_SEED_HI] = r[1][3] >> 16;
    const double m = c->scn_margin, hx = c->room_hx, hy = c->room_hy, hz = c->room_h;
    if (type == OR_SCN_PURSUIT_LISSAJOUS) {
        const double a[3] = {hx - m, hy - m, 0.5 * hz - m};
        rec[OR_R_C0 + 0] = -1.0 + 2.0 * or_uniform(r[1][0]);
        rec[OR_R_C0 + 1] = -1.0 + 2.0 * or_uniform(r[1][1]);
        rec[OR_R_C0 + 2] = 0.5 * hz - 1.0 + 2.0 * or_uniform(r[1][2]);
        for (int k = 0; k < 3; ++k) {
            rec[OR_R_C1 + k] = a[k] * (0.5 + 0.5 * or_uniform(r[2][k]));
            rec[OR_R_FREQ + k] = c->liss_f * (0.5 + or_uniform(r[3][k]));
            rec[OR_R_PHASE + k] = or_uniform(r[4][k]);
        }
    } else {
        for (int q = 0; q < 2; ++q) {
            double* cc = rec + (q ? OR_R_C1 : OR_R_C0);
            const uint32_t* rr = r[1 + q];
            cc[0] = -hx + m + 2.0 * (hx - m) * or_uniform(rr[0]);
            cc[1] = -hy + m + 2.0 * (hy - m) * or_uniform(rr[1]);
            cc[2] = m + (hz - 2.0 * m) * or_uniform(rr[2]);
        }
    }
}

static uint32_t rec_seed(const double* rec) {
    return (uint32_t)rec[OR_R_SEED_LO] | ((uint32_t)rec[OR_R_SEED_HI] << 16);
}

/* Goal slot of drone i after a swap: the rank of its key among the N keys of
 * the env (ties to the lower index), key_j = first word of the Philox block at
 * (seed, j, SWAP << 16) -- a uniformly random permutation of the slots. */
static int swap_slot(const or_env* h, uint32_t seed, int i, int N) {
    uint32_t r[4], ki;
    raw_block(h->key, seed, (uint32_t)i, OR_TAG_SWAP << 16, r);
    ki = r[0];
    int rank = 0;
    for (int j = 0; j < N; ++j) {
        raw_block(h->key, seed, (uint32_t)j, OR_TAG_SWAP << 16, r);
        if (r[0] < ki || (r[0] == ki && j < i)) ++rank;
    }
    return rank;
}

/* Evader waypoint j >= -1: uniform in the room shrunk by the clearance, from
 * the Philox block at (seed, j + 1, WAYPOINT << 16). */
static void waypoint(const or_env* h, uint32_t seed, int j, double w[3]) {
    const or_config* c = &h->cfg;
    const double m = c->scn_margin;
    uint32_t r[4];
    raw_block(h->key, seed, (uint32_t)(j + 1), OR_TAG_WAYPOINT << 16, r);
    w[0] = -c->room_hx + m + 2.0 * (c->room_hx - m) * or_uniform(r[0]);
    w[1] = -c->room_hy + m + 2.0 * (c->room_hy - m) * or_uniform(r[1]);
    w[2] = m + (c->room_h - 2.0 * m) * or_uniform(r[2]);
}

/* Goal of local drone i (of N) of env e at control step tau of its episode.
 *   single:          the env's goal;
 *   static:          formation F0 around centre 0;
 *   dynamic goals:   from the switch step on, formation F1 around centre 1;
 *   swap goals:      from the switch step on, drone i takes slot swap_slot(i);
 *   shrink & expand: formation F0 scaled by 1 - (1 - se_min)(1 - cos(2 pi tau / P)) / 2;
 *   swarm vs swarm:  the first ceil(N/2) drones form group 0, the rest group 1,
 *                    each a formation of its own size; group g is around centre g
 *                    in F0, and from the switch step on around the other
 *                    group's centre in F1;
 *   Lissajous:       every drone chases c + A sin(2 pi (f tau T + phase)) per axis,
 *                    T = substeps dt the control period;
 *   Bezier:          every drone chases a point moving through the waypoints, one
 *                    per S = bez_seg control steps: on segment q = floor(tau / S)
 *                    the cubic Bezier curve from W_q to W_{q+1} with inner control
 *                    points W_q + (W_{q+1} - W_{q-1})/6 and W_{q+1} - (W_{q+2} - W_q)/6
 *                    (Catmull-Rom tangents, so the path is C1), at u = (tau - qS)/S. */
static void drone_goal(const or_env* h, int e, int i, int N, int tau, double g[3]) {
    const or_config* c = &h->cfg;
    const double* rec = h->scn + (size_t)e * OR_NSCN;
    const int type = (int)rec[OR_R_TYPE];
    if ((c->scenarios & ~1u) == 0 || type == OR_SCN_SINGLE) {
        for (int k = 0; k < 3; ++k) g[k] = h->goal[(size_t)e * 3 + k];
        return;
    }
    const double s = c->form_spacing, rmax = c->form_rmax;
    const int sw = tau >= (int)rec[OR_R_TSW];
    const int f0 = (int)rec[OR_R_F0], f1 = (int)rec[OR_R_F1];
    const double *c0 = rec + OR_R_C0, *c1 = rec + OR_R_C1;
    double off[3];
    if (type == OR_SCN_STATIC || type == OR_SCN_SHRINK_EXPAND) {
        or_formation_offset(f0, i, N, s, rmax, off);
        double lam = 1.0;
        if (type == OR_SCN_SHRINK_EXPAND)
            lam = 1.0 - (1.0 - c->se_min) * 0.5 * (1.0 - cos(2.0 * M_PI * tau / c->se_period));
        for (int k = 0; k < 3; ++k) g[k] = c0[k] + lam * off[k];
    } else if (type == OR_SCN_DYNAMIC) {
        or_formation_offset(sw ? f1 : f0, i, N, s, rmax, off);
        for (int k = 0; k < 3; ++k) g[k] = (sw ? c1[k] : c0[k]) + off[k];
    } else if (type == OR_SCN_SWAP) {
        const int slot = sw ? swap_slot(h, rec_seed(rec), i, N) : i;
        or_formation_offset(f0, slot, N, s, rmax, off);
        for (int k = 0; k < 3; ++k) g[k] = c0[k] + off[k];
    } else if (type == OR_SCN_SWARM_VS_SWARM) {
        const int n0 = (N + 1) / 2, grp = i >= n0;
        const int kk = i - grp * n0, ng = grp ? N - n0 : n0;
        or_formation_offset(sw ? f1 : f0, kk, ng, s, rmax, off);
        const double* cc = (grp ^ sw) ? c1 : c0;
        for (int k = 0; k < 3; ++k) g[k] = cc[k] + off[k];
    } else if (type == OR_SCN_PURSUIT_LISSAJOUS) {
        const double T = c->substeps * c->dt;
        for (int k = 0; k < 3; ++k) {
            double p = rec[OR_R_FREQ + k] * tau * T + rec[OR_R_PHASE + k];
            g[k] = c0[k] + c1[k] * sin(2.0 * M_PI * (p - floor(p)));
        }
    } else if (type == OR_SCN_PURSUIT_BEZIER) {
        const int S = (int)c->bez_seg, q = tau / S;
        const double u = (double)(tau - q * S) / S, v = 1.0 - u;
        const uint32_t seed = rec_seed(rec);
        double wm[3], w0[3], w1[3], w2[3];
        waypoint(h, seed, q - 1, wm);
        waypoint(h, seed, q, w0);
        waypoint(h, seed, q + 1, w1);
        waypoint(h, seed, q + 2, w2);
        for (int k = 0; k < 3; ++k) {
            double p1 = w0[k] + (w1[k] - wm[k]) / 6.0, p2 = w1[k] - (w2[k] - w0[k]) / 6.0;
            g[k] = v * v * v * w0[k] + 3.0 * v * v * u * p1 + 3.0 * v * u * u * p2 + u * u * u * w1[k];
        }
    } else {
        for (int k = 0; k < 3; ++k) g[k] = h->goal[(size_t)e * 3 + k];
    }
}

/* S0: per-drone initial state. Position uniform in the room, velocity and
 * body rates uniform in [-1,1], orientation from a uniformly random unit
 * quaternion (Shoemake, "Uniform random rotations", Graphics Gems III, 1992),
 * filtered rotor speed at hover, motor noise zero, previous command = hover. */
static void reset_drone(or_env* h, const uint32_t key[2], uint32_t tick, uint32_t tag, int e, int d) {
    const or_config* c = &h->cfg;
    double u[12];
    draw_block_key(key, tick, (uint32_t)d, tag, 0, 0, u);
    draw_block_key(key, tick, (uint32_t)d, tag, 0, 1, u + 4);
    draw_block_key(key, tick, (uint32_t)d, tag, 0, 2, u + 8);
    double* s = h->st + (size_t)d * OR_NST;
    const double* p = h->prm + (size_t)e * OR_NPRM;
    s[OR_S_X + 0] = -c->room_hx + 2.0 * c->room_hx * u[0];
    s[OR_S_X + 1] = -c->room_hy + 2.0 * c->room_hy * u[1];
    s[OR_S_X + 2] = c->room_h * u[2];
    s[OR_S_V + 0] = -1.0 + 2.0 * u[3];
    s[OR_S_V + 1] = -1.0 + 2.0 * u[4];
    s[OR_S_V + 2] = -1.0 + 2.0 * u[5];
    double a = sqrt(1.0 - u[6]), b = sqrt(u[6]);
    double qx = a * sin(2.0 * M_PI * u[7]);
    double qy = a * cos(2.0 * M_PI * u[7]);
    double qz = b * sin(2.0 * M_PI * u[8]);
    double qw = b * cos(2.0 * M_PI * u[8]);
    double* R = s + OR_S_R;
    R[0] = 1.0 - 2.0 * (qy * qy + qz * qz);
    R[1] = 2.0 * (qx * qy - qz * qw);
    R[2] = 2.0 * (qx * qz + qy * qw);
    R[3] = 2.0 * (qx * qy + qz * qw);
    R[4] = 1.0 - 2.0 * (qx * qx + qz * qz);
    R[5] = 2.0 * (qy * qz - qx * qw);
    R[6] = 2.0 * (qx * qz - qy * qw);
    R[7] = 2.0 * (qy * qz + qx * qw);
    R[8] = 1.0 - 2.0 * (qx * qx + qy * qy);
    s[OR_S_W + 0] = -1.0 + 2.0 * u[9];
    s[OR_S_W + 1] = -1.0 + 2.0 * u[10];
    s[OR_S_W + 2] = -1.0 + 2.0 * u[11];
    double hov = hover_command(p);
    for (int r = 0; r < 4; ++r) {
        s[OR_S_UF + r] = sqrt(hov);
        s[OR_S_EPS + r] = 0.0;
        s[OR_S_FPREV + r] = hov;
    }
}

static void reset_env_all(or_env* h, const uint32_t key[2], uint32_t tick, uint32_t tag_env,
                          uint32_t tag_drone, int e) {
    reset_env_params(h, key, tick, tag_env, e);
    draw_scenario(h, key, tick, tag_env == OR_TAG_AUTO_ENV ? OR_TAG_AUTO_SCN : OR_TAG_SCN, e);
    for (int d = h->env_off[e]; d < h->env_off[e + 1]; ++d) reset_drone(h, key, tick, tag_drone, e, d);
    h->ep_t[e] = 0;
}

/* Full reset (mask == NULL): new key from seed, every env's counter back to
 * 0 and every env redrawn at counter 0. Partial reset: the masked envs are
 * redrawn from key = seed at their current counter; the noise key is kept. */
void or_reset(or_env* h, uint64_t seed, const uint8_t* mask) {
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    if (!mask) {
        h->key[0] = key[0]; h->key[1] = key[1];
        for (int e = 0; e < h->cfg.n_envs; ++e) {
            h->tick[e] = 0;
            reset_env_all(h, key, 0, OR_TAG_RESET_ENV, OR_TAG_RESET_DRONE, e);
        }
    } else {
        for (int e = 0; e < h->cfg.n_envs; ++e)
            if (mask[e]) reset_env_all(h, key, h->tick[e], OR_TAG_RESET_ENV, OR_TAG_RESET_DRONE, e);
    }
    for (int d = 0; d < h->n_drones; ++d) { h->ev[d] = 0; h->margin[d] = h->margin_knn[d] = h->cond[d] = INFINITY; }
}

/* ------------------------------------------------------------------------- */
/* Decision margins: every branch on a continuous quantity records how far    */
/* that quantity was from its threshold (normalised). A binary32 run can take */
/* the other branch only where this margin is at the level of its rounding.   */
/* ------------------------------------------------------------------------- */
static void note_margin(or_env* h, int d, double m) {
    m = fabs(m);
    if (m < h->margin[d]) h->margin[d] = m;
}

/* Margin of the decision a < b (or a <= b): |a - b| / max(|a|, |b|), the
 * relative cancellation that rounding of a and b would have to overcome. An
 * exact tie of exact values (a drone parked at z = 0, clamped onto a wall,
 * at rest) is not a near-decision: both implementations set those exactly. */
static void note_cmp(or_env* h, int d, double a, double b) {
    double den = fmax(fabs(a), fabs(b));
    if (den == 0.0) return;
    note_margin(h, d, (a - b) / den);
}

/* softplus_beta(u) = log(1 + exp(beta u)) / beta, evaluated without overflow */
static double softplus_b(double u, double beta) {
    double z = beta * u;
    return (fmax(z, 0.0) + log1p(exp(-fabs(z)))) / beta;
}

/* ------------------------------------------------------------------------- */
/* One physics substep of one drone (S1 .. S8).                               */
/* pair_acc: smooth-contact pair acceleration (NULL when not in smooth mode). */
/* ------------------------------------------------------------------------- */
static void substep_drone(or_env* h, int e, int d, int sub, const double a_in[4],
                          const double pair_acc[3], double fhat_out[4]) {
    const or_config* c = &h->cfg;
    const double* p = h->prm + (size_t)e * OR_NPRM;
    double* s = h->st + (size_t)d * OR_NST;
    const double dt = c->dt, g = c->gravity;
    const double m = p[OR_P_M], ixx = p[OR_P_IXX], iyy = p[OR_P_IYY], izz = p[OR_P_IZZ];
    const double t2w = p[OR_P_T2W], tau_m = p[OR_P_TAU], arm = p[OR_P_ARM];
    const double fmax = 0.25 * m * g * t2w;                /* per-rotor max thrust */
    const double alpha_lag = 1.0 - exp(-dt / tau_m);       /* 2% settling = tau_m ln 50 */
    const double alpha_ns = c->alpha_ns_frac * m * g / 4.0;
    const int smooth = (c->flags & OR_F_SMOOTH) != 0;

    double* x = s + OR_S_X; double* v = s + OR_S_V; double* R = s + OR_S_R; double* w = s + OR_S_W;
    double* uf = s + OR_S_UF; double* eps = s + OR_S_EPS;

    /* S1: normalised command f^ in [0,1], rotor speed u^ = sqrt(f^), first-order lag. */
    double f[4];
    for (int r = 0; r < 4; ++r) {
        double fh;
        if (c->flags & OR_F_ACTION_SYMMETRIC) {
            double a = a_in[r] < -1.0 ? -1.0 : (a_in[r] > 1.0 ? 1.0 : a_in[r]);
            fh = 0.5 * (a + 1.0);
        } else {
            fh = a_in[r] < 0.0 ? 0.0 : (a_in[r] > 1.0 ? 1.0 : a_in[r]);
        }
        fhat_out[r] = fh;
        double u = sqrt(fh);
        uf[r] = alpha_lag * (u - uf[r]) + uf[r];
    }
    /* S2: AR(1) motor noise, eps <- a_nd eps + a_ns N(0,1); per-rotor thrust. */
    if (c->flags & OR_F_MOTOR_NOISE) {
        double u[4], n[4];
        draw_block(h, h->tick[e], (uint32_t)d, OR_TAG_MOTOR, (uint32_t)sub, 0, u);
        box_muller(u[0], u[1], &n[0], &n[1]);
        box_muller(u[2], u[3], &n[2], &n[3]);
        for (int r = 0; r < 4; ++r) eps[r] = c->alpha_nd * eps[r] + alpha_ns * n[r];
    }
    for (int r = 0; r < 4; ++r) f[r] = fmax * uf[r] * uf[r] + eps[r];

    /* S3: X layout, rotor r at arm*(cos t_r, sin t_r, 0), t_r = 45,135,225,315 deg;
     * thrust along body +z; tau_th = sum p_r x (0,0,f_r); tau_p = (0,0,kappa sum s_r f_r)
     * with spin signs s = (-1,+1,-1,+1). */
    double T = f[0] + f[1] + f[2] + f[3];
    double tau[3] = {0.0, 0.0, 0.0};
    {
        /* cos / sin of 45, 135, 225, 315 degrees are exactly +-1/sqrt(2) */
        const double sx[4] = {1.0, -1.0, -1.0, 1.0}, sy[4] = {1.0, 1.0, -1.0, -1.0};
        const double s = arm * M_SQRT1_2;
        for (int r = 0; r < 4; ++r) {
            double px = s * sx[r], py = s * sy[r];
            tau[0] += py * f[r];
            tau[1] += -px * f[r];
        }
    }
    {
        const double spin[4] = {-1.0, 1.0, -1.0, 1.0};
        for (int r = 0; r < 4; ++r) tau[2] += c->kappa * spin[r] * f[r];
    }

    /* S4: world thrust F = R (0,0,T); acceleration g + F/m. */
    double F[3] = {R[2] * T, R[5] * T, R[8] * T};
    double acc[3] = {F[0] / m, F[1] / m, F[2] / m - g};
    int on_floor = 0, moving = 0;
    if (smooth) {
        double kc = c->smooth_kc * g; /* k_c / m, with k_c = smooth_kc * m g per metre */
        double beta = c->smooth_beta;
        acc[2] += kc * softplus_b(-x[2], beta);                 /* floor */
        acc[2] -= kc * softplus_b(x[2] - c->room_h, beta);      /* ceiling */
        acc[0] -= kc * softplus_b(x[0] - c->room_hx, beta);     /* walls */
        acc[0] += kc * softplus_b(-c->room_hx - x[0], beta);
        acc[1] -= kc * softplus_b(x[1] - c->room_hy, beta);
        acc[1] += kc * softplus_b(-c->room_hy - x[1], beta);
        if (pair_acc) { acc[0] += pair_acc[0]; acc[1] += pair_acc[1]; acc[2] += pair_acc[2]; }
    } else if (c->flags & OR_F_FLOOR) {
        /* Ground, "on the floor": thrust too weak to lift off -> friction arrests the
         * horizontal motion; no vertical motion. */
        if (x[2] <= 0.0) {
            note_cmp(h, d, F[2], m * g);
            if (F[2] < m * g) {
                on_floor = 1;
                h->ev[d] |= OR_EV_ON_FLOOR;
                double ffric = c->mu * (m * g - F[2]);
                double fx = F[0], fy = F[1];
                if (v[0] == 0.0 && v[1] == 0.0) {
                    /* at rest: friction opposes the horizontal thrust, up to its size */
                    double nf = sqrt(fx * fx + fy * fy);
                    note_cmp(h, d, nf, ffric);
                    double keep = nf > ffric ? (nf - ffric) / nf : 0.0;
                    fx *= keep; fy *= keep;
                } else {
                    /* sliding: friction of size mu (m g - F_z) against the velocity */
                    double nv = sqrt(v[0] * v[0] + v[1] * v[1]);
                    fx -= ffric * v[0] / nv;
                    fy -= ffric * v[1] / nv;
                    moving = 1;
                }
                acc[0] = fx / m; acc[1] = fy / m; acc[2] = 0.0;
                v[2] = 0.0;
            }
        }
    }

    /* S5: Euler's equation in the body frame, diagonal inertia. */
    double Iw[3] = {ixx * w[0], iyy * w[1], izz * w[2]};
    double gyro[3] = {w[1] * Iw[2] - w[2] * Iw[1], w[2] * Iw[0] - w[0] * Iw[2], w[0] * Iw[1] - w[1] * Iw[0]};
    double wdot[3] = {(tau[0] - gyro[0]) / ixx, (tau[1] - gyro[1]) / iyy, (tau[2] - gyro[2]) / izz};

    /* S6: semi-implicit Euler: velocities first, then positions with the new
     * velocities; dR/dt = R [w]x with body-frame w; polar re-orthonormalisation. */
    double vold[2] = {v[0], v[1]};
    const double x0[3] = {x[0], x[1], x[2]}; /* substep start (event-time contacts) */
    for (int k = 0; k < 3; ++k) v[k] += acc[k] * dt;
    if (on_floor && moving) {
        /* friction never reverses the sliding direction within one substep */
        double dot = v[0] * vold[0] + v[1] * vold[1];
        note_cmp(h, d, vold[0] * vold[0] + vold[1] * vold[1], vold[0] * vold[0] + vold[1] * vold[1] - dot);
        if (dot < 0.0) { v[0] = 0.0; v[1] = 0.0; }
    }
    for (int k = 0; k < 3; ++k) x[k] += v[k] * dt;
    /* body rates are bounded by |w_k| <= omega_max (the paper is silent; the
     * Crazyflie 2.x gyroscope saturates near 2000 deg/s); without a bound the
     * explicit gyroscopic term diverges under random per-rotor commands */
    for (int k = 0; k < 3; ++k) {
        w[k] += wdot[k] * dt;
        if (w[k] > c->omega_max) w[k] = c->omega_max;
        if (w[k] < -c->omega_max) w[k] = -c->omega_max;
    }
    double M[9];
    for (int i = 0; i < 3; ++i) {
        /* row_i(R [w]x) = row_i(R) x w */
        double r0 = R[3 * i + 0], r1 = R[3 * i + 1], r2 = R[3 * i + 2];
        M[3 * i + 0] = r0 + dt * (r1 * w[2] - r2 * w[1]);
        M[3 * i + 1] = r1 + dt * (r2 * w[0] - r0 * w[2]);
        M[3 * i + 2] = r2 + dt * (r0 * w[1] - r1 * w[0]);
    }
    or_polar(M, R);

    if (smooth) {
        if (x[2] < 0.0) h->ev[d] |= OR_EV_HIT_FLOOR;
        if (x[2] > c->room_h) h->ev[d] |= OR_EV_HIT_CEIL;
        if (fabs(x[0]) > c->room_hx || fabs(x[1]) > c->room_hy) h->ev[d] |= OR_EV_HIT_WALL;
        return;
    }

    /* S7: ground hit: velocities and momenta to zero, body z-axis set upright
     * keeping the heading (yaw) of the first body axis. */
    if (c->flags & OR_F_FLOOR) {
        note_cmp(h, d, x[2] - v[2] * dt, -v[2] * dt);          /* z+ = z + v dt vs 0 */
        if (x[2] <= 0.0) note_cmp(h, d, v[2] - acc[2] * dt, -acc[2] * dt); /* v+ = v + a dt vs 0 */
        if (x[2] <= 0.0 && v[2] < 0.0) {
            h->ev[d] |= OR_EV_HIT_FLOOR;
            if (c->flags & OR_F_EVENT_TIME) {
                /* the floor was crossed at time tau = -z0 / v_z of the substep's
                 * straight path x0 + v s; the drone is at rest from then on, so
                 * it travels horizontally only for tau */
                double tau = -x0[2] / v[2];
                tau = tau < 0.0 ? 0.0 : (tau > dt ? dt : tau);
                x[0] = x0[0] + v[0] * tau;
                x[1] = x0[1] + v[1] * tau;
            }
            x[2] = 0.0;
            for (int k = 0; k < 3; ++k) { v[k] = 0.0; w[k] = 0.0; }
            double cs, sn, hyp = sqrt(R[0] * R[0] + R[3] * R[3]);
            /* the heading is read off the horizontal part of the body x-axis, of
             * length hyp: an error e in R becomes about e / hyp in the heading */
            if (hyp < h->cond[d]) h->cond[d] = hyp;
            if (hyp >= 1e-6) { cs = R[0] / hyp; sn = R[3] / hyp; }
            else { double h2 = sqrt(R[1] * R[1] + R[4] * R[4]); cs = R[4] / h2; sn = -R[1] / h2; }
            double Rz[9] = {cs, -sn, 0.0, sn, cs, 0.0, 0.0, 0.0, 1.0};
            memcpy(R, Rz, sizeof Rz);
        }
    }

    /* S8: walls x = +-hx, y = +-hy and ceiling z = H. A drone past a boundary
     * is put back onto it. If it was moving outward, the quad-quad rule with a
     * static partner applies: the normal velocity component is removed (not
     * reflected), then v <- alpha_c (v + eps_v), w <- w + eps_w. (A drone whose
     * velocity the floor rule just zeroed is clamped without a response.) */
    if (c->flags & OR_F_WALLS) {
        int hit_wall = 0, hit_ceil = 0, clamped[3] = {0, 0, 0};
        double tau = dt;                                     /* earliest crossing (event-time contacts) */
        const double v1[3] = {v[0], v[1], v[2]};
        const double lim[2] = {c->room_hx, c->room_hy};
        for (int k = 0; k < 2; ++k) {
            note_cmp(h, d, x[k], lim[k]);
            note_cmp(h, d, x[k], -lim[k]);
            if (x[k] > lim[k]) {
                if (v[k] > 0.0) { v[k] = 0.0; hit_wall = 1; tau = fmin(tau, (lim[k] - x0[k]) / v1[k]); }
                x[k] = lim[k];
                clamped[k] = 1;
            } else if (x[k] < -lim[k]) {
                if (v[k] < 0.0) { v[k] = 0.0; hit_wall = 1; tau = fmin(tau, (-lim[k] - x0[k]) / v1[k]); }
                x[k] = -lim[k];
                clamped[k] = 1;
            }
        }
        note_cmp(h, d, x[2], c->room_h);
        if (x[2] > c->room_h) {
            if (v[2] > 0.0) { v[2] = 0.0; hit_ceil = 1; tau = fmin(tau, (c->room_h - x0[2]) / v1[2]); }
            x[2] = c->room_h;
            clamped[2] = 1;
        }
        if (hit_wall || hit_ceil) {
            double n[6];
            draw_six_normals(h, h->tick[e], (uint32_t)d, OR_TAG_WALL, (uint32_t)sub, n);
            for (int k = 0; k < 3; ++k) {
                v[k] = c->alpha_c * (v[k] + c->coll_sigma_v * n[k]);
                w[k] = w[k] + c->coll_sigma_w * n[3 + k];
            }
            if (c->flags & OR_F_EVENT_TIME) {
                /* the first boundary was crossed at tau on the straight path
                 * x0 + v1 s; the coordinates the boundaries do not hold move with
                 * the pre-contact velocity until tau and the post-contact one
                 * for the rest of the substep */
                tau = tau < 0.0 ? 0.0 : tau;
                for (int k = 0; k < 3; ++k)
                    if (!clamped[k]) x[k] = x0[k] + v1[k] * tau + v[k] * (dt - tau);
            }
            if (hit_wall) h->ev[d] |= OR_EV_HIT_WALL;
            if (hit_ceil) h->ev[d] |= OR_EV_HIT_CEIL;
        }
    }
}

/* Smooth-contact pair acceleration on drone i: sum over j != i of
 * k_c/m * softplus_beta(2l - d_ij) * n_ij, n_ij = (x_i - x_j)/d_ij. */
static void smooth_pair_acc(const or_env* h, int e, int i, double out[3]) {
    const or_config* c = &h->cfg;
    const double* p = h->prm + (size_t)e * OR_NPRM;
    const double* xi = h->st + (size_t)i * OR_NST + OR_S_X;
    double kc = c->smooth_kc * c->gravity;
    out[0] = out[1] = out[2] = 0.0;
    for (int j = h->env_off[e]; j < h->env_off[e + 1]; ++j) {
        if (j == i) continue;
        const double* xj = h->st + (size_t)j * OR_NST + OR_S_X;
        double dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
        double dist = sqrt(dx * dx + dy * dy + dz * dz);
        if (dist == 0.0) continue; /* direction undefined: no push */
        double mag = kc * softplus_b(2.0 * p[OR_P_ARM] - dist, c->smooth_beta);
        out[0] += mag * dx / dist; out[1] += mag * dy / dist; out[2] += mag * dz / dist;
    }
}

/* ------------------------------------------------------------------------- */
/* One control step of one environment (S1 .. S13).                           */
/* ------------------------------------------------------------------------- */
typedef struct { uint32_t key; int32_t j; } knn_item;

static int knn_cmp(const void* a, const void* b) {
    const knn_item* x = (const knn_item*)a; const knn_item* y = (const knn_item*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->j < y->j ? -1 : (x->j > y->j ? 1 : 0);
}

static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* S11: for each drone i of the env (local index), the keff nearest by
 * (binary32 key, local index) ascending over j != i; records near-ties. */
static void knn_env(or_env* h, int d0, int N, int keff, const float* xf, int32_t* nbr) {
    if (keff <= 0) return;
    knn_item* items = (knn_item*)malloc(sizeof(knn_item) * (size_t)N);
    for (int i = 0; i < N; ++i) {
        int m = 0;
        for (int j = 0; j < N; ++j)
            if (j != i) { items[m].key = f32_bits(or_pair_key(xf + 3 * i, xf + 3 * j)); items[m].j = j; ++m; }
        qsort(items, (size_t)m, sizeof(knn_item), knn_cmp);
        for (int k = 0; k < keff; ++k) nbr[i * keff + k] = items[k].j;
        /* near-ties at the ranks that matter (including the K-th vs the next);
         * they change only the observation, so they have their own margin */
        h->margin_knn[d0 + i] = INFINITY;
        for (int k = 0; k < keff && k + 1 < m; ++k) {
            float ka, kb; uint32_t ua = items[k].key, ub = items[k + 1].key;
            memcpy(&ka, &ua, 4); memcpy(&kb, &ub, 4);
            double den = fmax((double)ka, (double)kb);
            double mk = den > 0.0 ? ((double)kb - (double)ka) / den : 0.0;
            if (mk < h->margin_knn[d0 + i]) h->margin_knn[d0 + i] = mk;
        }
    }
    free(items);
}

/* S12: observation row of local drone i of env e: [x - g, v, R, w, then per
 * neighbour x_j - x_i, v_j - v_i; zeros past keff]. Sensor noise (Sec. III-C)
 * read as U(-s, s) on x and v and N(0, s^2) on w, from the OBS stream with
 * substream `sub` (0: control step, 1: observation of a freshly reset env). */
static void obs_row(or_env* h, int e, int i, const int32_t* nbr, int keff, uint32_t sub, const double goal[3],
                    double* o) {
    const or_config* c = &h->cfg;
    const int d0 = h->env_off[e], d = d0 + i, K = c->k_neighbors;
    const double* s = h->st + (size_t)d * OR_NST;
    const double *x = s + OR_S_X, *v = s + OR_S_V, *R = s + OR_S_R, *w = s + OR_S_W;
    double ex[3] = {0, 0, 0}, evv[3] = {0, 0, 0}, ew[3] = {0, 0, 0};
    if (c->flags & OR_F_OBS_NOISE) {
        double u0[4], u1[4], u2[4], n0, n1, n2, n3;
        draw_block(h, h->tick[e], (uint32_t)d, OR_TAG_OBS, sub, 0, u0);
        draw_block(h, h->tick[e], (uint32_t)d, OR_TAG_OBS, sub, 1, u1);
        draw_block(h, h->tick[e], (uint32_t)d, OR_TAG_OBS, sub, 2, u2);
        ex[0] = (2.0 * u0[0] - 1.0) * c->obs_sigma_x;
        ex[1] = (2.0 * u0[1] - 1.0) * c->obs_sigma_x;
        ex[2] = (2.0 * u0[2] - 1.0) * c->obs_sigma_x;
        evv[0] = (2.0 * u0[3] - 1.0) * c->obs_sigma_v;
        evv[1] = (2.0 * u1[0] - 1.0) * c->obs_sigma_v;
        evv[2] = (2.0 * u1[1] - 1.0) * c->obs_sigma_v;
        box_muller(u1[2], u1[3], &n0, &n1);
        box_muller(u2[0], u2[1], &n2, &n3);
        ew[0] = n0 * c->obs_sigma_w; ew[1] = n1 * c->obs_sigma_w; ew[2] = n2 * c->obs_sigma_w;
    }
    for (int k = 0; k < 3; ++k) {
        o[k] = x[k] - goal[k] + ex[k];
        o[3 + k] = v[k] + evv[k];
        o[15 + k] = w[k] + ew[k];
    }
    for (int k = 0; k < 9; ++k) o[6 + k] = R[k];
    for (int k = 0; k < K; ++k) {
        double* on = o + 18 + 6 * k;
        if (k < keff) {
            const double* sj = h->st + (size_t)(d0 + nbr[i * keff + k]) * OR_NST;
            for (int q = 0; q < 3; ++q) { on[q] = sj[OR_S_X + q] - x[q]; on[3 + q] = sj[OR_S_V + q] - v[q]; }
        } else {
            for (int q = 0; q < 6; ++q) on[q] = 0.0;
        }
    }
}

/* Conditioning instrument: one drone's state rounded to binary32 (see
 * OR_F_ROUND32), to nearest or stochastically. The stochastic choice hashes
 * (seed, salt, drone, tick, substep, component) with SplitMix64's finaliser. */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void round_state_f32(const or_env* h, double* s, int d, uint32_t tick, int sub) {
    const int sr = (h->cfg.flags & OR_F_ROUND32_SR) != 0;
    for (int k = 0; k < OR_NST; ++k) {
        float f = (float)s[k];
        if (sr && (double)f != s[k]) {
            float lo = (double)f < s[k] ? f : nextafterf(f, -INFINITY);
            float hi = (double)f < s[k] ? nextafterf(f, INFINITY) : f;
            double p = (s[k] - (double)lo) / ((double)hi - (double)lo);
            uint64_t z = mix64(h->cfg.seed ^ mix64(h->cfg.round_salt) ^
                               mix64(((uint64_t)(uint32_t)d << 32) ^ ((uint64_t)tick << 12) ^
                                     ((uint64_t)sub << 6) ^ (uint64_t)k));
            double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
            f = u < p ? hi : lo;
        }
        s[k] = (double)f;
    }
}

static void step_env(or_env* h, int e, const double* actions, double* obs, double* rew, uint8_t* done,
                     double* loss) {
    const or_config* c = &h->cfg;
    const int d0 = h->env_off[e], d1 = h->env_off[e + 1], N = d1 - d0;
    const int K = c->k_neighbors;
    const int keff = K < N - 1 ? K : N - 1;
    const int od = 18 + 6 * K;
    const double* p = h->prm + (size_t)e * OR_NPRM;
    const int smooth = (c->flags & OR_F_SMOOTH) != 0;

    double* fhat = (double*)malloc(sizeof(double) * 4 * (size_t)N);
    double* pacc = smooth ? (double*)malloc(sizeof(double) * 3 * (size_t)N) : NULL;
    for (int d = d0; d < d1; ++d) h->ev[d] = 0;

    /* substeps S1 .. S8 (drones of one env are coupled only through the smooth pair force) */
    for (int sub = 0; sub < c->substeps; ++sub) {
        if (smooth) for (int d = d0; d < d1; ++d) smooth_pair_acc(h, e, d, pacc + 3 * (d - d0));
        for (int d = d0; d < d1; ++d) {
            substep_drone(h, e, d, sub, actions + 4 * (size_t)d, smooth ? pacc + 3 * (d - d0) : NULL,
                          fhat + 4 * (d - d0));
            if (c->flags & OR_F_ROUND32) round_state_f32(h, h->st + (size_t)d * OR_NST, d, h->tick[e], sub);
        }
    }

    /* binary32 positions and arm length for the canonical keys */
    float* xf = (float*)malloc(sizeof(float) * 3 * (size_t)N);
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < 3; ++k) xf[3 * i + k] = (float)h->st[(size_t)(d0 + i) * OR_NST + OR_S_X + k];
    float lf = (float)p[OR_P_ARM];
    float thr = pair_threshold(lf, lf);

    /* S9: collision set: pair (i, j) collides iff key_ij < fl32((l_i + l_j)^2) */
    uint8_t* coll = (uint8_t*)calloc((size_t)N * N, 1);
    if ((c->flags & OR_F_COLLISIONS) && N >= 2) {
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) {
                float k = or_pair_key(xf + 3 * i, xf + 3 * j);
                note_margin(h, d0 + i, ((double)k - (double)thr) / (double)thr);
                note_margin(h, d0 + j, ((double)k - (double)thr) / (double)thr);
                if (k < thr) {
                    coll[i * N + j] = coll[j * N + i] = 1;
                    h->ev[d0 + i] |= OR_EV_HIT_QUAD; h->ev[d0 + j] |= OR_EV_HIT_QUAD;
                }
            }
    }
    /* S10: Jacobi response from pre-collision velocities: for every colliding and
     * approaching pair, v_i gets ((v_j - v_i).n) n with n = (x_i - x_j)/|x_i - x_j|;
     * then once per responding drone v <- alpha_c (v + sum + eps_v), w <- w + eps_w. */
    if (!smooth && (c->flags & OR_F_COLLISIONS) && N >= 2) {
        double* dv = (double*)calloc((size_t)3 * N, sizeof(double));
        double* dx_et = (double*)calloc((size_t)3 * N, sizeof(double)); /* sum_j v~_ij sigma_ij */
        double* smax = (double*)calloc((size_t)N, sizeof(double));      /* earliest contact of i */
        uint8_t* resp = (uint8_t*)calloc((size_t)N, 1);
        const int et = (c->flags & OR_F_EVENT_TIME) != 0;
        const double Tc = c->substeps * c->dt;
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                if (i == j || !coll[i * N + j]) continue;
                const double* xi = h->st + (size_t)(d0 + i) * OR_NST + OR_S_X;
                const double* xj = h->st + (size_t)(d0 + j) * OR_NST + OR_S_X;
                const double* vi = h->st + (size_t)(d0 + i) * OR_NST + OR_S_V;
                const double* vj = h->st + (size_t)(d0 + j) * OR_NST + OR_S_V;
                double dx[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
                double dvv[3] = {vi[0] - vj[0], vi[1] - vj[1], vi[2] - vj[2]};
                double app = dvv[0] * dx[0] + dvv[1] * dx[1] + dvv[2] * dx[2];
                double scl = sqrt((dvv[0] * dvv[0] + dvv[1] * dvv[1] + dvv[2] * dvv[2]) *
                                  (dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]));
                if (scl > 0.0) note_margin(h, d0 + i, app / scl);
                if (!(app < 0.0)) continue;
                double dist = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
                double n[3] = {0.0, 0.0, 1.0};
                if (dist > 0.0) { n[0] = dx[0] / dist; n[1] = dx[1] / dist; n[2] = dx[2] / dist; }
                double vn = (vj[0] - vi[0]) * n[0] + (vj[1] - vi[1]) * n[1] + (vj[2] - vi[2]) * n[2];
                for (int k = 0; k < 3; ++k) dv[3 * i + k] += vn * n[k];
                resp[i] = 1;
                if (et) {
                    /* contact time: run the pair's relative motion back from the
                     * end of the control step, r(s) = dx - dvv s; the separation
                     * reached the contact distance rho = l_i + l_j at
                     * sigma = -c0 / (sqrt(b^2 - a c0) - b), a = |dvv|^2,
                     * b = dx . dvv (< 0: approaching), c0 = |dx|^2 - rho^2 (< 0:
                     * overlapping); at most the control step's duration */
                    double rho = 2.0 * p[OR_P_ARM];
                    double a = dvv[0] * dvv[0] + dvv[1] * dvv[1] + dvv[2] * dvv[2];
                    double b = app;
                    double c0 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2] - rho * rho;
                    double sig = -c0 / (sqrt(b * b - a * c0) - b);
                    if (sig > Tc) sig = Tc;
                    if (sig < 0.0) sig = 0.0;
                    for (int k = 0; k < 3; ++k) dx_et[3 * i + k] += vn * n[k] * sig;
                    if (sig > smax[i]) smax[i] = sig;  /* ties keep the lower partner index */
                }
            }
        for (int i = 0; i < N; ++i) {
            if (!resp[i]) continue;
            double nn[6];
            draw_six_normals(h, h->tick[e], (uint32_t)(d0 + i), OR_TAG_COLL, 0, nn);
            double* vi = h->st + (size_t)(d0 + i) * OR_NST + OR_S_V;
            double* wi = h->st + (size_t)(d0 + i) * OR_NST + OR_S_W;
            double* xi = h->st + (size_t)(d0 + i) * OR_NST + OR_S_X;
            for (int k = 0; k < 3; ++k) {
                double vold_k = vi[k];
                vi[k] = c->alpha_c * (vi[k] + dv[3 * i + k] + c->coll_sigma_v * nn[k]);
                wi[k] = wi[k] + c->coll_sigma_w * nn[3 + k];
                if (et) {
                    /* each exchange acts from its own contact time, the decay and
                     * the perturbation from the drone's earliest contact */
                    double Dk = vi[k] - vold_k - c->alpha_c * dv[3 * i + k];
                    xi[k] += c->alpha_c * dx_et[3 * i + k] + Dk * smax[i];
                }
            }
        }
        free(dv); free(dx_et); free(smax); free(resp);
    }

    /* S10b: downwash (Sec. III-B "Downwash"). A drone j above drone i that
     * overlaps it in the xy plane (horizontal distance below l_i + l_j) within
     * dw_height vertically pushes i down with acceleration k1 (k2 dz + b1),
     * dz = z_j - z_i; several such drones add up. An affected drone also gets
     * acceleration noise N(0, s_a^2 I) and angular-acceleration noise
     * N(0, s_w^2 I). The test uses the post-substep positions, like the
     * collision set, and the effect acts over the control step (duration
     * substeps * dt) on the velocity and body rates. */
    if ((c->flags & OR_F_DOWNWASH) && N >= 2) {
        const double Tc = c->substeps * c->dt;
        const double r = 2.0 * p[OR_P_ARM];
        double* az = (double*)calloc((size_t)N, sizeof(double));
        uint8_t* hit = (uint8_t*)calloc((size_t)N, 1);
        for (int i = 0; i < N; ++i) {
            const double* xi = h->st + (size_t)(d0 + i) * OR_NST + OR_S_X;
            for (int j = 0; j < N; ++j) {
                if (j == i) continue;
                const double* xj = h->st + (size_t)(d0 + j) * OR_NST + OR_S_X;
                double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
                double rxy2 = dx * dx + dy * dy;
                note_cmp(h, d0 + i, rxy2, r * r);
                if (rxy2 < r * r) {
                    note_cmp(h, d0 + i, xj[2], xi[2]);
                    note_cmp(h, d0 + i, dz, c->dw_height);
                }
                if (rxy2 < r * r && dz > 0.0 && dz < c->dw_height) {
                    az[i] -= c->dw_k1 * (c->dw_k2 * dz + c->dw_b1);
                    hit[i] = 1;
                }
            }
        }
        for (int i = 0; i < N; ++i) {
            if (!hit[i]) continue;
            double nn[6];
            draw_six_normals(h, h->tick[e], (uint32_t)(d0 + i), OR_TAG_DOWNWASH, 0, nn);
            double* vi = h->st + (size_t)(d0 + i) * OR_NST + OR_S_V;
            double* wi = h->st + (size_t)(d0 + i) * OR_NST + OR_S_W;
            for (int k = 0; k < 3; ++k) {
                vi[k] += Tc * ((k == 2 ? az[i] : 0.0) + c->dw_sigma_a * nn[k]);
                wi[k] += Tc * c->dw_sigma_w * nn[3 + k];
            }
        }
        free(az); free(hit);
    }

    /* S11: K nearest by (key, local index) ascending over j != i. */
    int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(keff > 0 ? keff : 1) * N);
    knn_env(h, d0, N, keff, xf, nbr);
    if (c->flags & OR_F_RECORD_KNN) {
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < K; ++k) h->knn[(size_t)(d0 + i) * K + k] = k < keff ? nbr[i * keff + k] : -1;
    }

    /* S12 / S13: observation, reward */
    for (int i = 0; i < N; ++i) {
        int d = d0 + i;
        double* s = h->st + (size_t)d * OR_NST;
        const double *x = s + OR_S_X, *v = s + OR_S_V, *R = s + OR_S_R, *w = s + OR_S_W;
        double* fprev = s + OR_S_FPREV;
        const double* fh = fhat + 4 * i;
        /* the goal at the end of the step (Sec. III-D scenarios), tau = steps done */
        double goal[3];
        drone_goal(h, e, i, N, h->ep_t[e] + 1, goal);
        if (obs) obs_row(h, e, i, nbr, keff, 0, goal, obs + (size_t)d * od);
        if (rew) {
            const double* W = c->w;
            double dxg[3] = {x[0] - goal[0], x[1] - goal[1], x[2] - goal[2]};
            double dfa[4] = {fh[0] - fprev[0], fh[1] - fprev[1], fh[2] - fprev[2], fh[3] - fprev[3]};
            double r = 0.0;
            r += W[OR_W_POS] * sqrt(dxg[0] * dxg[0] + dxg[1] * dxg[1] + dxg[2] * dxg[2]);
            r += W[OR_W_VEL] * sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            r += W[OR_W_ORI] * R[8];
            r += W[OR_W_SPIN] * sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            r += W[OR_W_ACT] * sqrt(fh[0] * fh[0] + fh[1] * fh[1] + fh[2] * fh[2] + fh[3] * fh[3]);
            r += W[OR_W_DACT] * sqrt(dfa[0] * dfa[0] + dfa[1] * dfa[1] + dfa[2] * dfa[2] + dfa[3] * dfa[3]);
            r += W[OR_W_ROT] * (R[0] + R[4] + R[8] - 1.0) / 2.0;
            r += W[OR_W_YAW] * R[0];
            uint32_t ev = h->ev[d];
            r += W[OR_W_HIT_FLOOR] * ((ev & OR_EV_HIT_FLOOR) ? 1.0 : 0.0);
            r += W[OR_W_ON_FLOOR] * ((ev & OR_EV_ON_FLOOR) ? 1.0 : 0.0);
            r += W[OR_W_HIT_WALL] * ((ev & OR_EV_HIT_WALL) ? 1.0 : 0.0);
            r += W[OR_W_HIT_CEIL] * ((ev & OR_EV_HIT_CEIL) ? 1.0 : 0.0);
            r += W[OR_W_HIT_QUAD] * ((ev & OR_EV_HIT_QUAD) ? 1.0 : 0.0);
            double alpha_prox = c->prox_factor * p[OR_P_ARM];
            double near = 0.0;
            for (int k = 0; k < keff; ++k) {
                const double* xj = h->st + (size_t)(d0 + nbr[i * keff + k]) * OR_NST + OR_S_X;
                double dd = sqrt((xj[0] - x[0]) * (xj[0] - x[0]) + (xj[1] - x[1]) * (xj[1] - x[1]) +
                                 (xj[2] - x[2]) * (xj[2] - x[2]));
                near += fmax(1.0 - dd / alpha_prox, 0.0);
            }
            r += W[OR_W_NEAR] * near;
            rew[d] = r;
        }
        if (loss) {
            double l = 0.0;
            for (int k = 0; k < 3; ++k) l += (x[k] - goal[k]) * (x[k] - goal[k]);
            for (int r = 0; r < 4; ++r) l += 1e-3 * fh[r] * fh[r];
            loss[d] += l;
        }
        for (int r = 0; r < 4; ++r) fprev[r] = fh[r];
    }

    h->ep_t[e] += 1;
    int is_done = h->ep_t[e] >= c->episode_steps;
    if (done) done[e] = (uint8_t)is_done;
    if (is_done && (c->flags & OR_F_AUTO_RESET)) reset_env_all(h, h->key, h->tick[e], OR_TAG_AUTO_ENV, OR_TAG_AUTO_DRONE, e);
    h->tick[e] += 1;

    free(nbr); free(coll); free(xf); free(fhat); free(pacc);
}

typedef struct {
    or_env* h; int e0, e1; const double* actions; double* obs; double* rew; uint8_t* done; double* loss;
} step_job;

static void* step_worker(void* arg) {
    step_job* j = (step_job*)arg;
    for (int e = j->e0; e < j->e1; ++e) step_env(j->h, e, j->actions, j->obs, j->rew, j->done, j->loss);
    return NULL;
}

/* One control step of every environment. Environments are independent, so
 * they may be split over n_threads host threads by contiguous env ranges. */
void or_step(or_env* h, const double* actions, double* obs, double* rew, uint8_t* done, double* loss,
             int n_threads) {
    int E = h->cfg.n_envs;
    if (n_threads <= 1 || E < 2) {
        step_job j = {h, 0, E, actions, obs, rew, done, loss};
        step_worker(&j);
    } else {
        if (n_threads > E) n_threads = E;
        pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
        step_job* jobs = (step_job*)malloc(sizeof(step_job) * (size_t)n_threads);
        for (int t = 0; t < n_threads; ++t) {
            jobs[t].h = h; jobs[t].e0 = (int)((long)E * t / n_threads); jobs[t].e1 = (int)((long)E * (t + 1) / n_threads);
            jobs[t].actions = actions; jobs[t].obs = obs; jobs[t].rew = rew; jobs[t].done = done; jobs[t].loss = loss;
            pthread_create(&th[t], NULL, step_worker, &jobs[t]);
        }
        for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
        free(th); free(jobs);
    }
}


/* Observation of the current state of every env (S11 + S12, no dynamics),
 * with sensor noise from substream 1 of each env's current counter. */
void or_observe(or_env* h, double* obs) {
    const int K = h->cfg.k_neighbors, od = 18 + 6 * K;
    for (int e = 0; e < h->cfg.n_envs; ++e) {
        int d0 = h->env_off[e], N = h->env_off[e + 1] - d0;
        int keff = K < N - 1 ? K : N - 1;
        float* xf = (float*)malloc(sizeof(float) * 3 * (size_t)N);
        int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(keff > 0 ? keff : 1) * N);
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < 3; ++k) xf[3 * i + k] = (float)h->st[(size_t)(d0 + i) * OR_NST + OR_S_X + k];
        knn_env(h, d0, N, keff, xf, nbr);
        for (int i = 0; i < N; ++i) {
            double goal[3];
            drone_goal(h, e, i, N, h->ep_t[e], goal);
            obs_row(h, e, i, nbr, keff, 1, goal, obs + (size_t)(d0 + i) * od);
        }
        free(xf); free(nbr);
    }
}

/* ------------------------------------------------------------------------- */
/* State access (binary64 copies, caller-owned buffers; NULL skips a part).   */
/* ------------------------------------------------------------------------- */
void or_get_state(const or_env* h, double* st, double* prm, double* goal, int32_t* ep_t, uint32_t* tick) {
    if (tick) memcpy(tick, h->tick, sizeof(uint32_t) * (size_t)h->cfg.n_envs);
    if (st) memcpy(st, h->st, sizeof(double) * (size_t)h->n_drones * OR_NST);
    if (prm) memcpy(prm, h->prm, sizeof(double) * (size_t)h->cfg.n_envs * OR_NPRM);
    if (goal) memcpy(goal, h->goal, sizeof(double) * (size_t)h->cfg.n_envs * 3);
    if (ep_t) memcpy(ep_t, h->ep_t, sizeof(int32_t) * (size_t)h->cfg.n_envs);
}

void or_set_state(or_env* h, const double* st, const double* prm, const double* goal, const int32_t* ep_t,
                  const uint32_t* tick) {
    if (st) memcpy(h->st, st, sizeof(double) * (size_t)h->n_drones * OR_NST);
    if (prm) memcpy(h->prm, prm, sizeof(double) * (size_t)h->cfg.n_envs * OR_NPRM);
    if (goal) memcpy(h->goal, goal, sizeof(double) * (size_t)h->cfg.n_envs * 3);
    if (ep_t) memcpy(h->ep_t, ep_t, sizeof(int32_t) * (size_t)h->cfg.n_envs);
    if (tick) memcpy(h->tick, tick, sizeof(uint32_t) * (size_t)h->cfg.n_envs);
}

void or_get_scenario(const or_env* h, double* rec) {
    memcpy(rec, h->scn, sizeof(double) * (size_t)h->cfg.n_envs * OR_NSCN);
}

void or_set_scenario(or_env* h, const double* rec) {
    memcpy(h->scn, rec, sizeof(double) * (size_t)h->cfg.n_envs * OR_NSCN);
}

/* Goals [D][3] of every drone at its env's current control step. */
void or_goals(const or_env* h, double* goals) {
    for (int e = 0; e < h->cfg.n_envs; ++e) {
        const int d0 = h->env_off[e], N = h->env_off[e + 1] - d0;
        for (int i = 0; i < N; ++i) drone_goal(h, e, i, N, h->ep_t[e], goals + 3 * (size_t)(d0 + i));
    }
}

void or_get_events(const or_env* h, uint32_t* ev, int32_t* knn, double* margin, double* margin_knn, double* cond) {
    if (cond) memcpy(cond, h->cond, sizeof(double) * (size_t)h->n_drones);
    if (margin_knn) memcpy(margin_knn, h->margin_knn, sizeof(double) * (size_t)h->n_drones);
    if (ev) memcpy(ev, h->ev, sizeof(uint32_t) * (size_t)h->n_drones);
    if (knn && h->cfg.k_neighbors > 0)
        memcpy(knn, h->knn, sizeof(int32_t) * (size_t)h->n_drones * h->cfg.k_neighbors);
    if (margin) memcpy(margin, h->margin, sizeof(double) * (size_t)h->n_drones);
}

void or_clear_margin(or_env* h) {
    for (int d = 0; d < h->n_drones; ++d) h->margin[d] = h->cond[d] = INFINITY;
}

/* Standalone canonical KNN / collision set on given binary32 positions
 * (S9 + S11 only): used to check index decisions on inputs the dynamics
 * leave untouched. pos: [D][3]; arm: [E]; knn: [D][K] (-1 padded). */
void or_pairs_f32(const float* pos, const float* arm, const int32_t* env_off, int n_envs, int K,
                  int32_t* knn, uint8_t* hit) {
    for (int e = 0; e < n_envs; ++e) {
        int d0 = env_off[e], N = env_off[e + 1] - d0;
        int keff = K < N - 1 ? K : N - 1;
        float thr = pair_threshold(arm[e], arm[e]);
        knn_item* items = (knn_item*)malloc(sizeof(knn_item) * (size_t)(N > 0 ? N : 1));
        for (int i = 0; i < N; ++i) {
            int m = 0; hit[d0 + i] = 0;
            for (int j = 0; j < N; ++j) {
                if (j == i) continue;
                float k = or_pair_key(pos + 3 * (d0 + i), pos + 3 * (d0 + j));
                if (k < thr) hit[d0 + i] = 1;
                items[m].key = f32_bits(k); items[m].j = j; ++m;
            }
            qsort(items, (size_t)m, sizeof(knn_item), knn_cmp);
            for (int k = 0; k < K; ++k) knn[(size_t)(d0 + i) * K + k] = k < keff ? items[k].j : -1;
        }
        free(items);
    }
}
