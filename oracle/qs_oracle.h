/*
 * qs_oracle.h -- interface of the FP64 CPU oracle (test infrastructure only).
 * Used by qs_oracle.c and, through ctypes, by oracle/oracle.py. The CUDA
 * library neither includes nor links this file.
 */
#ifndef QS_ORACLE_H
#define QS_ORACLE_H
#include <stdint.h>

/* configuration flags */
#define OR_F_DR               (1u << 0)
#define OR_F_MOTOR_NOISE      (1u << 1)
#define OR_F_OBS_NOISE        (1u << 2)
#define OR_F_COLLISIONS       (1u << 3)
#define OR_F_FLOOR            (1u << 4)
#define OR_F_WALLS            (1u << 5)
#define OR_F_AUTO_RESET       (1u << 6)
#define OR_F_SMOOTH           (1u << 7)
#define OR_F_ACTION_SYMMETRIC (1u << 8)
#define OR_F_RECORD_KNN       (1u << 9)
#define OR_F_DOWNWASH         (1u << 10)
/* Conditioning instruments (off in every run of the model itself): after each
 * substep the drone state is rounded to binary32, to nearest (ROUND32) or
 * stochastically (ROUND32 | ROUND32_SR: up or down with probability given by
 * the distance to the two neighbours, from a hash of the seed, round_salt,
 * drone, tick, substep and component). Comparing such a run with a plain one
 * measures how much a trajectory amplifies perturbations of binary32 size. */
/* Event-time contacts (a variant of the model for gradients, beyond the
 * paper): a contact detected at the end of a substep (floor, walls,
 * ceiling) or control step (quad-quad) is resolved at its crossing time on
 * the straight path that led there, and the drone flies the rest of the
 * interval with its post-contact velocity. */
#define OR_F_EVENT_TIME       (1u << 13)
#define OR_F_ROUND32          (1u << 11)
#define OR_F_ROUND32_SR       (1u << 12)

/* per-drone event bits of the last control step */
#define OR_EV_HIT_FLOOR (1u << 0)
#define OR_EV_ON_FLOOR  (1u << 1)
#define OR_EV_HIT_WALL  (1u << 2)
#define OR_EV_HIT_CEIL  (1u << 3)
#define OR_EV_HIT_QUAD  (1u << 4)

/* Philox stream tags (third counter word = tag << 16 | substep << 8 | block) */
#define OR_TAG_RESET_ENV   1u
#define OR_TAG_RESET_DRONE 2u
#define OR_TAG_MOTOR       3u
#define OR_TAG_OBS         4u
#define OR_TAG_COLL        5u
#define OR_TAG_WALL        6u
#define OR_TAG_AUTO_ENV    7u
#define OR_TAG_AUTO_DRONE  8u
#define OR_TAG_DOWNWASH    9u
#define OR_TAG_SCN         10u /* scenario record of a reset */
#define OR_TAG_AUTO_SCN    11u /* scenario record of an auto-reset */
#define OR_TAG_WAYPOINT    12u /* evader waypoints (counter word 0 = the record's seed) */
#define OR_TAG_SWAP        13u /* goal-swap permutation keys (counter word 0 = the record's seed) */

/* training scenarios (Sec. III-D); or_config.scenarios is a mask of 1 << type */
enum {
    OR_SCN_SINGLE, OR_SCN_STATIC, OR_SCN_DYNAMIC, OR_SCN_SWAP, OR_SCN_SHRINK_EXPAND,
    OR_SCN_SWARM_VS_SWARM, OR_SCN_PURSUIT_LISSAJOUS, OR_SCN_PURSUIT_BEZIER, OR_NSCN_TYPES
};
/* goal formations */
enum { OR_FORM_CIRCLE, OR_FORM_GRID, OR_FORM_SPHERE, OR_FORM_CYLINDER, OR_FORM_CUBE, OR_NFORM };
/* per-env scenario record [OR_NSCN]: type, formation before / after the
 * switch, switch step, seed (low 16 bits), centre 0 (3), centre 1 or the
 * Lissajous amplitudes (3), Lissajous frequencies in Hz (3), Lissajous phases
 * in turns (3), seed (high 16 bits) */
#define OR_NSCN 18
#define OR_R_TYPE 0
#define OR_R_F0 1
#define OR_R_F1 2
#define OR_R_TSW 3
#define OR_R_SEED_LO 4
#define OR_R_C0 5
#define OR_R_C1 8
#define OR_R_FREQ 11
#define OR_R_PHASE 14
#define OR_R_SEED_HI 17

/* per-drone state row: x(3) v(3) R(9, row-major) w(3) uf(4) eps(4) fprev(4) */
#define OR_NST 30
#define OR_S_X 0
#define OR_S_V 3
#define OR_S_R 6
#define OR_S_W 15
#define OR_S_UF 18
#define OR_S_EPS 22
#define OR_S_FPREV 26

/* per-env randomised parameters: m, Ixx, Iyy, Izz, t2w, tau_m, arm */
#define OR_NPRM 7
#define OR_P_M 0
#define OR_P_IXX 1
#define OR_P_IYY 2
#define OR_P_IZZ 3
#define OR_P_T2W 4
#define OR_P_TAU 5
#define OR_P_ARM 6

/* reward weights */
enum {
    OR_W_POS, OR_W_VEL, OR_W_ORI, OR_W_SPIN, OR_W_ACT, OR_W_DACT, OR_W_ROT, OR_W_YAW,
    OR_W_HIT_FLOOR, OR_W_ON_FLOOR, OR_W_HIT_WALL, OR_W_HIT_CEIL, OR_W_HIT_QUAD, OR_W_NEAR,
    OR_NW
};

typedef struct {
    int32_t n_envs, k_neighbors, substeps, episode_steps;
    double dt;
    uint64_t seed;
    uint32_t flags, scenarios; /* scenarios: mask of 1 << OR_SCN_* drawn from at each reset */
    double mass, arm, ixx, iyy, izz, t2w, kappa, tau_m, gravity, mu;
    double alpha_nd, alpha_ns_frac, alpha_c, coll_sigma_v, coll_sigma_w;
    double obs_sigma_x, obs_sigma_v, obs_sigma_w;
    double room_hx, room_hy, room_h;
    double dr_lo, dr_hi;
    double smooth_beta, smooth_kc;
    double prox_factor;
    double omega_max;
    double dw_k1, dw_k2, dw_b1, dw_height, dw_sigma_a, dw_sigma_w; /* downwash */
    /* scenarios: goal spacing, radius cap of circles and cylinders, clearance of
     * centres from the room's faces, smallest scale of shrink & expand and its
     * period (control steps), base Lissajous frequency (Hz), control steps per
     * Bezier segment */
    double form_spacing, form_rmax, scn_margin, se_min, se_period, liss_f, bez_seg;
    double w[OR_NW];
    uint64_t round_salt; /* extra hash input of OR_F_ROUND32_SR */
} or_config;

typedef struct {
    or_config cfg;
    int32_t n_drones;
    int32_t* env_off;  /* [E+1] */
    double* prm;       /* [E][OR_NPRM] */
    double* goal;      /* [E][3] */
    double* scn;       /* [E][OR_NSCN] scenario records */
    double* st;        /* [D][OR_NST] */
    int32_t* ep_t;     /* [E] control steps since the env's episode began */
    uint32_t* ev;      /* [D] event bits of the last step */
    int32_t* knn;      /* [D][K] neighbour local indices of the last step (-1 padded) */
    double* margin;    /* [D] smallest normalised distance of a dynamics decision to its threshold */
    double* margin_knn; /* [D] smallest relative gap between ranked neighbour keys, last step */
    double* cond;      /* [D] smallest heading-extraction length of a floor reset (conditioning) */
    uint32_t* tick;    /* [E] control steps since the last full reset (Philox counter word 0) */
    uint32_t key[2];
} or_env;

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_philox4x32_10_n(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, size_t n);
double or_uniform(uint32_t r);
void or_polar(const double m[9], double r[9]);
float or_pair_key(const float xi[3], const float xj[3]);
void or_default_config(or_config* c);
or_env* or_create(const or_config* cfg, const int32_t* swarm_sizes);
void or_destroy(or_env* h);
int or_n_drones(const or_env* h);
void or_reset(or_env* h, uint64_t seed, const uint8_t* mask);
void or_step(or_env* h, const double* actions, double* obs, double* rew, uint8_t* done, double* loss,
             int n_threads);
void or_observe(or_env* h, double* obs);
void or_get_state(const or_env* h, double* st, double* prm, double* goal, int32_t* ep_t, uint32_t* tick);
void or_set_state(or_env* h, const double* st, const double* prm, const double* goal, const int32_t* ep_t,
                  const uint32_t* tick);
void or_get_scenario(const or_env* h, double* rec);
void or_set_scenario(or_env* h, const double* rec);
void or_goals(const or_env* h, double* goals);
void or_formation_offset(int form, int k, int n, double s, double rmax, double out[3]);
void or_get_events(const or_env* h, uint32_t* ev, int32_t* knn, double* margin, double* margin_knn, double* cond);
void or_clear_margin(or_env* h);
void or_pairs_f32(const float* pos, const float* arm, const int32_t* env_off, int n_envs, int K,
                  int32_t* knn, uint8_t* hit);

#endif
