/*
 * qs.h -- C ABI of libquadswarm_gpu.so, a GB300 (sm_103a) implementation of the
 * QuadSwarm forward-dynamics step (Huang et al., arXiv 2306.09537).
 *
 * The library simulates E independent environments ("envs"); env e holds N_e
 * quadrotors ("drones", 1 <= N_e <= 128), D = sum N_e drones in total. Drones
 * are numbered env by env: env e owns global drones [off_e, off_e + N_e).
 * One control step (100 Hz; two 200 Hz physics substeps by default, paper
 * Sec. IV) advances every drone by:
 *   motor lag and motor noise on the per-rotor command (Sec. III-A "Motor Lag",
 *   "Motor Noise"), thrust and torque from the rotor layout and rigid-body
 *   integration of position, velocity, rotation matrix and body rates
 *   (Sec. III-A dynamics block), floor, wall and ceiling contacts (Sec. III-B
 *   "Quadrotor to Ground", "Wall or Ceiling"), quadrotor-quadrotor collisions
 *   (Sec. III-B "Quadrotor to Quadrotor"), the K-nearest-neighbour observation
 *   with sensor noise (Sec. III-C) and the reward (Sec. III-E), under
 *   per-environment domain randomisation (Sec. I item (i)).
 *
 * Conventions shared by every entry point:
 *  - Pointers named *_dev are CUDA device pointers on the device that was
 *    current when the handle was created; *_host are host pointers. The
 *    caller owns every buffer it passes; the handle owns its internal state.
 *  - All work is enqueued on the handle's stream and the call returns without
 *    waiting, unless stated otherwise. Buffers passed to a call must stay
 *    valid until the stream reaches that work.
 *  - Argument errors (NULL handle or buffer, bad sizes, misaligned buffers)
 *    return QS_ERR_ARG at once and enqueue nothing. CUDA launch errors return
 *    QS_ERR_CUDA. Errors detected on the device (a non-finite state) set a
 *    status word that qs_sync() reports. qs_last_error() gives a message.
 *  - Floating point is binary32 throughout the device path.
 *  - A handle is used by one host thread at a time; distinct handles are
 *    independent (apart from qs_diff_grad_static's shared array).
 *  - Results do not depend on launch shapes (qs_set_block,
 *    qs_set_rollout_shape): the same state, parameters and commands give the
 *    same bits through qs_step, qs_step_host, qs_serve_step and qs_rollout.
 *
 * Layouts (row-major, contiguous):
 *  actions  [D][4]            per-rotor normalised commands (16-byte aligned)
 *  obs      [D][obs_dim]      obs_dim = 18 + 6 K  (8-byte aligned):
 *                             x - goal (3), v (3), R row-major (9), w (3),
 *                             then for k < K: x_j - x_i (3), v_j - v_i (3) of the
 *                             k-th nearest neighbour j, zeros past min(K, N_e - 1)
 *  reward   [D]
 *  done     [E]  uint8        1 when the env's episode reached episode_steps
 *  state    [D][30]           x(3) v(3) R(9) w(3) uf(4) eps(4) fprev(4)
 *  params   [E][7]            m, Ixx, Iyy, Izz, t2w, tau_m, arm
 *  goals    [E][3]            the single goal of each env (scenario "single")
 *  scenario [E][QS_NSCN]      scenario record of each env (see QS_SCN_*)
 *  drone goals [D][3]         each drone's goal at its env's current step
 */
#ifndef QS_H
#define QS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QS_ABI_VERSION 1
#define QS_MAX_SWARM 128    /* drones per env (the paper's largest team, Sec. V) */
#define QS_MAX_K 8          /* neighbours in the observation */
#define QS_STATE_DIM 30
#define QS_PARAM_DIM 7

typedef enum {
    QS_OK = 0,
    QS_ERR_ARG = 1,             /* invalid argument; nothing was enqueued */
    QS_ERR_CUDA = 2,            /* a CUDA call failed (message in qs_last_error) */
    QS_ERR_OOM = 3,             /* device allocation failed */
    QS_ERR_STATE_NONFINITE = 4, /* the device found a non-finite drone state */
    QS_ERR_TIMEOUT = 5,         /* reserved: a bounded device wait gave up */
    QS_ERR_UNSUPPORTED = 6,     /* e.g. a swarm larger than QS_MAX_SWARM */
    QS_ERR_INDEX = 7            /* debug build only: a device index check failed (qs_build_flags) */
} qs_status;

/* qs_config.flags */
#define QS_F_DR               (1u << 0) /* per-env randomisation of m, I, t2w, tau_m, arm */
#define QS_F_MOTOR_NOISE      (1u << 1) /* AR(1) motor noise (Sec. III-A) */
#define QS_F_OBS_NOISE        (1u << 2) /* sensor noise on the observation (Sec. III-C) */
#define QS_F_COLLISIONS       (1u << 3) /* quad-quad collisions (Sec. III-B) */
#define QS_F_FLOOR            (1u << 4) /* floor hit and friction (Sec. III-B) */
#define QS_F_WALLS            (1u << 5) /* walls and ceiling (Sec. III-B) */
#define QS_F_AUTO_RESET       (1u << 6) /* an env whose episode ends is redrawn in place */
#define QS_F_SMOOTH           (1u << 7) /* softplus penalty contacts (differentiable form) */
#define QS_F_ACTION_SYMMETRIC (1u << 8) /* f^ = (clip(a,-1,1)+1)/2 instead of clip(a,0,1) */
#define QS_F_RECORD_KNN       (1u << 9) /* keep neighbour indices for qs_get_events */
#define QS_F_DOWNWASH         (1u << 10) /* downwash from drones overlapping above (Sec. III-B) */
#define QS_F_EVENT_TIME       (1u << 11) /* differentiable rollout only: contacts at their crossing time */

/* Training scenarios (Sec. III-D). qs_config.scenarios is a mask of
 * (1u << QS_SCN_*); at every reset each env draws its scenario uniformly from
 * the enabled ones, together with a scenario record (below). The goal of each
 * drone is then a function of the record, the drone's index i in its swarm,
 * the swarm size N and the env's control step tau (the observation and reward
 * of a step use tau = the steps done at its end):
 *   SINGLE           the env's goal (goals [E][3]; the default, mask 0 or 1)
 *   STATIC           formation F0 around centre 0
 *   DYNAMIC          from the switch step on, formation F1 around centre 1
 *   SWAP             from the switch step on, the drones take the same goals
 *                    in a random order (drone i takes the rank of its Philox
 *                    key among the env's N keys)
 *   SHRINK_EXPAND    F0 scaled by 1 - (1 - se_min)(1 - cos(2 pi tau / se_period)) / 2
 *   SWARM_VS_SWARM   two groups (the first ceil(N/2) drones and the rest), each
 *                    a formation around its own centre; at the switch step the
 *                    formation becomes F1 and the groups swap centres
 *   PURSUIT_LISSAJOUS every drone chases c + A sin(2 pi (f tau T + phase)) per axis
 *                    (T = substeps dt)
 *   PURSUIT_BEZIER   every drone chases a point moving along cubic Bezier
 *                    segments (Catmull-Rom tangents) through random waypoints,
 *                    bez_seg control steps per segment
 * Formations (QS_FORM_*) of n goals, spacing form_spacing: a horizontal circle
 * (radius n s / 2 pi, at most form_rmax), a horizontal square grid, a
 * Fibonacci-lattice sphere (area s^2 per goal), stacked rings (cylinder), a
 * cubic grid. */
enum {
    QS_SCN_SINGLE, QS_SCN_STATIC, QS_SCN_DYNAMIC, QS_SCN_SWAP, QS_SCN_SHRINK_EXPAND, QS_SCN_SWARM_VS_SWARM,
    QS_SCN_PURSUIT_LISSAJOUS, QS_SCN_PURSUIT_BEZIER, QS_NSCN_TYPES
};
enum { QS_FORM_CIRCLE, QS_FORM_GRID, QS_FORM_SPHERE, QS_FORM_CYLINDER, QS_FORM_CUBE, QS_NFORM };
/* Scenario record (floats holding small integers where noted): type, formation
 * before and after the switch, switch step (uniform in [T/4, 3T/4] of the
 * episode), 32-bit seed as low / high 16 bits, centre 0 (3), centre 1 or the
 * Lissajous amplitudes (3), Lissajous frequencies in Hz (3) and phases in
 * turns (3). All zero under SINGLE. */
#define QS_NSCN 18
enum {
    QS_R_TYPE = 0, QS_R_F0 = 1, QS_R_F1 = 2, QS_R_TSW = 3, QS_R_SEED_LO = 4, QS_R_C0 = 5, QS_R_C1 = 8,
    QS_R_FREQ = 11, QS_R_PHASE = 14, QS_R_SEED_HI = 17
};

/* qs_get_events bits (per drone, last control step) */
#define QS_EV_HIT_FLOOR (1u << 0)
#define QS_EV_ON_FLOOR  (1u << 1)
#define QS_EV_HIT_WALL  (1u << 2)
#define QS_EV_HIT_CEIL  (1u << 3)
#define QS_EV_HIT_QUAD  (1u << 4)

/* reward weights, in qs_params.w (Sec. III-E; every weight carries its sign) */
enum {
    QS_W_POS, QS_W_VEL, QS_W_ORI, QS_W_SPIN, QS_W_ACT, QS_W_DACT, QS_W_ROT, QS_W_YAW,
    QS_W_HIT_FLOOR, QS_W_ON_FLOOR, QS_W_HIT_WALL, QS_W_HIT_CEIL, QS_W_HIT_QUAD, QS_W_NEAR,
    QS_NW
};

/* Physical and model constants. The paper states few of them; qs_config_default
 * fills the readings: Crazyflie 2.x mass 0.028 kg, arm 0.046 m, inertia
 * diag(1.657e-5, 1.666e-5, 2.926e-5) kg m^2, thrust-to-weight 2, yaw torque
 * coefficient 0.006 m, motor time constant 0.04 s, g 9.81, floor friction 0.3,
 * motor noise decay 0.9 and scale 2% of hover thrust per rotor, collision
 * decay 0.8 with perturbations N(0, 0.2^2) m/s and N(0, 0.5^2) rad/s, sensor
 * noise 5e-3 m, 1e-2 m/s, 1.75e-4 rad/s (Sec. III-C), room 10 x 10 x 10 m,
 * randomisation range [0.8, 1.2], softplus beta 200 1/m and stiffness 20 m g
 * per metre, proximity radius 4 arm lengths, body-rate bound 40 rad/s;
 * downwash (Sec. III-B, constants not given): a drone overlapping another from
 * above (horizontal distance < l_i + l_j, height difference dz in
 * (0, dw_height)) adds dw_k1 (dw_k2 dz + dw_b1) downward acceleration to it
 * for the control step, with k1 = 2.4525 m/s^2 (g/4), k2 = -2 1/m, b1 = 1,
 * dw_height 0.5 m, noise N(0, 0.1^2) m/s^2 on the acceleration and
 * N(0, 1^2) rad/s^2 on the angular acceleration; scenarios (Sec. III-D gives
 * no sizes or rates): goals 0.5 m apart, circle radius at most 4 m, centres
 * 1.5 m clear of the room's faces, shrink to half size and back every 400
 * steps, Lissajous base frequency 0.1 Hz, 300 steps per Bezier segment. */
typedef struct {
    float mass, arm, ixx, iyy, izz, t2w, kappa, tau_m, gravity, mu;
    float alpha_nd, alpha_ns_frac, alpha_c, coll_sigma_v, coll_sigma_w;
    float obs_sigma_x, obs_sigma_v, obs_sigma_w;
    float room_hx, room_hy, room_h;
    float dr_lo, dr_hi;
    float smooth_beta, smooth_kc, prox_factor, omega_max;
    float dw_k1, dw_k2, dw_b1, dw_height, dw_sigma_a, dw_sigma_w;
    float form_spacing, form_rmax, scn_margin, se_min, se_period, liss_f, bez_seg;
    float w[QS_NW];
} qs_params;

typedef struct {
    uint32_t size;              /* sizeof(qs_config); checked by qs_create */
    int32_t n_envs;             /* E >= 1 */
    const int32_t* swarm_sizes; /* host [E] drones per env, or NULL: n_per_env each */
    int32_t n_per_env;          /* used when swarm_sizes is NULL */
    int32_t k_neighbors;        /* K in [0, QS_MAX_K] */
    int32_t substeps;           /* physics substeps per control step (2) */
    float dt;                   /* physics substep (0.005 s) */
    int32_t episode_steps;      /* control steps per episode (1500 = 15 s) */
    uint64_t seed;              /* Philox key of the first reset */
    uint32_t flags;             /* QS_F_* */
    uint32_t scenarios;         /* mask of 1u << QS_SCN_* (0: single goal) */
    qs_params params;
} qs_config;

typedef struct qs_env qs_env;

/* Fills *cfg with the defaults above: 1 env x 1 drone, K = 6, 2 x 0.005 s
 * substeps, 1500-step episodes, seed 1, flags DR|MOTOR_NOISE|OBS_NOISE|
 * COLLISIONS|FLOOR|WALLS and the goal-reaching reward (pos -1, spin -0.1,
 * -1 per collision indicator). */
void qs_config_default(qs_config* cfg);

/* Environment definition of Sec. III (Gym-style multi-agent env, Table I).
 * Allocates the device state for cfg's envs on the current device and binds
 * the handle to cuda_stream (a cudaStream_t; NULL = the legacy default
 * stream). The state is drawn as by qs_reset(h, cfg->seed, NULL, NULL).
 * Errors: QS_ERR_ARG (bad config), QS_ERR_UNSUPPORTED (N_e > 128 or K > 8),
 * QS_ERR_OOM, QS_ERR_CUDA. On error *out is NULL. */
qs_status qs_create(const qs_config* cfg, void* cuda_stream, qs_env** out);

/* Frees the handle and its device memory after draining its stream. */
qs_status qs_destroy(qs_env* h);

/* D, E and obs_dim of the handle (any pointer may be NULL). Host-side only. */
qs_status qs_get_dims(const qs_env* h, int32_t* n_drones, int32_t* n_envs, int32_t* obs_dim);

/* Episode reset with domain randomisation (Sec. I (i), III-A). Draws per-env
 * parameters (each of m, Ixx, Iyy, Izz, t2w, tau_m, arm scaled by U(lo, hi)
 * when QS_F_DR), a goal uniform in the room, and per drone: position uniform
 * in the room, velocity and body rates uniform in [-1,1], a uniformly random
 * rotation, hovering motors. env_mask_dev == NULL: full reset, the Philox key
 * becomes `seed` and every env restarts at counter 0. Otherwise only envs with
 * env_mask_dev[e] != 0 are redrawn, from key `seed` at their current counter.
 * obs_dev (nullable) receives the observation of the new state. */
qs_status qs_reset(qs_env* h, uint64_t seed, const uint8_t* env_mask_dev, float* obs_dev);

/* One control step of every env (Sec. III-A .. III-E): actions_dev [D][4] in,
 * obs_dev [D][obs_dim], reward_dev [D], done_dev [E] out. obs_dev, reward_dev
 * and done_dev may be NULL (not written). A non-finite drone state found on
 * the device is reported by the next qs_sync() or qs_step_host(). One launch:
 * the per-call kernel of the handle's width class, or, when the swarm sizes
 * span several classes, one step of the rollout kernel (qs_rollout, T = 1). */
qs_status qs_step(qs_env* h, const float* actions_dev, float* obs_dev, float* reward_dev, uint8_t* done_dev);

/* qs_step for callers whose buffers live in host memory: actions_host [D][4]
 * in; obs/reward/done out (each nullable); waits for the stream and reports
 * like qs_sync. A page-locked buffer (cudaHostAlloc / cudaHostRegister, e.g.
 * torch pin_memory) that the device can address (actions 16-byte aligned, obs
 * 8-byte aligned) is read or written by the step kernel in place, over
 * NVLink-C2C on a Grace host; any other buffer goes through a device staging
 * buffer and one asynchronous copy. */
qs_status qs_step_host(qs_env* h, const float* actions_host, float* obs_host, float* reward_host,
                       uint8_t* done_host);

/* Resident stepping for synchronous host loops (the Gym wrapper of Sec. III:
 * post commands, wait, read the observations). qs_serve_begin starts one
 * cooperative launch that keeps every drone in registers and runs a control
 * step (the same computation and bits as qs_step) each time qs_serve_step is
 * called; the launch and completion round trip of a per-call step is replaced
 * by two words of page-locked host memory, one the host advances and one the
 * last CTA of a step advances.
 *
 *  actions_host [n_slots][D][4] in (n_slots >= 1 command slots; a step reads
 *  the slot qs_serve_step names, so commands can be written ahead), obs_host
 *  [D][obs_dim], reward_host [D], done_host [E] out (outputs nullable):
 *  page-locked host memory the device can map (cudaHostAlloc /
 *  cudaHostRegister, e.g. torch pin_memory; actions 16-byte, obs 8-byte
 *  aligned), owned by the caller, read and written in place by the server
 *  until qs_serve_end. Write a step's commands into a slot, call
 *  qs_serve_step(h, slot), read its outputs; a slot out of range returns
 *  QS_ERR_ARG.
 *  idle_ms: when no step is posted for about this long the server retires
 *  (the drones return to the handle's memory and the launch ends);
 *  qs_serve_step then starts it again, with no effect on the results. At
 *  most QS_SERVE_IDLE_MS_MAX (60 s): a resident launch holds every SM it
 *  occupies while it waits, so a longer wait on a shared GPU is refused
 *  (QS_ERR_ARG), as is idle_ms < 1.
 *
 * Requires every swarm to have at most 64 drones, a handle created on a
 * non-blocking stream (cudaStreamNonBlocking, as torch.cuda.Stream() makes;
 * the legacy default stream and streams that synchronise with it would wait
 * behind the resident launch), a device with native atomics on host memory
 * (a coherent host link such as NVLink-C2C) and room for all of the handle's
 * CTAs at once; QS_ERR_UNSUPPORTED otherwise. While serving, a device-wide
 * synchronisation (or a call that implies one, such as cudaFree) waits until
 * the server retires. Misaligned or unmapped buffers:
 * QS_ERR_ARG. While serving, every call that uses the handle's stream or
 * state returns QS_ERR_ARG; qs_serve_end (or qs_destroy) ends serving and
 * writes the drones back, after which they continue with qs_step or
 * qs_rollout exactly as if every step had been a qs_step. qs_serve_step
 * returns after the step's outputs are in host memory; a non-finite drone
 * state is reported as by qs_sync; a step that does not complete within 10 s
 * returns QS_ERR_TIMEOUT, after which qs_serve_step keeps waiting for that
 * same step and qs_serve_end stops the server once the step is done. */
#define QS_SERVE_IDLE_MS_MAX 60000
qs_status qs_serve_begin(qs_env* h, const float* actions_host, int32_t n_slots, float* obs_host, float* reward_host,
                         uint8_t* done_host, int32_t idle_ms);
qs_status qs_serve_step(qs_env* h, int32_t slot);
qs_status qs_serve_end(qs_env* h);

/* T control steps (T >= 1) of every env, batched: actions_dev [T][D][4],
 * obs_dev [T][D][obs_dim], reward_dev [T][D], done_dev [T][E] (outputs
 * nullable). Results equal T calls of qs_step. One persistent launch covers
 * envs of every swarm size: its CTAs take tiles of envs from a work counter
 * (largest swarms first) and keep each drone's state in registers across the
 * steps of a launch. The T steps run as ceil(T / fuse) launches (see
 * qs_set_rollout_shape). On a non-default stream the launches are captured
 * into a CUDA graph on the first call and replayed while T, the buffers and
 * the shape stay the same. Not callable during a caller's own stream capture
 * when a (re)capture is needed. */
qs_status qs_rollout(qs_env* h, int32_t T, const float* actions_dev, float* obs_dev, float* reward_dev,
                     uint8_t* done_dev);

/* Launch shape of qs_rollout: `block` threads per CTA of the persistent
 * kernel (32..256, a multiple of 32, at least the widest swarm class), or
 * QS_BLOCK_WARP_SPECIALISED (every class at most 64 wide; the default when
 * every class is at most 32 wide, all of the handle's such CTAs are
 * resident at once and neither scenarios nor downwash are on): per 32 drones
 * (64 when a class is wider than 32) one CTA whose dynamics warps integrate
 * while as many noise warps draw the noise and store the observation rows,
 * every step; `fuse` control steps per
 * launch (0 = all T steps in one launch), `use_graph` (0/1). Results do not
 * depend on the shape. Used by the autotuner. */
qs_status qs_set_rollout_shape(qs_env* h, int32_t block, int32_t fuse, int32_t use_graph);
qs_status qs_get_rollout_shape(const qs_env* h, int32_t* block, int32_t* fuse, int32_t* use_graph);

/* Differentiable rollout. From the initial drone states x0_dev [D][30] (state
 * layout above; the handle's parameters, goals and Philox counters; the
 * handle's own state is neither read nor changed) and commands actions_dev
 * [T][D][4], the forward pass writes the per-drone loss
 *     loss_dev[d] = sum_{t=1..T} |x_d(t) - goal|^2 + 1e-3 |f^_d(t)|^2
 * and stores a checkpoint every ckpt_every control steps in the caller's
 * workspace_dev (qs_diff_workspace_size bytes, 16-byte aligned). The backward
 * pass takes dloss_dev [D] (d objective / d loss_dev[d]) and the same T,
 * ckpt_every, actions and workspace, recomputes each checkpoint segment's
 * substeps into the workspace and runs the hand-written adjoint of the whole
 * step (dynamics, integrator with re-orthonormalisation, contacts), writing
 * grad_actions_dev [T][D][4] and grad_x0_dev [D][30] (zero for the
 * previous-command entries, which do not enter the loss). Motor noise is a
 * fixed additive draw. Two contact models:
 *  - QS_F_SMOOTH: the floor, walls, ceiling and quad-quad contacts of
 *    Sec. III-B become softplus penalty accelerations k_c sp_beta(pen)/m
 *    along the contact normal, so the step is smooth;
 *  - otherwise the contacts as the step runs them (floor friction and hit,
 *    walls and ceiling, collisions with their perturbations); the gradient is
 *    the derivative of the contact branch each decision took (the map is
 *    piecewise smooth; resets that set a state component to a constant pass
 *    no gradient through it);
 *  - with QS_F_EVENT_TIME (a variant of the model for gradients, beyond the
 *    paper's Sec. III-B), each contact detected at the end of a substep
 *    (floor, walls, ceiling) or control step (quad-quad) is resolved at its
 *    crossing time on the straight path that led there: a drone that hits the
 *    floor moves horizontally only until it crosses z = 0 (tau = -z0 / v_z),
 *    a wall or ceiling contact moves the coordinates the boundaries do not
 *    hold with the pre-contact velocity until the first crossing and with the
 *    post-contact velocity after it, and a colliding pair touched sigma =
 *    -c0 / (sqrt(b^2 - a c0) - b) before the end of the step (a = |v_i -
 *    v_j|^2, b = (v_i - v_j).(x_i - x_j), c0 = |x_i - x_j|^2 - (l_i + l_j)^2,
 *    at most the step's duration), each exchange acting on the position from
 *    its contact time and the decay and perturbation from the drone's
 *    earliest contact. The gradient then includes the terms through the
 *    crossing times (the saltation of the hybrid dynamics).
 * A handle created with QS_F_DOWNWASH or with scenarios other than the single
 * goal, or with QS_F_EVENT_TIME together with QS_F_SMOOTH, returns
 * QS_ERR_UNSUPPORTED. QS_F_EVENT_TIME changes only these entry points:
 * qs_step, qs_step_host, qs_rollout and qs_serve_begin return
 * QS_ERR_UNSUPPORTED for a handle created with it. */
qs_status qs_diff_workspace_size(const qs_env* h, int32_t T, int32_t ckpt_every, size_t* bytes);
qs_status qs_diff_forward(qs_env* h, int32_t T, int32_t ckpt_every, const float* x0_dev, const float* actions_dev,
                          float* loss_dev, void* workspace_dev);
qs_status qs_diff_backward(qs_env* h, int32_t T, int32_t ckpt_every, const float* actions_dev, const float* dloss_dev,
                           void* workspace_dev, float* grad_actions_dev, float* grad_x0_dev);

/* Allocation-free form of qs_diff_forward + qs_diff_backward. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory when they need a gradient, such as code running while a CUDA graph
 * is captured, real-time control loops that must not call cudaMalloc or
 * cudaFree (both can synchronise the device), or plugins whose host framework
 * owns the memory budget. It needs no workspace argument: the checkpoints and
 * recomputed substep states live in a fixed array of QS_DIFF_STATIC_BYTES
 * (64 MiB) inside the library's device image, held on every GPU that loads
 * the library until the process exits (a device reset or a released
 * primary context ends the array's life with the context; the next call made
 * outside a stream capture finds it again). The call allocates nothing; the
 * caller still passes every input and output: x0_dev [D][30], actions_dev
 * [T][D][4], dloss_dev [D] in; loss_dev [D], grad_actions_dev [T][D][4],
 * grad_x0_dev [D][30] out (same meaning as qs_diff_forward/_backward).
 * A rollout whose workspace (qs_diff_workspace_size) exceeds the array returns
 * QS_ERR_UNSUPPORTED and enqueues nothing. Each call made while the
 * handle's stream is not capturing looks the array's device address up
 * (cudaGetSymbolAddress); a call made during a capture reuses the address of
 * the last such call on that device, so make the first call on a device
 * before any stream capture (otherwise QS_ERR_UNSUPPORTED). All calls share the one array: calls whose work
 * overlaps on the GPU (other streams, other handles) race and must be
 * serialised by the caller. The array keeps the last call's contents; no call
 * depends on them. */
#define QS_DIFF_STATIC_BYTES (64u << 20)
qs_status qs_diff_grad_static(qs_env* h, int32_t T, int32_t ckpt_every, const float* x0_dev, const float* actions_dev,
                              const float* dloss_dev, float* loss_dev, float* grad_actions_dev, float* grad_x0_dev);

/* Copies the handle's state into caller buffers (each nullable): state_dev
 * [D][30], params_dev [E][7], goals_dev [E][3], ep_step_dev [E] control steps
 * into the episode, tick_dev [E] Philox step counter of each env. */
qs_status qs_get_state(qs_env* h, float* state_dev, float* params_dev, float* goals_dev, int32_t* ep_step_dev,
                       uint32_t* tick_dev);

/* Overwrites the handle's state from caller buffers (each nullable; layouts as
 * qs_get_state). Derived per-env constants are recomputed from params_dev. */
qs_status qs_set_state(qs_env* h, const float* state_dev, const float* params_dev, const float* goals_dev,
                       const int32_t* ep_step_dev, const uint32_t* tick_dev);

/* Scenario records [E][QS_NSCN] of every env (layout above): copied out to,
 * or overwritten from, a caller buffer. A record whose type is not enabled in
 * the handle's mask is still evaluated as written. */
qs_status qs_get_scenario(qs_env* h, float* records_dev);
qs_status qs_set_scenario(qs_env* h, const float* records_dev);

/* Goal of every drone at its env's current control step (Sec. III-D), into
 * goals_dev [D][3]: what the next observation after a reset, or the reward of
 * the step that ended at this control step, measured against. */
qs_status qs_get_goals(qs_env* h, float* goals_dev);

/* Event bits of the last step per drone (events_dev [D], QS_EV_*) and, when
 * the handle was created with QS_F_RECORD_KNN, the neighbour list knn_dev
 * [D][K] as local indices within the env, -1 past min(K, N_e - 1) (Sec.
 * III-C: ordered by distance, ties to the lower index). Either nullable. */
qs_status qs_get_events(qs_env* h, uint32_t* events_dev, int16_t* knn_dev);

/* Waits for the handle's stream and reports a device-detected error
 * (QS_ERR_STATE_NONFINITE stays reported until the next full qs_reset). */
qs_status qs_sync(qs_env* h);

/* The library's Philox4x32-10 counter-based generator (Salmon et al., SC'11),
 * which every random draw of the step, the resets and the scenarios uses,
 * exposed for checking it against other implementations:
 * out_dev[i][0..3] = Philox4x32-10(counter (ctr_dev[i][0], ctr_dev[i][1],
 * ctr_dev[i][2], 0), key (key0, key1)) for i < n, computed on the current
 * device and enqueued on cuda_stream (NULL: the legacy default stream).
 * ctr_dev [n][3] and out_dev [n][4] (16-byte aligned) are uint32 device
 * buffers owned by the caller. variant 0 uses the round keys precomputed on
 * the host (the form the step's draws use), 1 the inline key schedule (the
 * form of the reset draws). QS_ERR_ARG for NULL or misaligned buffers,
 * n < 0 or another variant. Needs no handle. */
qs_status qs_philox4x32_10(const uint32_t* ctr_dev, uint32_t key0, uint32_t key1, int32_t variant, uint32_t* out_dev,
                           int64_t n, void* cuda_stream);

/* Build of the loaded library. Bit QS_BUILD_DEBUG_CHECKS: the debug build
 * (libquadswarm_gpu_debug.so, compiled with -DQS_DEBUG_CHECKS; the paper has
 * no counterpart). In it the kernels check the indices they derive from
 * their launch geometry (each slot's env, first drone and size, the slot's
 * lanes within the CTA, a drone's env, a contiguous observation block) against
 * the buffers they address; a failed check sets a bit of the handle's status
 * word and the thread skips the work that would use the index (no access out
 * of range, no trap, no skipped barrier), and the next qs_sync returns
 * QS_ERR_INDEX. Results are otherwise those of the release build. */
#define QS_BUILD_DEBUG_CHECKS 1
int32_t qs_build_flags(void);

/* Debug build only: runs one check of the device index `index` against the
 * handle's drone count on its stream (a kernel that reads and rewrites the
 * event word of drone `index` when the check passes), so that a test can see
 * a failed check reported by qs_sync without any access out of range.
 * QS_ERR_UNSUPPORTED in the release build, which would not check. */
qs_status qs_debug_check_selftest(qs_env* h, int32_t index);

/* Launch shape of qs_step for one swarm-width class (the envs whose swarm size
 * rounds up to the power of two `width`, 1..128): `block` threads per CTA, a
 * multiple of 32 and of `width`, at most 256; or QS_BLOCK_WARP_SPECIALISED
 * (widths <= 32, the default there): CTAs of two warps per 32 drones, one
 * integrating the dynamics while the other draws the motor and sensor noise
 * and writes the observation rows. It shapes the steps of a handle whose envs
 * all fall in one class, and the reset observation; a handle with several
 * classes steps them all in one launch shaped by qs_set_rollout_shape. Used
 * by the autotuner; results do not depend on it. QS_ERR_ARG for an invalid
 * shape or a class the handle lacks. */
#define QS_BLOCK_WARP_SPECIALISED 1
qs_status qs_set_block(qs_env* h, int32_t width, int32_t block);

/* Reads back the launch shape of a class (block 0 when the handle has none). */
qs_status qs_get_block(const qs_env* h, int32_t width, int32_t* block);

/* Last error message of the handle (or of the last failed qs_create when h
 * is NULL). Never NULL; valid until the next call on the handle. */
const char* qs_last_error(const qs_env* h);

#ifdef __cplusplus
}
#endif
#endif /* QS_H */
