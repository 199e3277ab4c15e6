// qs_step.cu -- the fused control step (S1..S13) on sm_103a, in two forms:
//
//  k_step<W>   one control step per launch (qs_step): state read from and
//              written back to HBM.
//  k_rollout   T control steps per launch (qs_rollout): a persistent kernel
//              whose CTAs pull tiles of envs from a work counter (widest,
//              costliest classes first) and keep each drone's state in
//              registers across the T steps; one launch covers envs of every
//              swarm size.
//
// Layout: a CTA processes env "slots" of one width class W (a power of two >=
// the env's swarm size N); thread `lane` of a slot carries drone `lane` of the
// env. For W > 1 the slot exchanges positions and velocities through shared
// memory for the O(N^2) pair pass (collisions, Sec. III-B) and the K-nearest
// neighbour selection (Sec. II-B, III-C), which each thread keeps as a sorted
// register list of 64-bit keys (binary32 distance bits << 32 | index).
#include <cuda_runtime.h>
#include <stdint.h>

#include "qs_device.cuh"
#include "qs_internal.h"
#include "qs_scenario.cuh"

namespace qsk {

constexpr int MAX_BLOCK = 256;
// dynamic shared memory of the step and rollout kernels, per thread: staged
// position (3) and velocity (3) of the pair pass, swap key (1)
constexpr int SMEM_PLANES = 7;

// The step kernels come in two instances: EXT = true carries the training
// scenarios (per-drone goals), the downwash term and the smooth contacts,
// deciding each at run time; EXT = false is the common configuration (one
// goal, no downwash, the paper's discrete contacts) with these decided at
// compile time, so it keeps the smaller code and register budget, and the
// substep's contact branch is straight-line code (extended_instance()).
inline bool extended(const Consts& c) { return extended_instance(c); }

// Per-env values a thread keeps in registers.
struct EnvRegs {
    Prm p;
    float g0, g1, g2;
    int ep;
    uint32_t tick;
    int sel;       // active buffer of the env's scenario record
    bool redrawn;  // auto-reset drew new parameters / goal this launch
};

template <bool EXT>
__device__ __forceinline__ void load_env(EnvRegs& er, const Consts& c, const Dev& dv, int e) {
    er.p = load_prm(c, dv.prm, dv.E, e);
    er.g0 = dv.goal[e];
    er.g1 = dv.goal[dv.E + e];
    er.g2 = dv.goal[2 * dv.E + e];
    er.ep = dv.ep[e];
    er.tick = dv.tick[e];
    er.sel = (EXT && (c.scn_mask & ~1u)) ? dv.scn_sel[e] : 0;
    er.redrawn = false;
}

// Written by lane 0 of the slot at the end of a launch.
template <bool EXT>
__device__ __forceinline__ void store_env(const EnvRegs& er, const Dev& dv, int e) {
    dv.ep[e] = er.ep;
    dv.tick[e] = er.tick;
    if (er.redrawn) {
        const float v[NPRM_DEV] = {er.p.m, er.p.ixx, er.p.iyy, er.p.izz, er.p.t2w, er.p.tau, er.p.arm, er.p.fmax,
                                   er.p.alag, er.p.ans, er.p.inv_m, er.p.inv_ixx, er.p.inv_iyy, er.p.inv_izz,
                                   er.p.thr, er.p.prox};
        for (int k = 0; k < NPRM_DEV; ++k) dv.prm[(size_t)k * dv.E + e] = v[k];
        dv.goal[e] = er.g0;
        dv.goal[dv.E + e] = er.g1;
        dv.goal[2 * dv.E + e] = er.g2;
        if (EXT) dv.scn_sel[e] = (uint8_t)er.sel;
    }
}

// Goal slot of drone `lane` under an active swap: the rank of its key among
// the keys staged by its env's drones at skey[sbase .. sbase + N) (ties to
// the lower index).
__device__ __forceinline__ int swap_rank(const uint32_t* skey, int sbase, int N, int lane, uint32_t myk) {
    int slot = 0;
    for (int j = 0; j < N; ++j) {
        const uint32_t kj = skey[sbase + j];
        slot += (kj < myk || (kj == myk && j < lane)) ? 1 : 0;
    }
    return slot;
}

// Downwash over the control step (duration substeps * dt): v_z += T az plus
// acceleration noise, w += T * angular-acceleration noise.
__device__ __forceinline__ void apply_downwash(const Consts& c, Drone& s, uint32_t tick, int d, float az) {
    float n[6];
    six_normals(c, tick, (uint32_t)d, TAG_DOWNWASH, 0, n);
    const float Tc = c.dt * (float)c.substeps;
    s.v[0] = __fmaf_rn(Tc, __fmul_rn(c.dw_sa, n[0]), s.v[0]);
    s.v[1] = __fmaf_rn(Tc, __fmul_rn(c.dw_sa, n[1]), s.v[1]);
    s.v[2] = fmaf(Tc, fmaf(c.dw_sa, n[2], az), s.v[2]);
    const float tsw = __fmul_rn(Tc, c.dw_sw);
    comp_add_prod(s.w[0], s.wlo[0], tsw, n[3]);
    comp_add_prod(s.w[1], s.wlo[1], tsw, n[4]);
    comp_add_prod(s.w[2], s.wlo[2], tsw, n[5]);
}

// S13 reward of one drone (Sec. III-E): weighted state terms, event indicators
// and the proximity term over its neighbours (keys = squared distances).
__device__ __forceinline__ float compute_reward(const Consts& c, const Drone& s, float prox, const float g[3],
                                                const float fh[4], uint32_t ev, const uint64_t best[QS_MAX_K], int keff) {
    // explicit roundings: the same bits from every kernel that computes it
    const float dgx = __fsub_rn(s.x[0], g[0]), dgy = __fsub_rn(s.x[1], g[1]), dgz = __fsub_rn(s.x[2], g[2]);
    float r = __fmul_rn(c.w[QS_W_POS], sqrt_approx(dot3(dgx, dgy, dgz, dgx, dgy, dgz)));
    r = __fmaf_rn(c.w[QS_W_VEL], sqrt_approx(dot3(s.v[0], s.v[1], s.v[2], s.v[0], s.v[1], s.v[2])), r);
    r = __fmaf_rn(c.w[QS_W_ORI], s.R[8], r);
    r = __fmaf_rn(c.w[QS_W_SPIN], sqrt_approx(dot3(s.w[0], s.w[1], s.w[2], s.w[0], s.w[1], s.w[2])), r);
    const float na = __fmaf_rn(fh[3], fh[3], dot3(fh[0], fh[1], fh[2], fh[0], fh[1], fh[2]));
    r = __fmaf_rn(c.w[QS_W_ACT], sqrt_approx(na), r);
    const float q0 = __fsub_rn(fh[0], s.fp[0]), q1 = __fsub_rn(fh[1], s.fp[1]), q2 = __fsub_rn(fh[2], s.fp[2]),
                q3 = __fsub_rn(fh[3], s.fp[3]);
    r = __fmaf_rn(c.w[QS_W_DACT], sqrt_approx(__fmaf_rn(q3, q3, dot3(q0, q1, q2, q0, q1, q2))), r);
    const float tr = __fsub_rn(__fadd_rn(__fadd_rn(s.R[0], s.R[4]), s.R[8]), 1.0f);
    r = __fmaf_rn(__fmul_rn(c.w[QS_W_ROT], 0.5f), tr, r);
    r = __fmaf_rn(c.w[QS_W_YAW], s.R[0], r);
    r = __fadd_rn(r, (ev & EV_HIT_FLOOR) ? c.w[QS_W_HIT_FLOOR] : 0.0f);
    r = __fadd_rn(r, (ev & EV_ON_FLOOR) ? c.w[QS_W_ON_FLOOR] : 0.0f);
    r = __fadd_rn(r, (ev & EV_HIT_WALL) ? c.w[QS_W_HIT_WALL] : 0.0f);
    r = __fadd_rn(r, (ev & EV_HIT_CEIL) ? c.w[QS_W_HIT_CEIL] : 0.0f);
    r = __fadd_rn(r, (ev & EV_HIT_QUAD) ? c.w[QS_W_HIT_QUAD] : 0.0f);
    if (keff > 0 && c.w[QS_W_NEAR] != 0.0f) {
        float near = 0.0f;
        const float inv_prox = __frcp_rn(prox);
#pragma unroll
        for (int k = 0; k < QS_MAX_K; ++k) {
            if (k < keff) {
                const float key = __uint_as_float((uint32_t)(best[k] >> 32));
                near = __fadd_rn(near, fmaxf(__fmaf_rn(-sqrt_approx(key), inv_prox, 1.0f), 0.0f));
            }
        }
        r = __fmaf_rn(c.w[QS_W_NEAR], near, r);
    }
    return r;
}

// End of a control step: previous command, episode counter, done flag,
// Philox counter, in-place auto-reset, non-finite check.
template <bool EXT>
__device__ __forceinline__ void end_step(const Consts& c, const Dev& dv, Drone& s, EnvRegs& er, const float fh[4],
                                         int lane, int e, int d, uint8_t* __restrict__ done) {
    s.fp[0] = fh[0];
    s.fp[1] = fh[1];
    s.fp[2] = fh[2];
    s.fp[3] = fh[3];
    const uint32_t tick = er.tick;
    const int ep = er.ep + 1;
    const bool is_done = ep >= c.episode_steps;
    if (lane == 0 && done) done[e] = is_done ? 1 : 0;
    er.ep = (is_done && (c.flags & QS_F_AUTO_RESET)) ? 0 : ep;
    er.tick = tick + 1;
    if (is_done && (c.flags & QS_F_AUTO_RESET)) {
        // the env starts a new episode in place (new randomisation and goal);
        // every lane draws the env's values itself, so no exchange is needed
        float p7[QS_PARAM_DIM], goal[3], full[NPRM_DEV];
        draw_env(c, c.key0, c.key1, tick, TAG_AUTO_ENV, e, p7, goal);
        derive(c, p7, full);
        er.p = prm_from(full);
        er.g0 = goal[0];
        er.g1 = goal[1];
        er.g2 = goal[2];
        er.redrawn = true;
        draw_drone(c, c.key0, c.key1, tick, TAG_AUTO_DRONE, d, p7[P_T2W], s);
        if (EXT && (c.scn_mask & ~1u)) {
            // the next episode's record goes to the other buffer: lanes of
            // this env may still be reading the current one for this step
            er.sel ^= 1;
            if (lane == 0) {
                float rec[QS_NSCN];
                draw_scenario(c, c.key0, c.key1, tick, TAG_AUTO_SCN, e, rec);
                store_scenario(dv, er.sel, e, rec);
            }
        }
    }
    if (!finite_state(s)) atomicOr(dv.status, 1);
}

// One control step of the slot's drones. All threads of the CTA call it (the
// pair pass synchronises the CTA); `act` marks threads that carry a drone.
// Outputs for this step: obs/rew rows of drone d, done[e] (lane 0). W is
// uniform over the CTA; a compile-time W folds away after inlining.
template <bool EXT>
__device__ __forceinline__ void step_body(const int W, const Consts& c, const Dev& dv, Drone& s, EnvRegs& er, uint32_t& ev_out,
                                          float* sx, float* sv, const bool act, const int lane, const int N,
                                          const int sbase, const int e, const int d, const float4 a,
                                          float* __restrict__ obs, float* __restrict__ rew, uint8_t* __restrict__ done,
                                          const int observe_only, GoalCache& gc) {
    const int nt = blockDim.x;
    const int K = c.K;
    const int keff = min(K, N - 1);
    const uint32_t tick = er.tick;
    // the EXT = false instance carries neither scenario nor downwash code
    const bool scn = EXT && (c.scn_mask & ~1u) != 0;
    const bool dw = EXT && (c.flags & QS_F_DOWNWASH) != 0;
    const int tau = observe_only ? er.ep : er.ep + 1;  // the goal is the one at the step's end
    uint32_t* skey = reinterpret_cast<uint32_t*>(sv + 3 * nt);
    bool swp = false;
    uint32_t myk = 0;
    float fh[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t ev = 0;
    // smooth contacts of a swarm (general instance): the pair penalty from the
    // positions at each substep's start, staged like the pair pass (uniform
    // over the CTA: every thread meets the barriers)
    const bool spair = EXT && (c.flags & QS_F_SMOOTH) && W > 1 && !observe_only;
    if (spair) {
        if (act) {
            fh[0] = command(c, a.x);
            fh[1] = command(c, a.y);
            fh[2] = command(c, a.z);
            fh[3] = command(c, a.w);
        }
        const float u[4] = {sqrt_approx(fh[0]), sqrt_approx(fh[1]), sqrt_approx(fh[2]), sqrt_approx(fh[3])};
        for (int sub = 0; sub < c.substeps; ++sub) {
            float pacc[3] = {0.f, 0.f, 0.f};
            if (act) {
                sx[threadIdx.x] = s.x[0];
                sx[nt + threadIdx.x] = s.x[1];
                sx[2 * nt + threadIdx.x] = s.x[2];
            }
            __syncthreads();
            if (act && N > 1) pair_acc(c, s.x, sx, nt, sbase, lane, N, er.p.arm, pacc);
            __syncthreads();
            if (act) ev |= substep<false, EXT ? -1 : 0>(s, er.p, c, u, tick, d, sub, pacc);
        }
    } else if (act && !observe_only) {
        fh[0] = command(c, a.x);
        fh[1] = command(c, a.y);
        fh[2] = command(c, a.z);
        fh[3] = command(c, a.w);
        const float u[4] = {sqrt_approx(fh[0]), sqrt_approx(fh[1]), sqrt_approx(fh[2]), sqrt_approx(fh[3])};
        const float zero3[3] = {0.f, 0.f, 0.f};
        for (int sub = 0; sub < c.substeps; ++sub) ev |= substep<false, EXT ? -1 : 0>(s, er.p, c, u, tick, d, sub, zero3);
    }

    // ---- pair pass: collisions (S9, S10) and K nearest neighbours (S11)
    uint64_t best[QS_MAX_K];
#pragma unroll
    for (int k = 0; k < QS_MAX_K; ++k) best[k] = ~0ull;
    if (W > 1) {
        if (act) {
            sx[threadIdx.x] = s.x[0];
            sx[nt + threadIdx.x] = s.x[1];
            sx[2 * nt + threadIdx.x] = s.x[2];
            sv[threadIdx.x] = s.v[0];
            sv[nt + threadIdx.x] = s.v[1];
            sv[2 * nt + threadIdx.x] = s.v[2];
        }
        __syncthreads();
        float dvs[3] = {0.f, 0.f, 0.f};
        bool responded = false, dw_hit = false;
        float dw_az = 0.f;
        if (act && N > 1) {
            const bool coll = (c.flags & QS_F_COLLISIONS) && !(EXT && (c.flags & QS_F_SMOOTH)) && !observe_only;
            const bool flag_coll = (c.flags & QS_F_COLLISIONS) && !observe_only;
            responded = pair_scan(c, s, er.p.thr, lane, N, sbase, sx, sv, nt, keff, coll, flag_coll, ev, best, dvs,
                                  dw && !observe_only, dw_az, dw_hit);
        }
        if (responded) apply_response(c, s, tick, d, dvs);
        if (dw && dw_hit && !observe_only) apply_downwash(c, s, tick, d, dw_az);
        __syncthreads();
        if (act) {  // post-collision velocities for the neighbour observation
            sv[threadIdx.x] = s.v[0];
            sv[nt + threadIdx.x] = s.v[1];
            sv[2 * nt + threadIdx.x] = s.v[2];
            if (scn && !goal_cached(gc, tau) && swap_active(dv, er.sel, e, tau)) {
                swp = true;
                myk = swap_key(c, scn_seed(dv, er.sel, e), lane);
                skey[threadIdx.x] = myk;
            }
        }
        __syncthreads();
    }
    if (!act) return;

    // ---- the drone's goal at the end of the step (Sec. III-D scenarios)
    float gl[3] = {er.g0, er.g1, er.g2};
    if (scn) {
        if (goal_cached(gc, tau)) {
            gl[0] = gc.g[0];
            gl[1] = gc.g[1];
            gl[2] = gc.g[2];
        } else {
            const int slot = swp ? swap_rank(skey, sbase, N, lane, myk) : lane;
            scenario_goal(c, dv, er.sel, e, lane, N, tau, slot, gl, gl);
            goal_cache_set(gc, dv, er.sel, e, tau, gl);
        }
    }

    // ---- S12 observation
    if (obs) {
        float ex[3] = {0.f, 0.f, 0.f}, evv[3] = {0.f, 0.f, 0.f}, ew[3] = {0.f, 0.f, 0.f};
        if (c.flags & QS_F_OBS_NOISE) obs_noise(c, tick, d, observe_only ? 1u : 0u, ex, evv, ew);
        float2* o2 = reinterpret_cast<float2*>(obs + (size_t)d * c.obs_dim);
        o2[0] = make_float2(s.x[0] - gl[0] + ex[0], s.x[1] - gl[1] + ex[1]);
        o2[1] = make_float2(s.x[2] - gl[2] + ex[2], s.v[0] + evv[0]);
        o2[2] = make_float2(s.v[1] + evv[1], s.v[2] + evv[2]);
        o2[3] = make_float2(s.R[0], s.R[1]);
        o2[4] = make_float2(s.R[2], s.R[3]);
        o2[5] = make_float2(s.R[4], s.R[5]);
        o2[6] = make_float2(s.R[6], s.R[7]);
        o2[7] = make_float2(s.R[8], s.w[0] + ew[0]);
        o2[8] = make_float2(s.w[1] + ew[1], s.w[2] + ew[2]);
#pragma unroll
        for (int k = 0; k < QS_MAX_K; ++k) {
            if (k >= K) break;
            float2* on = o2 + 9 + 3 * k;
            if (W > 1 && k < keff) {
                const int tj = sbase + (int)(best[k] & 0xffffffffu);
                on[0] = make_float2(sx[tj] - s.x[0], sx[nt + tj] - s.x[1]);
                on[1] = make_float2(sx[2 * nt + tj] - s.x[2], sv[tj] - s.v[0]);
                on[2] = make_float2(sv[nt + tj] - s.v[1], sv[2 * nt + tj] - s.v[2]);
            } else {
                on[0] = make_float2(0.f, 0.f);
                on[1] = make_float2(0.f, 0.f);
                on[2] = make_float2(0.f, 0.f);
            }
        }
    }
    if (observe_only) return;

    if ((c.flags & QS_F_RECORD_KNN) && dv.knn) {
#pragma unroll
        for (int k = 0; k < QS_MAX_K; ++k)
            if (k < K) dv.knn[(size_t)k * dv.D + d] = k < keff ? (int16_t)(best[k] & 0xffffu) : (int16_t)-1;
    }
    ev_out = ev;

    // ---- S13 reward and done
    if (rew) rew[d] = compute_reward(c, s, er.p.prox, gl, fh, ev, best, W > 1 ? keff : 0);
    end_step<EXT>(c, dv, s, er, fh, lane, e, d, done);
    if (scn && er.ep == 0) gc.until = -1;  // an auto-reset drew a new record
}

struct SlotMap {
    int slot, lane, e, d0, N, d, sbase;
    bool act;
};

__device__ __forceinline__ SlotMap map_slot(const Dev& dv, const Tile& tile, const int* __restrict__ perm, int W) {
    SlotMap m;
    m.slot = threadIdx.x / W;
    m.lane = threadIdx.x - m.slot * W;
    const SlotGeo g = slot_geometry(dv, perm, tile, m.slot, W, blockDim.x);
    m.e = g.e;
    m.d0 = g.d0;
    m.N = g.N;
    m.act = m.lane < m.N;
    m.d = m.d0 + m.lane;
    m.sbase = m.slot * W;
    return m;
}

// W = 1 (one drone per env) is HBM-bound at scale: capping it at 80 registers
// (a few dozen bytes of spills to L1) keeps 12 CTAs of 64 threads per SM in
// flight instead of 9, +18% at 1M envs.
template <int W, bool EXT>
__global__ void __launch_bounds__(MAX_BLOCK, (W == 1 ? 3 : 1)) k_step(const Consts c, const Dev dv, const Tile* __restrict__ tiles,
                                                    const int* __restrict__ perm, const StepIO io, const int observe_only) {
    extern __shared__ float sm[];
    const SlotMap m = map_slot(dv, tile_at(dv, tiles, blockIdx.x, blockDim.x), perm, W);
    Drone s;
    EnvRegs er;
    uint32_t ev = 0;
    if (m.act) {
        load_drone(s, dv.st, dv.D, m.d);
        load_env<EXT>(er, c, dv, m.e);
    }
    const float4 a = (m.act && !observe_only) ? __ldg(reinterpret_cast<const float4*>(io.act) + m.d)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
    GoalCache gc{{0.f, 0.f, 0.f}, 0, -1};
    step_body<EXT>(W, c, dv, s, er, ev, sm, sm + 3 * blockDim.x, m.act, m.lane, m.N, m.sbase, m.e, m.d, a, io.obs,
              io.rew, io.done, observe_only, gc);
    if (!m.act || observe_only) return;
    dv.ev[m.d] = ev;
    store_drone(s, dv.st, dv.D, m.d);
    if (m.lane == 0) store_env<EXT>(er, dv, m.e);
}

// T steps of one tile with the state in registers. W1: every tile of the
// launch holds single-drone slots (a compile-time width of 1: no pair pass,
// neighbour or staging code).
template <bool EXT, bool W1>
__device__ __forceinline__ void rollout_tile(const Consts& c, const Dev& dv, const Tile& tile, const int* __restrict__ perm,
                                             float* sm, const RolloutIO& io, int t0, int nsteps) {
    const int W = W1 ? 1 : tile.W;
    const SlotMap m = map_slot(dv, tile, perm, W);
    Drone s;
    EnvRegs er;
    uint32_t ev = 0;
    if (m.act) {
        load_drone(s, dv.st, dv.D, m.d);
        load_env<EXT>(er, c, dv, m.e);
    }
    const size_t D = dv.D, E = dv.E;
    const float4* act4 = reinterpret_cast<const float4*>(io.act) + m.d;
    // the commands of step t + 1 are loaded while step t computes, so their
    // HBM latency leaves each step's dependent chain
    float4 a_next = m.act ? __ldg(act4 + (size_t)t0 * D) : make_float4(0.f, 0.f, 0.f, 0.f);
    GoalCache gc{{0.f, 0.f, 0.f}, 0, -1};
    for (int t = t0; t < t0 + nsteps; ++t) {
        const float4 a = a_next;
        if (m.act && t + 1 < t0 + nsteps) a_next = __ldg(act4 + (size_t)(t + 1) * D);
        step_body<EXT>(W, c, dv, s, er, ev, sm, sm + 3 * blockDim.x, m.act, m.lane, m.N, m.sbase, m.e, m.d, a,
                       io.obs ? io.obs + (size_t)t * D * c.obs_dim : nullptr, io.rew ? io.rew + (size_t)t * D : nullptr,
                       io.done ? io.done + (size_t)t * E : nullptr, 0, gc);
    }
    if (m.act) {
        dv.ev[m.d] = ev;
        store_drone(s, dv.st, dv.D, m.d);
        if (m.lane == 0) store_env<EXT>(er, dv, m.e);
    }
}

// Persistent rollout: CTAs take tiles from *counter (zeroed before the launch)
// until none is left. Tiles are ordered costliest first. The W1 instance
// (EXT = false only) serves handles whose envs all hold one drone: 107
// registers instead of 121 and no untaken swarm code in the step loop (with
// the smooth contacts compiled out of the EXT = false instances, batched
// 1,048,576 single-drone envs went from 1.75e10 to 1.90e10 quadrotor-steps/s,
// each change about half of it).
template <bool EXT, bool W1>
__global__ void __launch_bounds__(MAX_BLOCK, 2) k_rollout(const Consts c, const Dev dv, const Tile* __restrict__ tiles,
                                                       const int n_tiles, const int* __restrict__ perm,
                                                       int* __restrict__ counter, const RolloutIO io, const int t0,
                                                       const int nsteps) {
    extern __shared__ float sm[];
    __shared__ int s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
        __syncthreads();
        const int ti = s_next;
        __syncthreads();  // everyone has read s_next before thread 0 overwrites it
        if (ti >= n_tiles) return;
        rollout_tile<EXT, W1>(c, dv, tile_at(dv, tiles, ti, blockDim.x), perm, sm, io, t0, nsteps);
    }
}

// ---------------------------------------------------------------- warp-specialised step
// A CTA of 2P warps steps up to 32P drones: slots of width W <= 32P laid over
// the drone lanes of warps 0 .. P-1 (dynamics), which carry one drone per lane
// through the substeps and the pair pass. Warps P .. 2P-1 (noise) draw the
// motor-noise normals of the first WS_SUB substeps into shared memory ahead of
// the dynamics, then the observation noise while the dynamics run, and finally
// assemble the observation rows of the CTA's drones in shared memory and store
// them; when the CTA's drones are contiguous in memory the rows form one block
// written with 16-byte stores. The two sides meet at two CTA barriers: after
// the motor normals (B1) and after the dynamics warps publish the final states
// (B2). This takes the Philox and Box-Muller work off each drone's dependent
// chain. With P = 2 (swarms of 33..64) the dynamics warps also meet at named
// barrier 1 between staging and reading each other's positions, and the noise
// warps at named barrier 2 before storing the block of rows.
constexpr int WS_SUB = 4;
constexpr int WS_OBS_MAX = 18 + 6 * QS_MAX_K;

template <int P>
struct WsShared {
    float nrm[2][WS_SUB][4][32 * P];  // motor-noise normals [buffer][substep][rotor][drone lane]
    // the published end of a step, [buffer] by step parity:
    float st[2][18][32 * P];          // x v R w of each drone lane after the step (post-collision)
    float g[2][3][32 * P];            // goal of each lane's drone
    int nb[2][QS_MAX_K][32 * P];      // CTA drone lane of each neighbour
    int keff[2][32 * P];
    float rin[2][9][32 * P];          // reward inputs: command f^ (4), previous command (4), proximity radius
    uint32_t ev[2][32 * P];           // event bits
    float sx[3][32 * P];              // pair-pass staging: positions
    float sv[3][32 * P];              //                    velocities
    uint32_t key[32 * P];             // swap keys
    float rows[32 * P * WS_OBS_MAX];
};

// Barrier among the P warps of one side (id 1: dynamics, id 2: noise); one
// warp only needs its own lanes converged.
template <int P>
__device__ __forceinline__ void side_sync(int id) {
    if (P == 1)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(32 * P) : "memory");
}

// Slot geometry of a warp-specialised CTA: drone lane L (0 .. 32P-1) of both
// sides stands for slot-local drone `lane` of slot `slot` (W lanes per slot).
struct WsMap {
    int W, L, slot, lane, e, d0, N, d, sbase;
    bool act;
};

template <int P>
__device__ __forceinline__ WsMap ws_map(const Dev& dv, const Tile& tile, const int* __restrict__ perm) {
    WsMap m;
    m.W = tile.W;
    m.L = threadIdx.x & (32 * P - 1);
    m.slot = m.L / m.W;
    m.lane = m.L - m.slot * m.W;
    const SlotGeo g = slot_geometry(dv, perm, tile, m.slot, m.W, 32 * P);
    m.e = g.e;
    m.d0 = g.d0;
    m.N = g.N;
    m.act = m.lane < m.N;
    m.d = m.d0 + m.lane;
    m.sbase = m.slot * m.W;
    return m;
}

// Noise side: the motor-noise normals of the first WS_SUB substeps of the
// step at Philox counter `tick`, into shared-memory buffer nb.
template <int P>
__device__ __forceinline__ void ws_motor_normals(const Consts& c, WsShared<P>& sh, const WsMap& m, uint32_t tick,
                                                 int nb) {
    if (!m.act || !(c.flags & QS_F_MOTOR_NOISE)) return;
    const int nahead = min(c.substeps, WS_SUB);
    for (int sub = 0; sub < nahead; ++sub) {
        float n[4];
        motor_normals(c, tick, m.d, sub, n);
        sh.nrm[nb][sub][0][m.L] = n[0];
        sh.nrm[nb][sub][1][m.L] = n[1];
        sh.nrm[nb][sub][2][m.L] = n[2];
        sh.nrm[nb][sub][3][m.L] = n[3];
    }
}

// Noise side, after B2: the observation rows of the CTA's drones from the
// published post-step states plus sensor noise, assembled in shared memory and
// stored to obs; when the CTA's drones are contiguous the rows form one block
// written with 16-byte stores.
template <int P>
__device__ __forceinline__ void ws_store_obs(const Consts& c, const Dev& dv, const Tile& tile,
                                             const int* __restrict__ perm, WsShared<P>& sh, const WsMap& m, int b,
                                             float* __restrict__ obs, const float ex[3], const float evv[3],
                                             const float ew[3]) {
    const int od = c.obs_dim, K = c.K, L = m.L;
    const float(&st)[18][32 * P] = sh.st[b];
    const bool contig = tile.pad != 0 &&
                        qs_check(dv.status, tile.first >= 0 && tile.count >= 1 && tile.first + tile.count <= dv.E);
    const int d_first = contig ? env_first(dv, slot_env(dv, perm, tile.first)) : 0;
    const int ridx = contig ? m.d - d_first : L;
    if (m.act) {
        float* row = sh.rows + ridx * od;
        row[0] = st[0][L] - sh.g[b][0][L] + ex[0];
        row[1] = st[1][L] - sh.g[b][1][L] + ex[1];
        row[2] = st[2][L] - sh.g[b][2][L] + ex[2];
        row[3] = st[3][L] + evv[0];
        row[4] = st[4][L] + evv[1];
        row[5] = st[5][L] + evv[2];
        for (int k = 6; k < 15; ++k) row[k] = st[k][L];
        row[15] = st[15][L] + ew[0];
        row[16] = st[16][L] + ew[1];
        row[17] = st[17][L] + ew[2];
        const int ke = sh.keff[b][L];
        for (int k = 0; k < K; ++k) {
            float* on = row + 18 + 6 * k;
            if (k < ke) {
                const int j = sh.nb[b][k][L];
                for (int q = 0; q < 6; ++q) on[q] = st[q][j] - st[q][L];
            } else {
                for (int q = 0; q < 6; ++q) on[q] = 0.f;
            }
        }
    }
    side_sync<P>(2);
    const int e_last = contig ? slot_env(dv, perm, tile.first + tile.count - 1) : 0;
    const int d_end = contig ? env_first(dv, e_last + 1) : 0;
    if (contig && qs_check(dv.status, d_first >= 0 && d_end <= dv.D && d_end - d_first <= 32 * P)) {
        const int n_floats = (d_end - d_first) * od;
        float* dst = obs + (size_t)d_first * od;
        if (((uintptr_t)dst & 15u) == 0) {
            const int n4 = n_floats >> 2;
            const float4* src4 = reinterpret_cast<const float4*>(sh.rows);
            float4* dst4 = reinterpret_cast<float4*>(dst);
            for (int i = L; i < n4; i += 32 * P) dst4[i] = src4[i];
            for (int i = (n4 << 2) + L; i < n_floats; i += 32 * P) dst[i] = sh.rows[i];
        } else {
            const int n2 = n_floats >> 1;  // obs rows hold an even number of floats
            const float2* src2 = reinterpret_cast<const float2*>(sh.rows);
            float2* dst2 = reinterpret_cast<float2*>(dst);
            for (int i = L; i < n2; i += 32 * P) dst2[i] = src2[i];
        }
    } else if (m.act && !contig) {
        const float2* src2 = reinterpret_cast<const float2*>(sh.rows + ridx * od);
        float2* dst2 = reinterpret_cast<float2*>(obs + (size_t)m.d * od);
        for (int i = 0; i < od / 2; ++i) dst2[i] = src2[i];
    }
}

// Dynamics side: one control step of the lane's drone with command a and the
// motor normals of buffer nb. Meets the noise side at B1 (motor normals ready)
// and B2 (post-step state, goal and neighbours published for the observation
// rows), then writes the knn record, reward and done and ends the step. Every
// thread of the dynamics warps calls it.
template <bool EXT, int P, bool DEFER>
__device__ __forceinline__ void ws_dynamics_step(const Consts& c, const Dev& dv, WsShared<P>& sh, const WsMap& m,
                                                 Drone& s, EnvRegs& er, uint32_t& ev_out, const float4 a, const int nb,
                                                 float* __restrict__ rew, uint8_t* __restrict__ done, GoalCache& gc,
                                                 const bool b1 = true) {
    const int b = nb;  // the step's buffers: its motor normals and its published end
    const int W = m.W, L = m.L, lane = m.lane, N = m.N, e = m.e, d = m.d, sbase = m.sbase;
    const bool act = m.act;
    const int K = c.K;
    const int nahead = min(c.substeps, WS_SUB);
    const bool mnoise = (c.flags & QS_F_MOTOR_NOISE) != 0;
    const bool dw = EXT && (c.flags & QS_F_DOWNWASH) != 0;  // EXT = false: no downwash or scenario code
    float fh[4] = {0.f, 0.f, 0.f, 0.f}, u[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t ev = 0;
    if (act) {
        fh[0] = command(c, a.x);
        fh[1] = command(c, a.y);
        fh[2] = command(c, a.z);
        fh[3] = command(c, a.w);
        u[0] = sqrt_approx(fh[0]);
        u[1] = sqrt_approx(fh[1]);
        u[2] = sqrt_approx(fh[2]);
        u[3] = sqrt_approx(fh[3]);
    }
    if (b1) __syncthreads();  // B1: motor normals ready (the rollout's later steps: drawn before the last B2)
    // smooth contacts of a swarm (general instance): the pair penalty from the
    // positions at each substep's start, staged like the pair pass
    const bool spair = EXT && (c.flags & QS_F_SMOOTH) && W > 1;
    if (spair) {
        for (int sub = 0; sub < c.substeps; ++sub) {
            float pacc[3] = {0.f, 0.f, 0.f};
            if (act) {
                sh.sx[0][L] = s.x[0];
                sh.sx[1][L] = s.x[1];
                sh.sx[2][L] = s.x[2];
            }
            side_sync<P>(1);
            if (act && N > 1) pair_acc(c, s.x, &sh.sx[0][0], 32 * P, sbase, lane, N, er.p.arm, pacc);
            side_sync<P>(1);
            if (act) {
                if (mnoise && sub < nahead) {
                    const float n[4] = {sh.nrm[nb][sub][0][L], sh.nrm[nb][sub][1][L], sh.nrm[nb][sub][2][L],
                                        sh.nrm[nb][sub][3][L]};
                    ev |= substep<false, EXT ? -1 : 0>(s, er.p, c, u, er.tick, d, sub, pacc, n);
                } else {
                    ev |= substep<false, EXT ? -1 : 0>(s, er.p, c, u, er.tick, d, sub, pacc);
                }
            }
        }
    } else if (act) {
        const float zero3[3] = {0.f, 0.f, 0.f};
        for (int sub = 0; sub < c.substeps; ++sub) {
            if (mnoise && sub < nahead) {
                const float n[4] = {sh.nrm[nb][sub][0][L], sh.nrm[nb][sub][1][L], sh.nrm[nb][sub][2][L],
                                    sh.nrm[nb][sub][3][L]};
                ev |= substep<false, EXT ? -1 : 0>(s, er.p, c, u, er.tick, d, sub, zero3, n);
            } else {
                ev |= substep<false, EXT ? -1 : 0>(s, er.p, c, u, er.tick, d, sub, zero3);
            }
        }
    }
    const int keff = min(K, N - 1);
    uint64_t best[QS_MAX_K];
#pragma unroll
    for (int k = 0; k < QS_MAX_K; ++k) best[k] = ~0ull;
    if (W > 1) {
        if (act) {
            sh.sx[0][L] = s.x[0];
            sh.sx[1][L] = s.x[1];
            sh.sx[2][L] = s.x[2];
            sh.sv[0][L] = s.v[0];
            sh.sv[1][L] = s.v[1];
            sh.sv[2][L] = s.v[2];
        }
        side_sync<P>(1);
        float dvs[3] = {0.f, 0.f, 0.f};
        bool responded = false, dw_hit = false;
        float dw_az = 0.f;
        if (act && N > 1) {
            const bool coll = (c.flags & QS_F_COLLISIONS) && !(EXT && (c.flags & QS_F_SMOOTH));
            const bool flag_coll = (c.flags & QS_F_COLLISIONS) != 0;
            responded = pair_scan(c, s, er.p.thr, lane, N, sbase, &sh.sx[0][0], &sh.sv[0][0], 32 * P, keff, coll,
                                  flag_coll, ev, best, dvs, dw, dw_az, dw_hit);
        }
        if (responded) apply_response(c, s, er.tick, d, dvs);
        if (dw && dw_hit) apply_downwash(c, s, er.tick, d, dw_az);
    }
    // the drone's goal at the end of the step (Sec. III-D scenarios)
    float gl[3] = {er.g0, er.g1, er.g2};
    if (EXT && (c.scn_mask & ~1u)) {
        const int tau = er.ep + 1;
        const bool hit = goal_cached(gc, tau);  // the same for every lane of an env
        bool swp = false;
        uint32_t myk = 0;
        if (W > 1) {
            if (act && !hit && swap_active(dv, er.sel, e, tau)) {
                swp = true;
                myk = swap_key(c, scn_seed(dv, er.sel, e), lane);
                sh.key[L] = myk;
            }
            side_sync<P>(1);
        }
        if (act && hit) {
            gl[0] = gc.g[0];
            gl[1] = gc.g[1];
            gl[2] = gc.g[2];
        } else if (act) {
            const int slot = swp ? swap_rank(sh.key, sbase, N, lane, myk) : lane;
            scenario_goal(c, dv, er.sel, e, lane, N, tau, slot, gl, gl);
            goal_cache_set(gc, dv, er.sel, e, tau, gl);
        }
    }
    if (act) {  // publish the observed state (post-collision) for the noise side
        const float v18[18] = {s.x[0], s.x[1], s.x[2], s.v[0], s.v[1], s.v[2], s.R[0], s.R[1], s.R[2],
                               s.R[3], s.R[4], s.R[5], s.R[6], s.R[7], s.R[8], s.w[0], s.w[1], s.w[2]};
#pragma unroll
        for (int k = 0; k < 18; ++k) sh.st[b][k][L] = v18[k];
        sh.g[b][0][L] = gl[0];
        sh.g[b][1][L] = gl[1];
        sh.g[b][2][L] = gl[2];
        sh.keff[b][L] = W > 1 ? keff : 0;
#pragma unroll
        for (int k = 0; k < QS_MAX_K; ++k)
            if (k < keff) sh.nb[b][k][L] = sbase + (int)(best[k] & 0xffffffffu);
        if (DEFER) {  // the noise side computes the reward from these
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                sh.rin[b][r][L] = fh[r];
                sh.rin[b][4 + r][L] = s.fp[r];
            }
            sh.rin[b][8][L] = er.p.prox;
            sh.ev[b][L] = ev;
        }
    }
    __syncthreads();  // B2
    if (!act) return;
    if ((c.flags & QS_F_RECORD_KNN) && dv.knn) {
#pragma unroll
        for (int k = 0; k < QS_MAX_K; ++k)
            if (k < K) dv.knn[(size_t)k * dv.D + d] = (W > 1 && k < keff) ? (int16_t)(best[k] & 0xffffu) : (int16_t)-1;
    }
    if (!DEFER && rew) rew[d] = compute_reward(c, s, er.p.prox, gl, fh, ev, best, W > 1 ? keff : 0);
    end_step<EXT>(c, dv, s, er, fh, lane, e, d, done);
    if (EXT && er.ep == 0) gc.until = -1;  // an auto-reset drew a new record
    ev_out = ev;
}

// Noise side: the reward of the step published in buffer b (the same
// compute_reward as the dynamics side, on the published post-step state; the
// neighbour keys recomputed with the canonical pair key on the same positions).
template <int P>
__device__ __forceinline__ void ws_reward(const Consts& c, WsShared<P>& sh, const WsMap& m, int b,
                                          float* __restrict__ rew) {
    if (!m.act) return;
    const int L = m.L;
    Drone s;
    for (int k = 0; k < 3; ++k) {
        s.x[k] = sh.st[b][k][L];
        s.v[k] = sh.st[b][3 + k][L];
        s.w[k] = sh.st[b][15 + k][L];
    }
    for (int k = 0; k < 9; ++k) s.R[k] = sh.st[b][6 + k][L];
    float fh[4];
    for (int r = 0; r < 4; ++r) {
        fh[r] = sh.rin[b][r][L];
        s.fp[r] = sh.rin[b][4 + r][L];
    }
    const float g[3] = {sh.g[b][0][L], sh.g[b][1][L], sh.g[b][2][L]};
    const int keff = sh.keff[b][L];
    uint64_t best[QS_MAX_K];
#pragma unroll
    for (int k = 0; k < QS_MAX_K; ++k) {
        best[k] = ~0ull;
        if (k < keff) {
            const int j = sh.nb[b][k][L];
            float dx, dy, dz;
            const float key = pair_key(s.x[0], s.x[1], s.x[2], sh.st[b][0][j], sh.st[b][1][j], sh.st[b][2][j], dx, dy, dz);
            best[k] = (uint64_t)__float_as_uint(key) << 32;
        }
    }
    rew[m.d] = compute_reward(c, s, sh.rin[b][8][L], g, fh, sh.ev[b][L], best, keff);
}

template <bool EXT>
__global__ void __launch_bounds__(64) k_step_ws(const Consts c, const Dev dv, const Tile* __restrict__ tiles,
                                                const int* __restrict__ perm, const StepIO io) {
    __shared__ WsShared<1> sh;
    const Tile tile = tile_at(dv, tiles, blockIdx.x, 32);
    const WsMap m = ws_map<1>(dv, tile, perm);
    if (threadIdx.x >= 32) {
        // ---------------- noise warp
        const uint32_t tick = m.act ? dv.tick[m.e] : 0u;  // warp 0 writes it only after B2
        ws_motor_normals<1>(c, sh, m, tick, 0);
        __syncthreads();  // B1
        float ex[3] = {0.f, 0.f, 0.f}, evv[3] = {0.f, 0.f, 0.f}, ew[3] = {0.f, 0.f, 0.f};
        if (m.act && io.obs && (c.flags & QS_F_OBS_NOISE)) obs_noise(c, tick, m.d, 0u, ex, evv, ew);
        __syncthreads();  // B2
        if (io.obs) ws_store_obs<1>(c, dv, tile, perm, sh, m, 0, io.obs, ex, evv, ew);
        return;
    }
    // ---------------- dynamics warp
    Drone s;
    EnvRegs er;
    uint32_t ev = 0;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m.act) {
        load_drone(s, dv.st, dv.D, m.d);
        load_env<EXT>(er, c, dv, m.e);
        a = __ldg(reinterpret_cast<const float4*>(io.act) + m.d);
    }
    GoalCache gc{{0.f, 0.f, 0.f}, 0, -1};
    ws_dynamics_step<EXT, 1, false>(c, dv, sh, m, s, er, ev, a, 0, io.rew, io.done, gc);
    if (!m.act) return;
    dv.ev[m.d] = ev;
    store_drone(s, dv.st, dv.D, m.d);
    if (m.lane == 0) store_env<EXT>(er, dv, m.e);
}

// Persistent warp-specialised rollout for latency-bound handles (every swarm
// class at most 32P wide): one CTA per tile of 32P drone lanes runs steps
// t0 .. t0 + nsteps - 1 with the drones in the dynamics warps' registers.
// While the dynamics side integrates step t, the noise side draws step t's
// sensor noise and step t + 1's motor normals (double-buffered) and finishes
// step t - 1's rewards and observation rows. For single-drone slots the two
// sides meet once per step, at B2 (and at B1 before the first step): step
// t + 1's normals are drawn before B2 of step t, so the noise side's work for
// a step overlaps the dynamics side's end of the previous one (plain 8192 /
// 4864 / 2432 envs: +2% / +5% / +7%); swarm slots meet at B1 and B2 of every
// step (without B1, 3.56e9 -> 3.50e9 quadrotor-steps/s for 2048 x 8).
template <bool EXT, int P>
__global__ void __launch_bounds__(64 * P, (P == 1 ? 6 : 1)) k_rollout_ws(const Consts c, const Dev dv, const Tile* __restrict__ tiles,
                                                       const int* __restrict__ perm, const RolloutIO io, const int t0,
                                                       const int nsteps) {
    __shared__ WsShared<P> sh;
    const Tile tile = tile_at(dv, tiles, blockIdx.x, 32 * P);
    const WsMap m = ws_map<P>(dv, tile, perm);
    const size_t D = dv.D, E = dv.E;
    if (threadIdx.x >= 32 * P) {
        // ---------------- noise side; the env's Philox counter advances by one per step
        // Step t's observation rows and reward are finished during step t + 1's
        // dynamics, from the end of step t published in buffer t & 1.
        const uint32_t tick0 = m.act ? dv.tick[m.e] : 0u;  // the dynamics side writes it after the last step
        ws_motor_normals<P>(c, sh, m, tick0, 0);
        float px[3] = {0.f, 0.f, 0.f}, pv[3] = {0.f, 0.f, 0.f}, pw[3] = {0.f, 0.f, 0.f};  // step t-1's sensor noise
        for (int t = 0; t < nsteps; ++t) {
            // buffer t & 1 holds step t's normals, drawn before B2 of step t - 1:
            // B1 is needed before the first step only; swarm slots (whose
            // dynamics side takes the longer step) keep it every step, measured
            // faster there
            if (t == 0 || m.W > 1) __syncthreads();  // B1
            const uint32_t tick = tick0 + (uint32_t)t;
            float ex[3] = {0.f, 0.f, 0.f}, evv[3] = {0.f, 0.f, 0.f}, ew[3] = {0.f, 0.f, 0.f};
            if (m.act && io.obs && (c.flags & QS_F_OBS_NOISE)) obs_noise(c, tick, m.d, 0u, ex, evv, ew);
            // the other buffer was last read by the dynamics side before B2 of step t - 1
            if (t + 1 < nsteps) ws_motor_normals<P>(c, sh, m, tick + 1, (t + 1) & 1);
            if (t > 0) {
                const int pb = (t - 1) & 1;
                if (io.obs) ws_store_obs<P>(c, dv, tile, perm, sh, m, pb, io.obs + (size_t)(t0 + t - 1) * D * c.obs_dim,
                                            px, pv, pw);
                if (io.rew) ws_reward<P>(c, sh, m, pb, io.rew + (size_t)(t0 + t - 1) * D);
            }
            for (int k = 0; k < 3; ++k) {
                px[k] = ex[k];
                pv[k] = evv[k];
                pw[k] = ew[k];
            }
            __syncthreads();  // B2 of step t
        }
        if (nsteps > 0) {  // the last step, after its B2
            const int pb = (nsteps - 1) & 1;
            if (io.obs)
                ws_store_obs<P>(c, dv, tile, perm, sh, m, pb, io.obs + (size_t)(t0 + nsteps - 1) * D * c.obs_dim, px, pv, pw);
            if (io.rew) ws_reward<P>(c, sh, m, pb, io.rew + (size_t)(t0 + nsteps - 1) * D);
        }
        return;
    }
    // ---------------- dynamics side
    Drone s;
    EnvRegs er;
    uint32_t ev = 0;
    if (m.act) {
        load_drone(s, dv.st, dv.D, m.d);
        load_env<EXT>(er, c, dv, m.e);
    }
    const float4* act4 = reinterpret_cast<const float4*>(io.act) + m.d;
    float4 a_next = m.act ? __ldg(act4 + (size_t)t0 * D) : make_float4(0.f, 0.f, 0.f, 0.f);
    GoalCache gc{{0.f, 0.f, 0.f}, 0, -1};
    for (int t = 0; t < nsteps; ++t) {
        const float4 a = a_next;
        if (m.act && t + 1 < nsteps) a_next = __ldg(act4 + (size_t)(t0 + t + 1) * D);
        ws_dynamics_step<EXT, P, true>(c, dv, sh, m, s, er, ev, a, t & 1,
                                 io.rew ? io.rew + (size_t)(t0 + t) * D : nullptr,
                                 io.done ? io.done + (size_t)(t0 + t) * E : nullptr, gc, t == 0 || m.W > 1);
    }
    if (!m.act) return;
    dv.ev[m.d] = ev;
    store_drone(s, dv.st, dv.D, m.d);
    if (m.lane == 0) store_env<EXT>(er, dv, m.e);
}

// ---------------------------------------------------------------- resident step server
// A synchronous host loop (post commands, wait, read the outputs) pays a
// launch and a completion round trip per step on the per-call path. The
// server is one cooperative launch of the warp-specialised CTAs that keeps the
// drones in the dynamics warps' registers and steps them each time the host
// posts a step, with commands read from and outputs written to page-locked
// host memory in place. Handshake words in page-locked host memory: `go`
// holds in its low half the steps the host has posted (SERVE_STOP: end the
// launch; SERVE_IDLE: the server retired after waiting too long) and in its
// high half the command slot of the last posted step; `fin` counts the
// steps completed, written by the last CTA to finish each step (found with a
// counter in device memory). Only CTA 0 polls `go` over the host link; it
// relays what it reads through a word in device memory that the other CTAs
// poll (one reader of the host's line instead of one per CTA). Measured on
// GB300 at 8192 single-drone envs: one system-scope fence per CTA instead of
// one per thread, and the relay instead of every CTA polling the host, took a
// posted step from 15.8 to 11.1 us, and an acquire-release count instead of
// a second system-scope fence in the last CTA a synchronous host loop from
// 11.5 to 11.0 us per step; a completion byte
// per CTA polled by the host instead of the counter and fin was slower (11.7
// us: 64 CTAs write each line the host re-reads), and so were several reads
// of go (or of the relay) kept in flight at once instead of one (7.2 -> 11.2
// us for a one-CTA server: the reads keep taking the line from the host
// while it posts).
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_sys(int* p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long atom_add_acq_rel_gpu(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ void st_release_gpu(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// The step count (or stop code) and the command slot of a go word.
__device__ __forceinline__ int go_steps(unsigned long long v) { return (int)(unsigned int)(v & 0xffffffffull); }
__device__ __forceinline__ int go_slot(unsigned long long v) { return (int)(unsigned int)(v >> 32); }

// Thread 0 of CTAs other than 0: the relayed value once it leaves `posted`.
// CTA 0 relays every value it acts on, so this wait ends once CTA 0's does;
// its bound (4 idle_ns + 1 s, well past CTA 0's) only guards against a CTA 0
// that stopped answering, after which the CTA stops as if the server had
// retired.
__device__ __forceinline__ unsigned long long serve_follow(const unsigned long long* relay, int posted, long long idle_ns) {
    const unsigned long long t0 = global_ns(), limit = 4ull * (unsigned long long)idle_ns + 1000000000ull;
    for (;;) {
        const unsigned long long v = ld_acquire_gpu(relay);
        if (go_steps(v) != posted) return v;
        if (global_ns() - t0 > limit) return (unsigned long long)(unsigned int)SERVE_IDLE;
        __nanosleep(64);
    }
}

// Thread 0 of CTA 0: the value of `go` once its step count leaves `posted`
// (the steps already run). After idle_ns without an answer the server retires
// by swapping go from the value it last read to SERVE_IDLE; the swap fails
// only when the host posted a step (or stopped) first, so every CTA of the
// launch sees one outcome.
__device__ __forceinline__ unsigned long long serve_wait(unsigned long long* go, int posted, long long idle_ns) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        const unsigned long long v = ld_acquire_sys(go);
        if (go_steps(v) != posted) return v;
        if (global_ns() - t0 > (unsigned long long)idle_ns) {
            const unsigned long long idle = (v & ~0xffffffffull) | (unsigned long long)(unsigned int)SERVE_IDLE;
            const unsigned long long old = atomicCAS_system(go, v, idle);
            __threadfence_system();
            return old == v ? idle : old;
        }
        __nanosleep(32);
    }
}

// Step k of the launch (global step k0 + k): B0 (the host posted it; the
// noise side has drawn its motor normals into buffer k & 1), the per-call
// warp-specialised step (B1, B2) with the observation rows of step k stored
// by the noise side after B2 and the next step's normals drawn after them,
// then B3, after which thread 0 fences the CTA's host writes at system scope
// and counts the CTA done; the last CTA publishes fin = k0 + k + 1.
template <bool EXT, int P>
__global__ void __launch_bounds__(64 * P, (P == 1 ? 6 : 1)) k_serve(const Consts c, const Dev dv, const Tile* __restrict__ tiles,
                                                                  const int* __restrict__ perm, const ServeIO io, const int k0) {
    __shared__ WsShared<P> sh;
    __shared__ unsigned long long s_go;
    const Tile tile = tile_at(dv, tiles, blockIdx.x, 32 * P);
    const WsMap m = ws_map<P>(dv, tile, perm);
    const bool noise = threadIdx.x >= 32 * P;
    const uint32_t tick0 = (noise && m.act) ? dv.tick[m.e] : 0u;  // the dynamics side writes it back at the end
    Drone s;
    EnvRegs er;
    uint32_t ev = 0;
    GoalCache gc{{0.f, 0.f, 0.f}, 0, -1};
    if (!noise && m.act) {
        load_drone(s, dv.st, dv.D, m.d);
        load_env<EXT>(er, c, dv, m.e);
    }
    if (noise) ws_motor_normals<P>(c, sh, m, tick0, 0);
    for (int k = 0;; ++k) {
        if (threadIdx.x == 0) {
            if (blockIdx.x == 0) {
                s_go = serve_wait(io.go, k0 + k, io.idle_ns);
                st_release_gpu(io.relay, s_go);
            } else {
                s_go = serve_follow(io.relay, k0 + k, io.idle_ns);
            }
        }
        __syncthreads();  // B0
        const unsigned long long g = s_go;
        // SERVE_STOP, SERVE_IDLE, or a slot the host never checked
        if (go_steps(g) != k0 + k + 1 || go_slot(g) >= io.n_slots) break;
        const int b = k & 1;
        if (noise) {
            const uint32_t tick = tick0 + (uint32_t)k;
            __syncthreads();  // B1
            float ex[3] = {0.f, 0.f, 0.f}, evv[3] = {0.f, 0.f, 0.f}, ew[3] = {0.f, 0.f, 0.f};
            if (m.act && io.obs && (c.flags & QS_F_OBS_NOISE)) obs_noise(c, tick, m.d, 0u, ex, evv, ew);
            __syncthreads();  // B2
            if (io.obs) ws_store_obs<P>(c, dv, tile, perm, sh, m, b, io.obs, ex, evv, ew);
            ws_motor_normals<P>(c, sh, m, tick + 1, b ^ 1);
        } else {
            // the host's commands of this step: fetched again, never from a cached line
            const float4* act4 = reinterpret_cast<const float4*>(io.act + (size_t)go_slot(g) * 4 * dv.D) + m.d;
            const float4 a = m.act ? __ldcv(act4) : make_float4(0.f, 0.f, 0.f, 0.f);
            ws_dynamics_step<EXT, P, false>(c, dv, sh, m, s, er, ev, a, b, io.rew, io.done, gc);
        }
        __syncthreads();  // B3
        if (threadIdx.x == 0) {
            // the CTA's host writes of the step (ordered before it by B3) performed
            // at system scope before its count; the count's acquire side orders
            // every CTA's count before the last one's release of fin
            __threadfence_system();
            const unsigned long long n = atom_add_acq_rel_gpu(io.count, 1ull) + 1ull;
            if (n == (unsigned long long)gridDim.x * (unsigned long long)(k + 1)) st_release_sys(io.fin, k0 + k + 1);
        }
    }
    if (noise || !m.act) return;
    dv.ev[m.d] = ev;
    store_drone(s, dv.st, dv.D, m.d);
    if (m.lane == 0) store_env<EXT>(er, dv, m.e);
}

cudaError_t launch_serve(const Consts& c, const Dev& dv, const Tile* tiles, int n_tiles, int P, const int* perm,
                         const ServeIO& io, int k0, cudaStream_t st) {
    const bool ext = extended(c);
    const void* fn = P == 1 ? (ext ? (const void*)k_serve<true, 1> : (const void*)k_serve<false, 1>)
                            : (ext ? (const void*)k_serve<true, 2> : (const void*)k_serve<false, 2>);
    if (P != 1 && P != 2) return cudaErrorInvalidValue;
    Consts cc = c;
    Dev dd = dv;
    ServeIO ii = io;
    const Tile* tt = tiles;
    const int* pp = perm;
    int kk = k0;
    void* args[] = {&cc, &dd, &tt, &pp, &ii, &kk};
    return cudaLaunchCooperativeKernel(fn, dim3(n_tiles), dim3(64 * P), args, 0, st);
}

int serve_resident_ctas(const Consts& c, int P) {
    int dev = 0, n_sm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const bool ext = extended(c);
    const void* fn = P == 1 ? (ext ? (const void*)k_serve<true, 1> : (const void*)k_serve<false, 1>)
                            : (ext ? (const void*)k_serve<true, 2> : (const void*)k_serve<false, 2>);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 64 * P, 0) != cudaSuccess) return 0;
    return occ * n_sm;
}

int rollout_ws_resident_ctas(const Consts& c, int P) {
    int dev = 0, n_sm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const bool ext = extended(c);
    const void* fn = P == 1 ? (ext ? (const void*)k_rollout_ws<true, 1> : (const void*)k_rollout_ws<false, 1>)
                            : (ext ? (const void*)k_rollout_ws<true, 2> : (const void*)k_rollout_ws<false, 2>);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 64 * P, 0) != cudaSuccess) return 0;
    return occ * n_sm;
}

template <bool EXT>
cudaError_t launch_k_step(const Consts& c, const Dev& dv, const ClassPlan& cp, const Tile* t, const int* perm,
                          const StepIO& io, int observe_only, size_t smem, cudaStream_t st) {
    switch (cp.W) {
        case 1: k_step<1, EXT><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 2: k_step<2, EXT><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 4: k_step<4, EXT><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 8: k_step<8, EXT><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 16: k_step<16, EXT><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 32: k_step<32, EXT><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 64: k_step<64, EXT><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 128: k_step<128, EXT><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_step(const Consts& c, const Dev& dv, const ClassPlan& cp, const Tile* tiles, const int* perm,
                        const StepIO& io, int observe_only, cudaStream_t st) {
    if (cp.n_tiles == 0) return cudaSuccess;
    const bool ext = extended(c);
    if (cp.ws && !observe_only) {
        if (ext)
            k_step_ws<true><<<cp.n_tiles, 64, 0, st>>>(c, dv, tiles + cp.tile_off, perm, io);
        else
            k_step_ws<false><<<cp.n_tiles, 64, 0, st>>>(c, dv, tiles + cp.tile_off, perm, io);
        return cudaGetLastError();
    }
    const size_t smem = (cp.W > 1) ? sizeof(float) * SMEM_PLANES * cp.block : 0;
    const Tile* t = tiles + cp.tile_off;
    return ext ? launch_k_step<true>(c, dv, cp, t, perm, io, observe_only, smem, st)
               : launch_k_step<false>(c, dv, cp, t, perm, io, observe_only, smem, st);
}

// The k_rollout instance for a handle: the general one, or without scenarios,
// downwash and smooth contacts, and of those the single-drone one.
const void* rollout_kernel(bool ext, bool single) {
    if (ext) return (const void*)k_rollout<true, false>;
    return single ? (const void*)k_rollout<false, true> : (const void*)k_rollout<false, false>;
}

int rollout_grid(int block, bool ext, bool single) {
    int dev = 0, n_sm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rollout_kernel(ext, single), block,
                                                  sizeof(float) * SMEM_PLANES * block);
    return (occ > 0 ? occ : 1) * n_sm;
}

cudaError_t launch_rollout_ws(const Consts& c, const Dev& dv, const Tile* tiles, int n_tiles, int P, const int* perm,
                              const RolloutIO& io, int t0, int nsteps, cudaStream_t st) {
    if (n_tiles == 0) return cudaSuccess;
    const bool ext = extended(c);
    if (P == 1) {
        if (ext)
            k_rollout_ws<true, 1><<<n_tiles, 64, 0, st>>>(c, dv, tiles, perm, io, t0, nsteps);
        else
            k_rollout_ws<false, 1><<<n_tiles, 64, 0, st>>>(c, dv, tiles, perm, io, t0, nsteps);
    } else if (P == 2) {
        if (ext)
            k_rollout_ws<true, 2><<<n_tiles, 128, 0, st>>>(c, dv, tiles, perm, io, t0, nsteps);
        else
            k_rollout_ws<false, 2><<<n_tiles, 128, 0, st>>>(c, dv, tiles, perm, io, t0, nsteps);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rollout(const Consts& c, const Dev& dv, const Tile* tiles, int n_tiles, int block, const int* perm,
                           int* counter, const RolloutIO& io, int t0, int nsteps, int grid, bool single,
                           cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(float) * SMEM_PLANES * block;
    const int g = grid > 0 ? grid : n_tiles;
    const int grid_n = g < n_tiles ? g : n_tiles;
    if (extended(c))
        k_rollout<true, false><<<grid_n, block, smem, st>>>(c, dv, tiles, n_tiles, perm, counter, io, t0, nsteps);
    else if (single)
        k_rollout<false, true><<<grid_n, block, smem, st>>>(c, dv, tiles, n_tiles, perm, counter, io, t0, nsteps);
    else
        k_rollout<false, false><<<grid_n, block, smem, st>>>(c, dv, tiles, n_tiles, perm, counter, io, t0, nsteps);
    return cudaGetLastError();
}

}  // namespace qsk
