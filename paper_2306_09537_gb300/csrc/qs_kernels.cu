// qs_kernels.cu -- sm_103a kernels of the QuadSwarm step: reset, the fused
// control step, state access.
//
// Step kernel layout: a CTA processes envs of one width class W (a power of
// two >= the env's swarm size). Each env owns a "slot" of W consecutive
// threads; thread `lane` of the slot carries drone `lane` of the env in
// registers through the fused physics substeps, then the slot exchanges
// positions and velocities through shared memory for the O(N^2) pair pass
// (collisions, Sec. III-B) and the K-nearest-neighbour selection (Sec. III-C),
// which each thread keeps as a sorted register list.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace qsk {

constexpr int MAX_BLOCK = 256;

// Inserts (key, j) into the ascending list best[0..K) (64-bit key: float bits
// of the distance key << 32 | index, so equal keys order by index).
__device__ __forceinline__ void topk_insert(uint64_t best[QS_MAX_K], int K, uint64_t cand) {
#pragma unroll
    for (int k = 0; k < QS_MAX_K; ++k) {
        if (k < K && cand < best[k]) {
            const uint64_t t = best[k];
            best[k] = cand;
            cand = t;
        }
    }
}

template <int W>
__global__ void __launch_bounds__(MAX_BLOCK) k_step(const Consts c, const Dev dv, const Tile* __restrict__ tiles,
                                                    const int* __restrict__ perm, const StepIO io, const int observe_only) {
    extern __shared__ float sm[];
    const int nt = blockDim.x;
    float* sx = sm;           // [3][nt]
    float* sv = sm + 3 * nt;  // [3][nt]

    const Tile tile = tiles[blockIdx.x];
    const int slot = threadIdx.x / W, lane = threadIdx.x % W;
    const bool slot_ok = slot < tile.count;
    const int e = slot_ok ? perm[tile.first + slot] : 0;
    const int d0 = slot_ok ? dv.env_off[e] : 0;
    const int N = slot_ok ? dv.env_off[e + 1] - d0 : 0;
    const bool act = lane < N;
    const int d = d0 + lane;
    const int sbase = slot * W;
    const int K = c.K;
    const int keff = min(K, N - 1);

    Drone s;
    Prm p;
    uint32_t tick = 0;
    int ep0 = 0;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    float fh[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t ev = 0;
    if (act) {
        load_drone(s, dv.st, dv.D, d);
        p = load_prm(dv.prm, dv.E, e);
        tick = dv.tick[e];
        ep0 = dv.ep[e];
        g0 = dv.goal[e];
        g1 = dv.goal[dv.E + e];
        g2 = dv.goal[2 * dv.E + e];
        if (!observe_only) {
            const float4 a = reinterpret_cast<const float4*>(io.act)[d];
            fh[0] = command(c, a.x);
            fh[1] = command(c, a.y);
            fh[2] = command(c, a.z);
            fh[3] = command(c, a.w);
            const float u[4] = {sqrtf(fh[0]), sqrtf(fh[1]), sqrtf(fh[2]), sqrtf(fh[3])};
            const float zero3[3] = {0.f, 0.f, 0.f};
            for (int sub = 0; sub < c.substeps; ++sub) ev |= substep(s, p, c, u, tick, d, sub, zero3);
        }
    }

    // ---- pair pass: collisions (S9, S10) and K nearest neighbours (S11)
    uint64_t best[QS_MAX_K];
#pragma unroll
    for (int k = 0; k < QS_MAX_K; ++k) best[k] = ~0ull;
    if constexpr (W > 1) {
        if (act) {
            sx[threadIdx.x] = s.x[0];
            sx[nt + threadIdx.x] = s.x[1];
            sx[2 * nt + threadIdx.x] = s.x[2];
            sv[threadIdx.x] = s.v[0];
            sv[nt + threadIdx.x] = s.v[1];
            sv[2 * nt + threadIdx.x] = s.v[2];
        }
        __syncthreads();
        float dvs0 = 0.f, dvs1 = 0.f, dvs2 = 0.f;
        bool responded = false;
        if (act && N > 1) {
            const bool coll = (c.flags & QS_F_COLLISIONS) && !(c.flags & QS_F_SMOOTH) && !observe_only;
            const bool flag_coll = (c.flags & QS_F_COLLISIONS) && !observe_only;
            for (int j = 0; j < N; ++j) {
                if (j == lane) continue;
                const int tj = sbase + j;
                float dx, dy, dz;
                const float key = pair_key(s.x[0], s.x[1], s.x[2], sx[tj], sx[nt + tj], sx[2 * nt + tj], dx, dy, dz);
                if (flag_coll && key < p.thr) {
                    ev |= EV_HIT_QUAD;
                    if (coll) {
                        // approaching iff (v_i - v_j) . (x_i - x_j) < 0
                        const float rv0 = s.v[0] - sv[tj], rv1 = s.v[1] - sv[nt + tj], rv2 = s.v[2] - sv[2 * nt + tj];
                        const float app = -(rv0 * dx + rv1 * dy + rv2 * dz);
                        if (app < 0.0f) {
                            float n0 = 0.f, n1 = 0.f, n2 = 1.f;
                            if (key > 0.0f) {
                                const float inv = rsqrtf(key);
                                n0 = -dx * inv;
                                n1 = -dy * inv;
                                n2 = -dz * inv;
                            }
                            // ((v_j - v_i) . n) n
                            const float vn = -(rv0 * n0 + rv1 * n1 + rv2 * n2);
                            dvs0 = fmaf(vn, n0, dvs0);
                            dvs1 = fmaf(vn, n1, dvs1);
                            dvs2 = fmaf(vn, n2, dvs2);
                            responded = true;
                        }
                    }
                }
                if (keff > 0) topk_insert(best, keff, ((uint64_t)__float_as_uint(key) << 32) | (uint32_t)j);
            }
        }
        if (responded) {
            float n[6];
            six_normals(c, tick, (uint32_t)d, TAG_COLL, 0, n);
            s.v[0] = c.alpha_c * (s.v[0] + dvs0 + c.sig_cv * n[0]);
            s.v[1] = c.alpha_c * (s.v[1] + dvs1 + c.sig_cv * n[1]);
            s.v[2] = c.alpha_c * (s.v[2] + dvs2 + c.sig_cv * n[2]);
            comp_add(s.w[0], s.wlo[0], c.sig_cw * n[3]);
            comp_add(s.w[1], s.wlo[1], c.sig_cw * n[4]);
            comp_add(s.w[2], s.wlo[2], c.sig_cw * n[5]);
        }
        __syncthreads();
        if (act) {  // post-collision velocities for the neighbour observation
            sv[threadIdx.x] = s.v[0];
            sv[nt + threadIdx.x] = s.v[1];
            sv[2 * nt + threadIdx.x] = s.v[2];
        }
        __syncthreads();
    }
    if (!act) return;

    // ---- S12 observation
    if (io.obs) {
        float* o = io.obs + (size_t)d * c.obs_dim;
        float ex[3] = {0.f, 0.f, 0.f}, evv[3] = {0.f, 0.f, 0.f}, ew[3] = {0.f, 0.f, 0.f};
        if (c.flags & QS_F_OBS_NOISE) obs_noise(c, tick, d, observe_only ? 1u : 0u, ex, evv, ew);
        float2* o2 = reinterpret_cast<float2*>(o);
        o2[0] = make_float2(s.x[0] - g0 + ex[0], s.x[1] - g1 + ex[1]);
        o2[1] = make_float2(s.x[2] - g2 + ex[2], s.v[0] + evv[0]);
        o2[2] = make_float2(s.v[1] + evv[1], s.v[2] + evv[2]);
        o2[3] = make_float2(s.R[0], s.R[1]);
        o2[4] = make_float2(s.R[2], s.R[3]);
        o2[5] = make_float2(s.R[4], s.R[5]);
        o2[6] = make_float2(s.R[6], s.R[7]);
        o2[7] = make_float2(s.R[8], s.w[0] + ew[0]);
        o2[8] = make_float2(s.w[1] + ew[1], s.w[2] + ew[2]);
        for (int k = 0; k < K; ++k) {
            float2* on = o2 + 9 + 3 * k;
            if (k < keff) {
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
        for (int k = 0; k < K; ++k) dv.knn[(size_t)k * dv.D + d] = k < keff ? (int16_t)(best[k] & 0xffffu) : (int16_t)-1;
    }
    dv.ev[d] = ev;

    // ---- S13 reward and done
    if (io.rew) {
        const float dgx = s.x[0] - g0, dgy = s.x[1] - g1, dgz = s.x[2] - g2;
        float r = c.w[QS_W_POS] * sqrtf(dgx * dgx + dgy * dgy + dgz * dgz);
        r += c.w[QS_W_VEL] * sqrtf(s.v[0] * s.v[0] + s.v[1] * s.v[1] + s.v[2] * s.v[2]);
        r += c.w[QS_W_ORI] * s.R[8];
        r += c.w[QS_W_SPIN] * sqrtf(s.w[0] * s.w[0] + s.w[1] * s.w[1] + s.w[2] * s.w[2]);
        r += c.w[QS_W_ACT] * sqrtf(fh[0] * fh[0] + fh[1] * fh[1] + fh[2] * fh[2] + fh[3] * fh[3]);
        const float q0 = fh[0] - s.fp[0], q1 = fh[1] - s.fp[1], q2 = fh[2] - s.fp[2], q3 = fh[3] - s.fp[3];
        r += c.w[QS_W_DACT] * sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
        r += c.w[QS_W_ROT] * 0.5f * (s.R[0] + s.R[4] + s.R[8] - 1.0f);
        r += c.w[QS_W_YAW] * s.R[0];
        r += (ev & EV_HIT_FLOOR) ? c.w[QS_W_HIT_FLOOR] : 0.0f;
        r += (ev & EV_ON_FLOOR) ? c.w[QS_W_ON_FLOOR] : 0.0f;
        r += (ev & EV_HIT_WALL) ? c.w[QS_W_HIT_WALL] : 0.0f;
        r += (ev & EV_HIT_CEIL) ? c.w[QS_W_HIT_CEIL] : 0.0f;
        r += (ev & EV_HIT_QUAD) ? c.w[QS_W_HIT_QUAD] : 0.0f;
        if (W > 1 && c.w[QS_W_NEAR] != 0.0f) {
            float near = 0.0f;
            for (int k = 0; k < keff; ++k) {
                const float key = __uint_as_float((uint32_t)(best[k] >> 32));
                near += fmaxf(1.0f - sqrtf(key) / p.prox, 0.0f);
            }
            r += c.w[QS_W_NEAR] * near;
        }
        io.rew[d] = r;
    }
    s.fp[0] = fh[0];
    s.fp[1] = fh[1];
    s.fp[2] = fh[2];
    s.fp[3] = fh[3];

    const int ep = ep0 + 1;
    const bool done = ep >= c.episode_steps;
    if (lane == 0) {
        if (io.done) io.done[e] = done ? 1 : 0;
        dv.ep[e] = (done && (c.flags & QS_F_AUTO_RESET)) ? 0 : ep;
        dv.tick[e] = tick + 1;
    }
    if (done && (c.flags & QS_F_AUTO_RESET)) {
        // the env starts a new episode in place (new randomisation and goal)
        float p7[QS_PARAM_DIM], goal[3];
        draw_env(c, c.key0, c.key1, tick, TAG_AUTO_ENV, e, p7, goal);
        draw_drone(c, c.key0, c.key1, tick, TAG_AUTO_DRONE, d, p7[P_T2W], s);
        if (lane == 0) {
            float full[NPRM_DEV];
            derive(c, p7, full);
            for (int k = 0; k < NPRM_DEV; ++k) dv.prm[(size_t)k * dv.E + e] = full[k];
            dv.goal[e] = goal[0];
            dv.goal[dv.E + e] = goal[1];
            dv.goal[2 * dv.E + e] = goal[2];
        }
    }
    if (!finite_state(s)) atomicOr(dv.status, 1);
    store_drone(s, dv.st, dv.D, d);
}

cudaError_t launch_step(const Consts& c, const Dev& dv, const ClassPlan& cp, const Tile* tiles, const int* perm,
                        const StepIO& io, int observe_only, cudaStream_t st) {
    if (cp.n_tiles == 0) return cudaSuccess;
    const size_t smem = (cp.W > 1) ? sizeof(float) * 6 * cp.block : 0;
    const Tile* t = tiles + cp.tile_off;
    switch (cp.W) {
        case 1: k_step<1><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 2: k_step<2><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 4: k_step<4><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 8: k_step<8><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 16: k_step<16><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 32: k_step<32><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        case 64: k_step<64><<<cp.n_tiles, cp.block, smem, st>>>(c, dv, t, perm, io, observe_only); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- reset
__global__ void k_reset_env(const Consts c, const Dev dv, uint32_t k0, uint32_t k1, const uint8_t* __restrict__ mask) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= dv.E) return;
    if (mask && !mask[e]) return;
    const uint32_t tick = mask ? dv.tick[e] : 0u;
    float p7[QS_PARAM_DIM], goal[3], full[NPRM_DEV];
    draw_env(c, k0, k1, tick, TAG_RESET_ENV, e, p7, goal);
    derive(c, p7, full);
    for (int k = 0; k < NPRM_DEV; ++k) dv.prm[(size_t)k * dv.E + e] = full[k];
    dv.goal[e] = goal[0];
    dv.goal[dv.E + e] = goal[1];
    dv.goal[2 * dv.E + e] = goal[2];
    dv.ep[e] = 0;
    if (!mask) dv.tick[e] = 0;
}

__global__ void k_reset_drone(const Consts c, const Dev dv, uint32_t k0, uint32_t k1, const uint8_t* __restrict__ mask) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= dv.D) return;
    const int e = dv.env_of[d];
    if (mask && !mask[e]) return;
    const uint32_t tick = dv.tick[e];  // 0 after a full reset (set by k_reset_env)
    Drone s;
    draw_drone(c, k0, k1, tick, TAG_RESET_DRONE, d, dv.prm[(size_t)P_T2W * dv.E + e], s);
    store_drone(s, dv.st, dv.D, d);
    dv.ev[d] = 0;
}

cudaError_t launch_reset(const Consts& c, const Dev& dv, uint32_t k0, uint32_t k1, const uint8_t* mask, cudaStream_t st) {
    k_reset_env<<<(dv.E + 127) / 128, 128, 0, st>>>(c, dv, k0, k1, mask);
    k_reset_drone<<<(dv.D + 127) / 128, 128, 0, st>>>(c, dv, k0, k1, mask);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- state access
__global__ void k_get_drones(const Dev dv, float* __restrict__ out) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= dv.D) return;
    float4 q[NPLANE];
    for (int p = 0; p < NPLANE; ++p) q[p] = dv.st[(size_t)p * dv.D + d];
    const float* f = reinterpret_cast<const float*>(q);
    for (int k = 0; k < QS_STATE_DIM; ++k) out[(size_t)d * QS_STATE_DIM + k] = f[k];
}

__global__ void k_get_envs(const Dev dv, float* params, float* goals, int32_t* ep, uint32_t* tick) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= dv.E) return;
    if (params)
        for (int k = 0; k < QS_PARAM_DIM; ++k) params[(size_t)e * QS_PARAM_DIM + k] = dv.prm[(size_t)k * dv.E + e];
    if (goals)
        for (int k = 0; k < 3; ++k) goals[(size_t)e * 3 + k] = dv.goal[(size_t)k * dv.E + e];
    if (ep) ep[e] = dv.ep[e];
    if (tick) tick[e] = dv.tick[e];
}

cudaError_t launch_get_state(const Dev& dv, float* state, float* params, float* goals, int32_t* ep, uint32_t* tick,
                             cudaStream_t st) {
    if (state) k_get_drones<<<(dv.D + 127) / 128, 128, 0, st>>>(dv, state);
    if (params || goals || ep || tick) k_get_envs<<<(dv.E + 127) / 128, 128, 0, st>>>(dv, params, goals, ep, tick);
    return cudaGetLastError();
}

__global__ void k_set_drones(const Dev dv, const float* __restrict__ in) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= dv.D) return;
    float4 q[NPLANE];
    float* f = reinterpret_cast<float*>(q);
    for (int k = 0; k < QS_STATE_DIM; ++k) f[k] = in[(size_t)d * QS_STATE_DIM + k];
    for (int k = QS_STATE_DIM; k < 4 * NPLANE; ++k) f[k] = 0.f;  // pads and body-rate low parts
    for (int p = 0; p < NPLANE; ++p) dv.st[(size_t)p * dv.D + d] = q[p];
}

__global__ void k_set_envs(const Consts c, const Dev dv, const float* params, const float* goals, const int32_t* ep,
                           const uint32_t* tick) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= dv.E) return;
    if (params) {
        float p7[QS_PARAM_DIM], full[NPRM_DEV];
        for (int k = 0; k < QS_PARAM_DIM; ++k) p7[k] = params[(size_t)e * QS_PARAM_DIM + k];
        derive(c, p7, full);
        for (int k = 0; k < NPRM_DEV; ++k) dv.prm[(size_t)k * dv.E + e] = full[k];
    }
    if (goals)
        for (int k = 0; k < 3; ++k) dv.goal[(size_t)k * dv.E + e] = goals[(size_t)e * 3 + k];
    if (ep) dv.ep[e] = ep[e];
    if (tick) dv.tick[e] = tick[e];
}

cudaError_t launch_set_state(const Consts& c, const Dev& dv, const float* state, const float* params, const float* goals,
                             const int32_t* ep, const uint32_t* tick, cudaStream_t st) {
    if (state) k_set_drones<<<(dv.D + 127) / 128, 128, 0, st>>>(dv, state);
    if (params || goals || ep || tick) k_set_envs<<<(dv.E + 127) / 128, 128, 0, st>>>(c, dv, params, goals, ep, tick);
    return cudaGetLastError();
}

__global__ void k_get_events(const Dev dv, int K, uint32_t* events, int16_t* knn) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= dv.D) return;
    if (events) events[d] = dv.ev[d];
    if (knn)
        for (int k = 0; k < K; ++k) knn[(size_t)d * K + k] = dv.knn ? dv.knn[(size_t)k * dv.D + d] : (int16_t)-1;
}

cudaError_t launch_get_events(const Dev& dv, int K, uint32_t* events, int16_t* knn, cudaStream_t st) {
    k_get_events<<<(dv.D + 127) / 128, 128, 0, st>>>(dv, K, events, knn);
    return cudaGetLastError();
}

}  // namespace qsk
