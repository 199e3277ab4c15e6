// qs_kernels.cu -- sm_103a kernels around the step: episode reset with domain
// randomisation (S0) and state / event access.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qs_device.cuh"
#include "qs_internal.h"
#include "qs_scenario.cuh"

namespace qsk {

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
    float rec[QS_NSCN];
    draw_scenario(c, k0, k1, tick, TAG_SCN, e, rec);
    store_scenario(dv, 0, e, rec);
    dv.scn_sel[e] = 0;
    dv.ep[e] = 0;
    if (!mask) dv.tick[e] = 0;
}

__global__ void k_reset_drone(const Consts c, const Dev dv, uint32_t k0, uint32_t k1, const uint8_t* __restrict__ mask) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= dv.D) return;
    const int e = dv.env_of[d];
    if (!qs_check(dv.status, e >= 0 && e < dv.E)) return;
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

// ---------------------------------------------------------------- scenarios
// Copies the active scenario records out to [E][QS_NSCN] (out != null) or in
// from it.
__global__ void k_scenario_io(const Dev dv, float* __restrict__ out, const float* __restrict__ in) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= dv.E) return;
    if (!qs_check(dv.status, dv.scn_sel[e] == 0 || dv.scn_sel[e] == 1)) return;
    float* base = dv.scn + (size_t)dv.scn_sel[e] * QS_NSCN * dv.E + e;
    for (int k = 0; k < QS_NSCN; ++k) {
        if (out)
            out[(size_t)e * QS_NSCN + k] = base[(size_t)k * dv.E];
        else
            base[(size_t)k * dv.E] = in[(size_t)e * QS_NSCN + k];
    }
}

cudaError_t launch_scenario_io(const Dev& dv, float* out, const float* in, cudaStream_t st) {
    k_scenario_io<<<(dv.E + 127) / 128, 128, 0, st>>>(dv, out, in);
    return cudaGetLastError();
}

// Goal [3] of every drone at its env's current control step; a swap slot is
// the rank of the drone's key among its env's keys (recomputed per drone:
// this kernel serves inspection, not the step).
__global__ void k_goals(const Consts c, const Dev dv, float* __restrict__ goals) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= dv.D) return;
    const int e = dv.env_of[d];
    if (!qs_check(dv.status, e >= 0 && e < dv.E)) return;
    const int d0 = dv.env_off[e], N = dv.env_off[e + 1] - d0, i = d - d0;
    if (!qs_check(dv.status, i >= 0 && i < N)) return;
    const int tau = dv.ep[e], sel = dv.scn_sel[e];
    const float genv[3] = {dv.goal[e], dv.goal[dv.E + e], dv.goal[2 * dv.E + e]};
    float g[3] = {genv[0], genv[1], genv[2]};
    if (c.scn_mask & ~1u) {
        int slot = i;
        if (swap_active(dv, sel, e, tau)) {
            const uint32_t seed = scn_seed(dv, sel, e), ki = swap_key(c, seed, i);
            slot = 0;
            for (int j = 0; j < N; ++j) {
                const uint32_t kj = swap_key(c, seed, j);
                slot += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
            }
        }
        scenario_goal(c, dv, sel, e, i, N, tau, slot, genv, g);
    }
    goals[(size_t)d * 3 + 0] = g[0];
    goals[(size_t)d * 3 + 1] = g[1];
    goals[(size_t)d * 3 + 2] = g[2];
}

cudaError_t launch_goals(const Consts& c, const Dev& dv, float* goals, cudaStream_t st) {
    k_goals<<<(dv.D + 127) / 128, 128, 0, st>>>(c, dv, goals);
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

// ---------------------------------------------------------------- Philox check
// out[i] = Philox4x32-10(ctr[i][0..2], 0; key) through the same device
// functions the step and the resets draw with: the precomputed round keys
// (variant 0) or the inline key schedule (variant 1).
struct RoundKeys {
    uint32_t rk[20];
};

__global__ void k_philox(const uint32_t* __restrict__ ctr, RoundKeys rk, uint32_t key0, uint32_t key1, int variant,
                         uint4* __restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t c0 = ctr[3 * i], c1 = ctr[3 * i + 1], c2 = ctr[3 * i + 2];
        out[i] = variant == 0 ? philox_rk(c0, c1, c2, rk.rk) : philox(c0, c1, c2, key0, key1);
    }
}

#ifdef QS_DEBUG_CHECKS
// One index check (debug build): the event word of drone `index` is read and
// written back only when the check passes.
__global__ void k_check_selftest(const Dev dv, int index) {
    if (qs_check(dv.status, index >= 0 && index < dv.D)) dv.ev[index] = dv.ev[index];
}
#endif

cudaError_t launch_check_selftest(const Dev& dv, int index, cudaStream_t st) {
#ifdef QS_DEBUG_CHECKS
    k_check_selftest<<<1, 1, 0, st>>>(dv, index);
    return cudaGetLastError();
#else
    (void)dv;
    (void)index;
    (void)st;
    return cudaErrorNotSupported;  // the release build has no checks: never launched
#endif
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t key0, uint32_t key1, int variant, uint32_t* out, long long n,
                          cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    Consts c{};
    c.key0 = key0;
    c.key1 = key1;
    set_round_keys(c);
    RoundKeys rk;
    for (int k = 0; k < 20; ++k) rk.rk[k] = c.rk[k];
    const long long want = (n + 255) / 256;
    const int grid = (int)(want < 4096 ? want : 4096);
    k_philox<<<grid, 256, 0, st>>>(ctr, rk, key0, key1, variant, reinterpret_cast<uint4*>(out), n);
    return cudaGetLastError();
}

}  // namespace qsk
