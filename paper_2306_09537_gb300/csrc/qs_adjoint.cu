// qs_adjoint.cu -- the differentiable rollout: a forward pass in the smooth-
// contact form that stores checkpoints, and the hand-written adjoint (reverse
// mode) of the whole step, recomputing each checkpoint segment's substeps.
//
// Loss of a rollout of T control steps from x0 under commands a_t:
//   L_d = sum_t |x_d(t) - g_e|^2 + 1e-3 |f^_d(t)|^2   (per drone d; x after step t)
// The smooth form replaces the floor, wall, ceiling and pair responses by
// softplus penalty accelerations k_c sp_beta(penetration) / m along the
// contact normal (sp_beta(u) = log(1 + exp(beta u)) / beta); motor noise is a
// fixed additive draw (its Philox counters do not depend on the state).
//
// Adjoint of one substep (state s -> s'; all quantities of drone i):
//   uf' = uf + alpha (u - uf),  eps' = a_nd eps + a_ns n,  f_r = fmax uf'_r^2 + eps'_r
//   T = sum f, tau = (sa(f0+f1-f2-f3), sa(f1+f2-f0-f3), kappa(f1+f3-f0-f2))
//   a = T R e_z / m + g + wall(x) + sum_j psi(d_ij) (x_i - x_j),  psi(d) = k sp(2l - d) / d
//   wdot = I^-1 (tau - w x I w),  v' = v + a dt,  x' = x + v' dt,  w' = clamp(w + wdot dt)
//   R' = B(R Q(w')),  Q = I + a(w) [w]x + b(w) [w]x^2 (the polar factor of I + dt [w]x),
//   B(M) = M (3 I - M^T M) / 2 (one Bjorck step).
// The reverse pass applies the transposed Jacobian of each line in reverse
// order; the pair term couples drone i to its partners through
// lambda_x_i += sum_j J_ij (lambda_a_i - lambda_a_j), J_ij = psi I + (psi'/d) r r^T,
// with lambda_a exchanged through shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace qsk {

constexpr int ADJ_BLOCK_MAX = 256;
constexpr int NSUB = 29;
// steps of a checkpoint segment whose collision responses the backward records
constexpr int RFLAG_WORDS = 32, RFLAG_BITS = 32 * RFLAG_WORDS;  // floats of a saved substep input: x v R w wlo uf eps

// Logistic function 1 / (1 + exp(-z)) from e = exp(-|z|) in (0, 1]: the
// reciprocal of 1 + e in [1, 2] never meets an infinite or denormal operand
// (1 + exp(-z) overflows for a drone far from a wall, z ~ -1000).
__device__ __forceinline__ float sigmoidf_(float z) {
    const float e = exp_approx(-fabsf(z));
    const float s = rcp_approx(1.0f + e);
    return z >= 0.0f ? s : e * s;
}

// Diagonal derivative of the wall / floor / ceiling penalty acceleration
// (the acceleration itself is the substep's).
__device__ __forceinline__ void wall_dacc(const Consts& c, const float x[3], float dacc[3]) {
    const float kcg = c.kc * c.g, b = c.beta;
    dacc[0] = -kcg * (sigmoidf_(b * (-c.room_hx - x[0])) + sigmoidf_(b * (x[0] - c.room_hx)));
    dacc[1] = -kcg * (sigmoidf_(b * (-c.room_hy - x[1])) + sigmoidf_(b * (x[1] - c.room_hy)));
    dacc[2] = -kcg * (sigmoidf_(-b * x[2]) + sigmoidf_(b * (x[2] - c.room_h)));
}

// lambda_x += sum_j J_ij (lam_a_i - lam_a_j)
__device__ __forceinline__ void pair_vjp(const Consts& c, const float x[3], const float la[3], const float* sx,
                                         const float* sla, int nt, int sbase, int lane, int N, float arm, float lx[3]) {
    const float kcg = c.kc * c.g, b = c.beta, far2 = pair_far_d2(arm, c.inv_beta);
    for (int j = 0; j < N; ++j) {
        if (j == lane) continue;
        const int tj = sbase + j;
        const float r0 = x[0] - sx[tj], r1 = x[1] - sx[nt + tj], r2 = x[2] - sx[2 * nt + tj];
        const float d2 = r0 * r0 + r1 * r1 + r2 * r2;
        if (d2 == 0.f || d2 > far2) continue;
        const float d = sqrtf(d2), id = rcp_approx(d);
        const float pen = 2.f * arm - d;
        const float sp = softplus_b(pen, b, c.inv_beta), sg = sigmoidf_(b * pen);
        const float psi = kcg * sp * id;
        const float dpsi = kcg * (-sg * id - sp * id * id);  // d psi / d d
        const float q0 = la[0] - sla[tj], q1 = la[1] - sla[nt + tj], q2 = la[2] - sla[2 * nt + tj];
        const float rq = (r0 * q0 + r1 * q1 + r2 * q2) * dpsi * id;
        lx[0] += psi * q0 + rq * r0;
        lx[1] += psi * q1 + rq * r1;
        lx[2] += psi * q2 + rq * r2;
    }
}

// Adjoint of R' = B(R Q(w1)) (Q the polar factor of I + dt [w1]x, B one
// Bjorck step): lR holds lambda of R' on entry and lambda of R on return;
// lw1 receives lambda of w1 (added to its entry value). The products are
// written out with the identities of a skew matrix W = [w]x:
// W^2 = w w^T - |w|^2 I, <G, W> = w . vex(G), <G, W^2> = w^T G w - |w|^2 tr G,
// vex(-(G W + W G)) = (G + G^T) w - 2 tr(G) w, with
// vex(X) = (X21 - X12, X02 - X20, X10 - X01); and for the Bjorck step
// M L^T M + M M^T L = M (X + X^T), X = L^T M.
__device__ __forceinline__ void rotation_vjp(const float R[9], const float w1[3], float dt, float lR[9], float lw1[3]) {
    const float w0 = w1[0], wy = w1[1], w2 = w1[2];
    const float n2 = w0 * w0 + wy * wy + w2 * w2;
    const float cc = rsqrt_approx_ge1(fmaf(dt * dt, n2, 1.0f));
    const float inv1c = rcp_approx(1.0f + cc);  // 1 + c in (1, 2]: one reciprocal for both quotients below
    const float qa = dt * cc;
    const float qb = dt * dt * cc * cc * inv1c;
    // Q = I + qa W + qb W^2
    const float p01 = w0 * wy, p02 = w0 * w2, p12 = wy * w2;
    const float Q[9] = {1.f + qb * (w0 * w0 - n2), qb * p01 - qa * w2,         qb * p02 + qa * wy,
                        qb * p01 + qa * w2,         1.f + qb * (wy * wy - n2), qb * p12 - qa * w0,
                        qb * p02 - qa * wy,         qb * p12 + qa * w0,         1.f + qb * (w2 * w2 - n2)};
    // M = R Q
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i] * Q[j] + R[3 * i + 1] * Q[3 + j] + R[3 * i + 2] * Q[6 + j];

    // ---- reverse
    // R' = B(M) = M (1.5 I - 0.5 S), S = M^T M:
    // G_M = 1.5 L - 0.5 (L S + M (X + X^T)), X = L^T M
    float S[9], Y[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            S[3 * i + j] = M[i] * M[j] + M[3 + i] * M[3 + j] + M[6 + i] * M[6 + j];
            S[3 * j + i] = S[3 * i + j];
        }
    float X[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) X[3 * i + j] = lR[i] * M[j] + lR[3 + i] * M[3 + j] + lR[6 + i] * M[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            Y[3 * i + j] = X[3 * i + j] + X[3 * j + i];
            Y[3 * j + i] = Y[3 * i + j];
        }
    float GM[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) t += lR[3 * i + k] * S[3 * k + j] + M[3 * i + k] * Y[3 * k + j];
            GM[3 * i + j] = 1.5f * lR[3 * i + j] - 0.5f * t;
        }
    // M = R Q: lambda_R = G_M Q^T, G_Q = R^T G_M
    float GQ[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            lR[3 * i + j] = GM[3 * i] * Q[3 * j] + GM[3 * i + 1] * Q[3 * j + 1] + GM[3 * i + 2] * Q[3 * j + 2];
            GQ[3 * i + j] = R[i] * GM[j] + R[3 + i] * GM[3 + j] + R[6 + i] * GM[6 + j];
        }
    // Q(w1) = I + qa W + qb W^2: lambda_w1 = qa vex(G_Q) + qb vex(-(G_Q W + W G_Q))
    //   + (<G_Q, W> da/dc + <G_Q, W^2> db/dc) dc/dw
    const float vG[3] = {GQ[7] - GQ[5], GQ[2] - GQ[6], GQ[3] - GQ[1]};
    const float tr = GQ[0] + GQ[4] + GQ[8];
    const float Gw[3] = {GQ[0] * w0 + GQ[1] * wy + GQ[2] * w2, GQ[3] * w0 + GQ[4] * wy + GQ[5] * w2,
                         GQ[6] * w0 + GQ[7] * wy + GQ[8] * w2};
    const float Gtw[3] = {GQ[0] * w0 + GQ[3] * wy + GQ[6] * w2, GQ[1] * w0 + GQ[4] * wy + GQ[7] * w2,
                          GQ[2] * w0 + GQ[5] * wy + GQ[8] * w2};
    const float gA = w0 * vG[0] + wy * vG[1] + w2 * vG[2];
    const float gB = (w0 * Gw[0] + wy * Gw[1] + w2 * Gw[2]) - n2 * tr;
    // a = dt c, b = dt^2 c^2 / (1 + c), c = (1 + dt^2 |w|^2)^(-1/2):
    // dc/dw = -dt^2 c^3 w, da/dw = dt dc/dw, db/dw = dt^2 c (2 + c) / (1 + c)^2 dc/dw
    const float dcs = -dt * dt * cc * cc * cc;
    const float dadc = dt, dbdc = dt * dt * cc * (2.f + cc) * inv1c * inv1c;
    const float gc = (gA * dadc + gB * dbdc) * dcs;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        lw1[k] += qa * vG[k] + qb * ((Gw[k] + Gtw[k]) - 2.f * tr * w1[k]) + gc * w1[k];
}

// Adjoint of the substep map of the smooth form. s: substep input (as saved);
// l: in = lambda of the output state, out = lambda of the input state
// (x v R w uf eps); la: lambda of the acceleration (for the pair exchange);
// lu: accumulated lambda of the rotor-speed command u.
__device__ __forceinline__ void substep_vjp(const Drone& s, const Prm& p, const Consts& c, const float u[4],
                                            const float eps1s[4], float lx[3], float lv[3],
                                            float lR[9], float lw[3], float luf[4], float leps[4], float la[3],
                                            float lu[4]) {
    const float dt = c.dt;
    // ---- recompute the forward intermediates
    float uf1[4], eps1[4], f[4];
    for (int r = 0; r < 4; ++r) uf1[r] = fmaf(p.alag, u[r] - s.uf[r], s.uf[r]);
    // the motor noise after the update, as the forward left it (saved with the
    // next substep's input): the draw itself is additive and drops out
    for (int r = 0; r < 4; ++r) eps1[r] = eps1s[r];
    for (int r = 0; r < 4; ++r) f[r] = fmaf(p.fmax * uf1[r], uf1[r], eps1[r]);
    const float T = (f[0] + f[1]) + (f[2] + f[3]);
    const float sa = p.arm * 0.70710678118654752f;
    const float Iw[3] = {__fmul_rn(p.ixx, s.w[0]), __fmul_rn(p.iyy, s.w[1]), __fmul_rn(p.izz, s.w[2])};
    const float tx = sa * ((f[0] + f[1]) - (f[2] + f[3]));
    const float ty = sa * ((f[1] + f[2]) - (f[0] + f[3]));
    const float tz = c.kappa * ((f[1] + f[3]) - (f[0] + f[2]));
    const float wd[3] = {__fmul_rn(__fsub_rn(tx, cross_c(s.w[1], Iw[2], s.w[2], Iw[1])), p.inv_ixx),
                         __fmul_rn(__fsub_rn(ty, cross_c(s.w[2], Iw[0], s.w[0], Iw[2])), p.inv_iyy),
                         __fmul_rn(__fsub_rn(tz, cross_c(s.w[0], Iw[1], s.w[1], Iw[0])), p.inv_izz)};
    // w' exactly as the forward computed it (compensated), and the clamp mask
    float w1[3], pass[3];
    for (int k = 0; k < 3; ++k) {
        float hi = s.w[k], lo = s.wlo[k];
        comp_add_prod(hi, lo, wd[k], dt);
        pass[k] = fabsf(hi) > c.omega_max ? 0.f : 1.f;
        w1[k] = fabsf(hi) > c.omega_max ? copysignf(c.omega_max, hi) : hi;
    }
    // R' = B(R Q(w1))
    float lw1[3] = {lw[0], lw[1], lw[2]};
    float lRin[9];
    for (int k = 0; k < 9; ++k) lRin[k] = lR[k];
    rotation_vjp(s.R, w1, dt, lRin, lw1);
    // w1 = clamp(w + wdot dt)
    float lwd[3];
    for (int k = 0; k < 3; ++k) {
        const float g = lw1[k] * pass[k];
        lw[k] = g;
        lwd[k] = g * dt;
    }
    // x' = x + v' dt ; v' = v + a dt
    float lv1[3];
    for (int k = 0; k < 3; ++k) lv1[k] = lv[k] + dt * lx[k];
    for (int k = 0; k < 3; ++k) {
        lv[k] = lv1[k];
        la[k] = dt * lv1[k];
    }
    // wdot = I^-1 (tau - w x I w): lambda_tau = mu, lambda_w -= (I w) x mu + I (mu x w)
    const float mu[3] = {lwd[0] * p.inv_ixx, lwd[1] * p.inv_iyy, lwd[2] * p.inv_izz};
    const float c1[3] = {Iw[1] * mu[2] - Iw[2] * mu[1], Iw[2] * mu[0] - Iw[0] * mu[2], Iw[0] * mu[1] - Iw[1] * mu[0]};
    const float c2[3] = {mu[1] * s.w[2] - mu[2] * s.w[1], mu[2] * s.w[0] - mu[0] * s.w[2], mu[0] * s.w[1] - mu[1] * s.w[0]};
    lw[0] -= c1[0] + p.ixx * c2[0];
    lw[1] -= c1[1] + p.iyy * c2[1];
    lw[2] -= c1[2] + p.izz * c2[2];
    // a = T R e_z / m + g + wall(x) + pair: walls on the diagonal, thrust
    float dwall[3];
    wall_dacc(c, s.x, dwall);
    for (int k = 0; k < 3; ++k) lx[k] += dwall[k] * la[k];
    const float b3[3] = {s.R[2], s.R[5], s.R[8]};
    const float lT = (la[0] * b3[0] + la[1] * b3[1] + la[2] * b3[2]) * p.inv_m;
    lRin[2] += T * la[0] * p.inv_m;
    lRin[5] += T * la[1] * p.inv_m;
    lRin[8] += T * la[2] * p.inv_m;
    for (int k = 0; k < 9; ++k) lR[k] = lRin[k];
    // T, tau from f
    const float gx = mu[0] * sa, gy = mu[1] * sa, gz = mu[2] * c.kappa;
    const float lf[4] = {lT + gx - gy - gz, lT + gx + gy + gz, lT - gx + gy - gz, lT - gx - gy + gz};
    // f = fmax uf1^2 + eps1; eps1 = a_nd eps + a_ns n; uf1 = uf + alpha (u - uf)
    for (int r = 0; r < 4; ++r) {
        const float luf1 = luf[r] + 2.f * p.fmax * uf1[r] * lf[r];
        const float leps1 = leps[r] + lf[r];
        leps[r] = (c.flags & QS_F_MOTOR_NOISE) ? c.alpha_nd * leps1 : leps1;
        luf[r] = (1.f - p.alag) * luf1;
        lu[r] += p.alag * luf1;
    }
}

// ---------------------------------------------------------------- workspace
// [n_ckpt][NPLANE][D] float4 checkpoints, then [C * (substeps + 1)][NSUB][D]
// floats (each substep's input and, for the discrete form, each step's
// pre-collision state).
size_t diff_workspace_bytes(int D, int T, int C, int substeps) {
    const int nck = (T + C - 1) / C;
    const size_t ck = (size_t)nck * NPLANE * D * sizeof(float4);
    // two scratch buffers: the backward pass recomputes one segment while it reverses the next
    const size_t sc = 2 * (size_t)C * (substeps + 1) * NSUB * D * sizeof(float);
    return ck + sc + 256;
}

__device__ __forceinline__ void save_sub(float* sc, size_t D, int idx, int d, const Drone& s) {
    float* b = sc + (size_t)idx * NSUB * D + d;
    int k = 0;
    for (int q = 0; q < 3; ++q) b[(k++) * D] = s.x[q];
    for (int q = 0; q < 3; ++q) b[(k++) * D] = s.v[q];
    for (int q = 0; q < 9; ++q) b[(k++) * D] = s.R[q];
    for (int q = 0; q < 3; ++q) b[(k++) * D] = s.w[q];
    for (int q = 0; q < 3; ++q) b[(k++) * D] = s.wlo[q];
    for (int q = 0; q < 4; ++q) b[(k++) * D] = s.uf[q];
    for (int q = 0; q < 4; ++q) b[(k++) * D] = s.eps[q];
}

__device__ __forceinline__ void load_sub(const float* sc, size_t D, int idx, int d, Drone& s) {
    const float* b = sc + (size_t)idx * NSUB * D + d;
    int k = 0;
    for (int q = 0; q < 3; ++q) s.x[q] = b[(k++) * D];
    for (int q = 0; q < 3; ++q) s.v[q] = b[(k++) * D];
    for (int q = 0; q < 9; ++q) s.R[q] = b[(k++) * D];
    for (int q = 0; q < 3; ++q) s.w[q] = b[(k++) * D];
    for (int q = 0; q < 3; ++q) s.wlo[q] = b[(k++) * D];
    for (int q = 0; q < 4; ++q) s.uf[q] = b[(k++) * D];
    for (int q = 0; q < 4; ++q) s.eps[q] = b[(k++) * D];
}

// The motor-noise state (eps) of saved entry idx.
__device__ __forceinline__ void load_eps(const float* sc, size_t D, int idx, int d, float e[4]) {
    const float* b = sc + (size_t)idx * NSUB * D + d + (size_t)25 * D;  // x v R w wlo uf: 25 floats first
    for (int q = 0; q < 4; ++q) e[q] = b[q * D];
}

// The velocity of saved entry idx.
__device__ __forceinline__ void load_v(const float* sc, size_t D, int idx, int d, float v[3]) {
    const float* b = sc + (size_t)idx * NSUB * D + d + (size_t)3 * D;
    for (int q = 0; q < 3; ++q) v[q] = b[q * D];
}

// The position of saved entry idx.
__device__ __forceinline__ void load_x(const float* sc, size_t D, int idx, int d, float x[3]) {
    const float* b = sc + (size_t)idx * NSUB * D + d;
    for (int q = 0; q < 3; ++q) x[q] = b[q * D];
}

__device__ __forceinline__ void read_x0(Drone& s, const float* __restrict__ x0, int d) {
    const float* r = x0 + (size_t)d * QS_STATE_DIM;
    for (int k = 0; k < 3; ++k) s.x[k] = r[k];
    for (int k = 0; k < 3; ++k) s.v[k] = r[3 + k];
    for (int k = 0; k < 9; ++k) s.R[k] = r[6 + k];
    for (int k = 0; k < 3; ++k) s.w[k] = r[15 + k];
    for (int k = 0; k < 4; ++k) s.uf[k] = r[18 + k];
    for (int k = 0; k < 4; ++k) s.eps[k] = r[22 + k];
    for (int k = 0; k < 4; ++k) s.fp[k] = r[26 + k];
    s.wlo[0] = s.wlo[1] = s.wlo[2] = 0.f;
}

// Barrier of the threads that share the staged positions: the whole CTA (id
// 0), or one group of n threads of the pipelined adjoint (named barrier id; a
// group of one warp only needs its lanes converged).
__device__ __forceinline__ void group_sync(int id, int n) {
    if (id == 0)
        __syncthreads();
    else if (n == 32)
        __syncwarp();
    else if (id == 1)
        asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
    else
        asm volatile("bar.sync 2, %0;" ::"r"(n) : "memory");
}

// group_sync that also returns whether v holds for any thread of the group.
__device__ __forceinline__ bool group_sync_or(int id, int n, bool v) {
    if (id == 0) return __syncthreads_or(v) != 0;
    if (n == 32) return __any_sync(0xffffffffu, v);
    uint32_t r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
                 : "=r"(r) : "r"((uint32_t)v), "r"(id), "r"(n) : "memory");
    return r != 0;
}

// One smooth substep of the slot's drones (pair force from the positions at
// the substep start, staged in shared memory at the thread's group-local
// index lt; bid, bn: the barrier of the threads sharing them).
__device__ __forceinline__ void smooth_substep(const Consts& c, Drone& s, const Prm& p, const float u[4], uint32_t tick,
                                               int d, int sub, bool act, float* sx, int nt, int sbase, int lane, int N,
                                               int lt, int bid, int bn, const float* nrm = nullptr) {
    if (act) {
        sx[lt] = s.x[0];
        sx[nt + lt] = s.x[1];
        sx[2 * nt + lt] = s.x[2];
    }
    group_sync(bid, bn);
    float pa[3] = {0.f, 0.f, 0.f};
    if (act) pair_acc(c, s.x, sx, nt, sbase, lane, N, p.arm, pa);
    group_sync(bid, bn);
    if (act) substep<false, 1>(s, p, c, u, tick, d, sub, pa, nrm);
}

// The forward kernels run two groups of nb threads over the same drones: group
// 0 integrates, group 1 draws the motor-noise normals of the next control
// step (up to FWD_SUB substeps) into shared memory, double-buffered by step
// parity, so that the Philox and Box-Muller work is off the integration chain.
constexpr int FWD_SUB = 4;

__device__ __forceinline__ float* fwd_normals(float* base, int nb, int b, int sub, int r, int lt) {
    return base + ((b * FWD_SUB + sub) * 4 + r) * nb + lt;
}

// Group 1 of a forward kernel: step t's normals are ready at the t-th CTA
// barrier of the loop; the next step's are drawn while group 0 integrates.
__device__ __forceinline__ void fwd_noise_group(const Consts& c, float* nbase, int nb, int lt, bool act, bool ahead,
                                                uint32_t tick0, int d, int T) {
    const int S = c.substeps;
    auto draw = [&](int t) {
        for (int sub = 0; sub < S; ++sub) {
            float n[4];
            motor_normals(c, tick0 + (uint32_t)t, d, sub, n);
            for (int r = 0; r < 4; ++r) *fwd_normals(nbase, nb, t & 1, sub, r, lt) = n[r];
        }
    };
    if (ahead && act && T > 0) draw(0);
    for (int t = 0; t < T; ++t) {
        __syncthreads();  // buffer t & 1 holds step t's normals; buffer (t + 1) & 1 is free
        if (ahead && act && t + 1 < T) draw(t + 1);
    }
}

struct DiffArgs {
    const float* x0;       // [D][30]
    const float* act;      // [T][D][4]
    float* loss;           // [D]
    const float* dloss;    // [D]
    float* grad_act;       // [T][D][4]
    float* grad_x0;        // [D][30]
    float4* ckpt;          // [nck][NPLANE][D]
    float* scratch;        // [C * substeps][NSUB][D]
    int T, C;
};

__device__ __forceinline__ void command4(const Consts& c, const float* act, size_t D, int t, int d, float fh[4], float u[4],
                                         float msk[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(act + (size_t)t * D * 4) + d);
    const float av[4] = {a.x, a.y, a.z, a.w};
    for (int r = 0; r < 4; ++r) {
        fh[r] = command(c, av[r]);
        u[r] = sqrt_approx(fh[r]);  // as the step computes it
        // d f^ / d a: 1 inside the clip range (1/2 for the symmetric map), 0 outside
        const bool in = (c.flags & QS_F_ACTION_SYMMETRIC) ? (av[r] > -1.f && av[r] < 1.f) : (av[r] > 0.f && av[r] < 1.f);
        msk[r] = in ? ((c.flags & QS_F_ACTION_SYMMETRIC) ? 0.5f : 1.f) : 0.f;
    }
}

__global__ void __launch_bounds__(ADJ_BLOCK_MAX) k_diff_fwd(const Consts c, const Dev dv, const Tile* __restrict__ tiles,
                                                            const int* __restrict__ perm, const DiffArgs a) {
    extern __shared__ float sm[];
    const int nb = blockDim.x >> 1, grp = threadIdx.x >= nb ? 1 : 0, lt = threadIdx.x - grp * nb;
    const Tile tile = tile_at(dv, tiles, blockIdx.x, nb);
    const int W = tile.W, nt = nb;
    const int slot = lt / W, lane = lt - slot * W;
    const SlotGeo geo = slot_geometry(dv, perm, tile, slot, W, nt);
    const int e = geo.e, d0 = geo.d0, N = geo.N;
    const bool act = lane < N;
    const int d = d0 + lane, sbase = slot * W;
    const size_t D = dv.D;
    const bool ahead = (c.flags & QS_F_MOTOR_NOISE) && c.substeps <= FWD_SUB;
    float* nbase = sm + 9 * nb;  // [2][FWD_SUB][4][nb] motor normals
    const uint32_t tick0 = act ? dv.tick[e] : 0u;
    if (grp == 1) {
        fwd_noise_group(c, nbase, nb, lt, act, ahead, tick0, d, a.T);
        return;
    }
    Drone s;
    Prm p;
    float g[3] = {0.f, 0.f, 0.f};
    if (act) {
        read_x0(s, a.x0, d);
        p = load_prm(c, dv.prm, dv.E, e);
        g[0] = dv.goal[e];
        g[1] = dv.goal[dv.E + e];
        g[2] = dv.goal[2 * dv.E + e];
    }
    float L = 0.f;
    for (int t = 0; t < a.T; ++t) {
        __syncthreads();  // step t's motor normals ready (group 1)
        if (act && t % a.C == 0) {
            float4 q[NPLANE];
            pack(s, q);
            float4* ck = a.ckpt + (size_t)(t / a.C) * NPLANE * D;
            for (int pl = 0; pl < NPLANE; ++pl) ck[(size_t)pl * D + d] = q[pl];
        }
        float fh[4] = {0.f, 0.f, 0.f, 0.f}, u[4] = {0.f, 0.f, 0.f, 0.f}, msk[4];
        if (act) command4(c, a.act, D, t, d, fh, u, msk);
        for (int sub = 0; sub < c.substeps; ++sub) {
            float n[4];
            if (ahead)
                for (int r = 0; r < 4; ++r) n[r] = *fwd_normals(nbase, nb, t & 1, sub, r, lt);
            smooth_substep(c, s, p, u, tick0 + t, d, sub, act, sm, nt, sbase, lane, N, lt, 1, nb, ahead ? n : nullptr);
        }
        if (act) {
            const float dx = s.x[0] - g[0], dy = s.x[1] - g[1], dz = s.x[2] - g[2];
            L += dx * dx + dy * dy + dz * dz + 1e-3f * (fh[0] * fh[0] + fh[1] * fh[1] + fh[2] * fh[2] + fh[3] * fh[3]);
        }
    }
    if (act) {
        a.loss[d] = L;
        if (!finite_state(s)) atomicOr(dv.status, 1);
    }
}

// Adjoint of the smooth rollout, pipelined over checkpoint segments. The CTA
// holds two groups of nb threads over the same drones: while group 1 runs the
// reverse of segment s from its saved substep inputs, group 0 recomputes
// segment s - 1 from its checkpoint into the other scratch buffer and leaves
// the segment's final position and motor noise in shared memory; one CTA
// barrier per segment hands a buffer from group 0 to group 1. Each group
// synchronises its staged positions with its own barrier. The reverse takes
// each substep's updated motor noise (and each step's end position) from the
// next saved input instead of drawing it again.
__global__ void __launch_bounds__(ADJ_BLOCK_MAX) k_diff_bwd(const Consts c, const Dev dv, const Tile* __restrict__ tiles,
                                                            const int* __restrict__ perm, const DiffArgs a) {
    extern __shared__ float sm[];
    const int nb = blockDim.x >> 1, grp = threadIdx.x >= nb ? 1 : 0, lt = threadIdx.x - grp * nb, bid = 1 + grp;
    const Tile tile = tile_at(dv, tiles, blockIdx.x, nb);
    const int W = tile.W, nt = nb;
    const int slot = lt / W, lane = lt - slot * W;
    const SlotGeo geo = slot_geometry(dv, perm, tile, slot, W, nt);
    const int e = geo.e, d0 = geo.d0, N = geo.N;
    const bool act = lane < N;
    const int d = d0 + lane, sbase = slot * W;
    const size_t D = dv.D;
    float* sx = sm + grp * 3 * nb;  // [3][nb] positions of the group
    float* sla = sm + 6 * nb;       // [3][nb] lambda of the acceleration (group 1)
    float* fin = sm + 9 * nb;       // [2][7][nb] position and motor noise at the end of a recomputed segment
    const int S = c.substeps;
    const size_t sbuf = (size_t)a.C * (S + 1) * NSUB * D;  // floats of one scratch buffer (each substep's input)
    Prm p;
    float g[3] = {0.f, 0.f, 0.f};
    uint32_t tick0 = 0;
    float dl = 0.f;
    if (act) {
        p = load_prm(c, dv.prm, dv.E, e);
        g[0] = dv.goal[e];
        g[1] = dv.goal[dv.E + e];
        g[2] = dv.goal[2 * dv.E + e];
        tick0 = dv.tick[e];
        dl = a.dloss[d];
    }
    float lx[3] = {0.f, 0.f, 0.f}, lv[3] = {0.f, 0.f, 0.f}, lR[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float lw[3] = {0.f, 0.f, 0.f}, luf[4] = {0.f, 0.f, 0.f, 0.f}, leps[4] = {0.f, 0.f, 0.f, 0.f};
    const int nseg = (a.T + a.C - 1) / a.C;
    for (int it = 0; it <= nseg; ++it) {
        if (grp == 0 && it < nseg) {
            // recompute segment nseg - 1 - it, saving every substep input
            const int seg = nseg - 1 - it, tb = seg * a.C, te = min(a.T, tb + a.C);
            float* scr = a.scratch + (size_t)(it & 1) * sbuf;
            Drone s;
            if (act) {
                float4 q[NPLANE];
                const float4* ck = a.ckpt + (size_t)seg * NPLANE * D;
                for (int pl = 0; pl < NPLANE; ++pl) q[pl] = ck[(size_t)pl * D + d];
                unpack(s, q);
            }
            for (int t = tb; t < te; ++t) {
                float fh[4] = {0.f, 0.f, 0.f, 0.f}, u[4] = {0.f, 0.f, 0.f, 0.f}, msk[4];
                if (act) command4(c, a.act, D, t, d, fh, u, msk);
                for (int sub = 0; sub < S; ++sub) {
                    if (act) save_sub(scr, D, (t - tb) * S + sub, d, s);
                    smooth_substep(c, s, p, u, tick0 + t, d, sub, act, sx, nt, sbase, lane, N, lt, bid, nb);
                }
            }
            if (act) {
                float* f = fin + (it & 1) * 7 * nb;
                for (int k = 0; k < 3; ++k) f[k * nb + lt] = s.x[k];
                for (int r = 0; r < 4; ++r) f[(3 + r) * nb + lt] = s.eps[r];
            }
        } else if (grp == 1 && it >= 1) {
            // reverse through segment nseg - it, recomputed in the previous round
            const int seg = nseg - it, tb = seg * a.C, te = min(a.T, tb + a.C);
            const float* scr = a.scratch + (size_t)((it - 1) & 1) * sbuf;
            const float* f = fin + ((it - 1) & 1) * 7 * nb;
            for (int t = te - 1; t >= tb; --t) {
                float fh[4] = {0.f, 0.f, 0.f, 0.f}, u[4] = {0.f, 0.f, 0.f, 0.f}, msk[4] = {0.f, 0.f, 0.f, 0.f};
                // the state after step t: the next step's first input, or the segment's end
                float xpost[3] = {0.f, 0.f, 0.f}, eps_end[4] = {0.f, 0.f, 0.f, 0.f};
                if (act) {
                    command4(c, a.act, D, t, d, fh, u, msk);
                    if (t + 1 < te) {
                        load_x(scr, D, (t + 1 - tb) * S, d, xpost);
                        load_eps(scr, D, (t + 1 - tb) * S, d, eps_end);
                    } else {
                        for (int k = 0; k < 3; ++k) xpost[k] = f[k * nb + lt];
                        for (int r = 0; r < 4; ++r) eps_end[r] = f[(3 + r) * nb + lt];
                    }
                }
                // loss of step t: |x(t) - g|^2 + 1e-3 |f^|^2
                for (int k = 0; k < 3; ++k) lx[k] += dl * 2.f * (xpost[k] - g[k]);
                float lu[4] = {0.f, 0.f, 0.f, 0.f};
                for (int sub = S - 1; sub >= 0; --sub) {
                    Drone si;
                    float eps1[4] = {0.f, 0.f, 0.f, 0.f};
                    if (act) {
                        load_sub(scr, D, (t - tb) * S + sub, d, si);
                        if (sub + 1 < S)
                            load_eps(scr, D, (t - tb) * S + sub + 1, d, eps1);
                        else
                            for (int r = 0; r < 4; ++r) eps1[r] = eps_end[r];
                    }
                    if (act) {
                        sx[lt] = si.x[0];
                        sx[nt + lt] = si.x[1];
                        sx[2 * nt + lt] = si.x[2];
                    }
                    group_sync(bid, nb);
                    float la[3] = {0.f, 0.f, 0.f};
                    if (act) {
                        substep_vjp(si, p, c, u, eps1, lx, lv, lR, lw, luf, leps, la, lu);
                        sla[lt] = la[0];
                        sla[nt + lt] = la[1];
                        sla[2 * nt + lt] = la[2];
                    }
                    group_sync(bid, nb);
                    if (act) pair_vjp(c, si.x, la, sx, sla, nt, sbase, lane, N, p.arm, lx);
                    group_sync(bid, nb);
                }
                if (act) {
                    float ga[4];
                    for (int r = 0; r < 4; ++r) {
                        // u = sqrt(f^): du/df^ = 1 / (2u)
                        const float du = u[r] > 0.f ? 0.5f * rcp_approx(u[r]) : 0.f;
                        ga[r] = msk[r] * (lu[r] * du + dl * 2e-3f * fh[r]);
                    }
                    reinterpret_cast<float4*>(a.grad_act + (size_t)t * D * 4)[d] = make_float4(ga[0], ga[1], ga[2], ga[3]);
                }
            }
        }
        __syncthreads();  // hand over: buffer it & 1 recomputed; buffer (it - 1) & 1 free again
    }
    if (grp == 1 && act) {
        float* gx = a.grad_x0 + (size_t)d * QS_STATE_DIM;
        for (int k = 0; k < 3; ++k) gx[k] = lx[k];
        for (int k = 0; k < 3; ++k) gx[3 + k] = lv[k];
        for (int k = 0; k < 9; ++k) gx[6 + k] = lR[k];
        for (int k = 0; k < 3; ++k) gx[15 + k] = lw[k];
        for (int k = 0; k < 4; ++k) gx[18 + k] = luf[k];
        for (int k = 0; k < 4; ++k) gx[22 + k] = leps[k];
        for (int k = 0; k < 4; ++k) gx[26 + k] = 0.f;  // f^_prev does not enter the loss
    }
}

// ---------------------------------------------------------------- discrete contacts
// The differentiable rollout of the step as the simulator runs it: floor,
// wall and ceiling contacts and quadrotor collisions resolved at the substep
// or step where they are detected (Sec. III-B). The map is piecewise smooth;
// its derivative is the Jacobian of the branch each contact decision took
// (a decision's threshold is met on a set of measure zero). Contact resets
// whose outcome does not depend on the state (the floor hit zeroes the
// velocity and body rates; a wall removes the normal velocity and holds the
// drone on the boundary) pass no gradient through the reset components; the
// perturbations are additive draws and drop out.

// Adjoint of one discrete substep. s: substep input; the lambdas hold the
// output's on entry and the input's on return; lu accumulates lambda of u.
// ET: the event-time contacts (QS_F_EVENT_TIME): the floor hit moves the
// drone horizontally only up to the crossing time tau = -z0 / v1_z, a wall or
// ceiling contact moves the coordinates the boundaries do not hold with v1
// up to the first crossing tau = (L - x0_k) / v1_k and with the post-contact
// velocity v' after it; the reverse adds the terms through tau.
template <bool ET>
__device__ __forceinline__ void discrete_substep_vjp(const Drone& s, const Prm& p, const Consts& c, const float u[4],
                                                     const float eps1s[4], const float vo[3], float lx[3], float lv[3],
                                                     float lR[9], float lw[3], float luf[4], float leps[4],
                                                     float lu[4]) {
    const float dt = c.dt, g = c.g;
    // ---- the forward substep again, with its decisions (as in substep())
    float uf1[4], eps1[4], f[4];
    for (int r = 0; r < 4; ++r) uf1[r] = fmaf(p.alag, u[r] - s.uf[r], s.uf[r]);
    // the motor noise after the update, as the forward left it (saved with the
    // next substep's input or the step's pre-collision state)
    for (int r = 0; r < 4; ++r) eps1[r] = eps1s[r];
    for (int r = 0; r < 4; ++r) f[r] = fmaf(p.fmax * uf1[r], uf1[r], eps1[r]);
    const float T = (f[0] + f[1]) + (f[2] + f[3]);
    const float sa = p.arm * 0.70710678118654752f;
    const float tx = sa * ((f[0] + f[1]) - (f[2] + f[3]));
    const float ty = sa * ((f[1] + f[2]) - (f[0] + f[3]));
    const float tz = c.kappa * ((f[1] + f[3]) - (f[0] + f[2]));
    const float F0 = s.R[2] * T, F1 = s.R[5] * T, F2 = s.R[8] * T;
    float a[3] = {F0 * p.inv_m, F1 * p.inv_m, fmaf(F2, p.inv_m, -g)};
    const float mg = __fmul_rn(p.m, g);
    const bool on_floor = (c.flags & QS_F_FLOOR) && s.x[2] <= 0.0f && F2 < mg;
    const bool still = on_floor && s.v[0] == 0.0f && s.v[1] == 0.0f;
    const float ffric = on_floor ? __fmul_rn(c.mu, __fsub_rn(mg, F2)) : 0.0f;
    float nf = 0.f, keep = 0.f, vh[2] = {0.f, 0.f}, inv_nv = 0.f;
    if (on_floor) {
        float fx = F0, fy = F1;
        if (still) {
            nf = sqrtf(__fmaf_rn(fy, fy, __fmul_rn(fx, fx)));
            keep = nf > ffric ? __fmul_rn(__fsub_rn(nf, ffric), __frcp_rn(nf)) : 0.0f;
            fx = __fmul_rn(fx, keep);
            fy = __fmul_rn(fy, keep);
        } else {
            inv_nv = rsqrtf(__fmaf_rn(s.v[1], s.v[1], __fmul_rn(s.v[0], s.v[0])));
            vh[0] = s.v[0] * inv_nv;
            vh[1] = s.v[1] * inv_nv;
            fx = __fmaf_rn(-__fmul_rn(ffric, s.v[0]), inv_nv, fx);
            fy = __fmaf_rn(-__fmul_rn(ffric, s.v[1]), inv_nv, fy);
        }
        a[0] = __fmul_rn(fx, p.inv_m);
        a[1] = __fmul_rn(fy, p.inv_m);
        a[2] = 0.0f;
    }
    const float Iw[3] = {__fmul_rn(p.ixx, s.w[0]), __fmul_rn(p.iyy, s.w[1]), __fmul_rn(p.izz, s.w[2])};
    const float wd[3] = {__fmul_rn(__fsub_rn(tx, cross_c(s.w[1], Iw[2], s.w[2], Iw[1])), p.inv_ixx),
                         __fmul_rn(__fsub_rn(ty, cross_c(s.w[2], Iw[0], s.w[0], Iw[2])), p.inv_iyy),
                         __fmul_rn(__fsub_rn(tz, cross_c(s.w[0], Iw[1], s.w[1], Iw[0])), p.inv_izz)};
    float v1[3] = {fmaf(a[0], dt, s.v[0]), fmaf(a[1], dt, s.v[1]), fmaf(a[2], dt, on_floor ? 0.0f : s.v[2])};
    const bool stop = on_floor && !still && __fmaf_rn(v1[1], s.v[1], __fmul_rn(v1[0], s.v[0])) < 0.0f;
    if (stop) v1[0] = v1[1] = 0.0f;
    float x1[3] = {fmaf(v1[0], dt, s.x[0]), fmaf(v1[1], dt, s.x[1]), fmaf(v1[2], dt, s.x[2])};
    float w1[3], pass[3];
    for (int k = 0; k < 3; ++k) {
        float hi = s.w[k], lo = s.wlo[k];
        comp_add_prod(hi, lo, wd[k], dt);
        pass[k] = fabsf(hi) > c.omega_max ? 0.f : 1.f;
        w1[k] = fabsf(hi) > c.omega_max ? copysignf(c.omega_max, hi) : hi;
    }
    float R1[9];
    for (int k = 0; k < 9; ++k) R1[k] = s.R[k];
    rotate_polar(R1, w1, dt);
    const bool hit = (c.flags & QS_F_FLOOR) && x1[2] <= 0.0f && v1[2] < 0.0f;
    // event-time floor: crossing time and the velocity that led there
    float tf = dt, vz_hit = 0.f;
    bool tf_free = false;
    if (ET && hit) {
        vz_hit = v1[2];
        const float t_raw = -s.x[2] / v1[2];
        tf_free = t_raw > 0.0f && t_raw < dt;
        tf = fminf(fmaxf(t_raw, 0.0f), dt);
        x1[0] = fmaf(v1[0], tf, s.x[0]);
        x1[1] = fmaf(v1[1], tf, s.x[1]);
    }
    const float vh1[2] = {v1[0], v1[1]};  // horizontal velocity before the floor reset
    if (hit) {
        x1[2] = 0.0f;
        v1[0] = v1[1] = v1[2] = 0.0f;
    }
    bool clamp_x[3] = {false, false, false}, zero_v[3] = {false, false, false}, bump = false;
    float tw = dt;  // event-time walls: earliest crossing and the axis that set it
    int kw = -1;
    if (c.flags & QS_F_WALLS) {
        const float lim[3] = {c.room_hx, c.room_hy, c.room_h};
        for (int k = 0; k < 3; ++k) {
            float bound = 0.f;
            if (x1[k] > lim[k]) {
                clamp_x[k] = true;
                zero_v[k] = v1[k] > 0.0f;
                bound = lim[k];
            } else if (k < 2 && x1[k] < -lim[k]) {
                clamp_x[k] = true;
                zero_v[k] = v1[k] < 0.0f;
                bound = -lim[k];
            }
            if (ET && zero_v[k]) {
                const float tk = (bound - s.x[k]) / v1[k];
                if (tk < tw) {
                    tw = tk;
                    kw = k;
                }
            }
            bump |= zero_v[k];
        }
    }
    const bool tw_free = ET && bump && kw >= 0 && tw > 0.0f;
    if (ET && bump) tw = fmaxf(tw, 0.0f);
    // the post-contact velocity of the event-time walls, alpha_c (v1 + sigma_v n)
    // with the outward parts removed: the substep's output velocity (saved)
    const float* vpost = vo;

    // ---- reverse
    // event-time walls: x_j = x0_j + v1_j tau + v'_j (dt - tau) for the coordinates
    // the boundaries do not hold; lambda of tau, and v' receives (dt - tau) lambda x_j
    float ltw = 0.f, twf[3] = {dt, dt, dt};
    if (ET && bump) {
        for (int k = 0; k < 3; ++k) {
            if (clamp_x[k]) continue;
            ltw += lx[k] * (v1[k] - vpost[k]);
            lv[k] = fmaf(dt - tw, lx[k], lv[k]);
            twf[k] = tw;
        }
    }
    // walls: v <- alpha_c (v + eps) after the outward components are removed; x held on the boundary
    if (bump)
        for (int k = 0; k < 3; ++k) lv[k] *= c.alpha_c;
    for (int k = 0; k < 3; ++k) {
        if (zero_v[k]) lv[k] = 0.0f;
        if (clamp_x[k]) lx[k] = 0.0f;
    }
    // floor hit: x_z = 0, v = w = 0, R upright keeping the heading of R1's x-axis
    if (hit) {
        lx[2] = 0.0f;
        lv[0] = lv[1] = lv[2] = 0.0f;
        lw[0] = lw[1] = lw[2] = 0.0f;
        const float lcs = lR[0] + lR[4], lsn = lR[3] - lR[1];
        for (int k = 0; k < 9; ++k) lR[k] = 0.0f;
        const float h2 = R1[0] * R1[0] + R1[3] * R1[3];
        if (h2 >= 1e-12f) {  // cs = R0 / h, sn = R3 / h
            const float ih = rsqrtf(h2), ih3 = ih * ih * ih;
            lR[0] = (lcs * R1[3] * R1[3] - lsn * R1[0] * R1[3]) * ih3;
            lR[3] = (lsn * R1[0] * R1[0] - lcs * R1[0] * R1[3]) * ih3;
        } else {  // cs = R4 / h, sn = -R1 / h
            const float ih = rsqrtf(R1[1] * R1[1] + R1[4] * R1[4]), ih3 = ih * ih * ih;
            lR[1] = (-lcs * R1[1] * R1[4] - lsn * R1[4] * R1[4]) * ih3;
            lR[4] = (lcs * R1[1] * R1[1] + lsn * R1[1] * R1[4]) * ih3;
        }
    }
    // R1 = B(R Q(w1))
    float lw1[3] = {lw[0], lw[1], lw[2]};
    rotation_vjp(s.R, w1, dt, lR, lw1);
    // w1 = clamp(w + wdot dt)
    float lwd[3];
    for (int k = 0; k < 3; ++k) {
        const float gk = lw1[k] * pass[k];
        lw[k] = gk;
        lwd[k] = gk * dt;
    }
    // x1 = x + v1 dt; the stop rule; v1 = v + a dt (v_z first set to 0 on the floor)
    float lv1[3];
    for (int k = 0; k < 3; ++k) lv1[k] = lv[k] + (ET ? twf[k] : dt) * lx[k];
    if (ET && hit) {
        // event-time floor: x_xy = x0_xy + v1_xy tau, tau = -z0 / v1_z
        const float ltf = lx[0] * vh1[0] + lx[1] * vh1[1];
        lv1[0] = lv[0] + tf * lx[0];
        lv1[1] = lv[1] + tf * lx[1];
        if (tf_free) {
            lx[2] -= ltf / vz_hit;
            lv1[2] -= ltf * tf / vz_hit;
        }
    }
    if (tw_free) {  // tau = (L - x0_k) / v1_k of the axis that crossed first
        lx[kw] -= ltw / v1[kw];
        lv1[kw] -= ltw * tw / v1[kw];
    }
    if (stop) lv1[0] = lv1[1] = 0.0f;
    float la[3];
    for (int k = 0; k < 3; ++k) {
        la[k] = dt * lv1[k];
        lv[k] = lv1[k];
    }
    if (on_floor) lv[2] = 0.0f;
    // Euler: lambda_tau = mu, lambda_w -= (I w) x mu + I (mu x w)
    const float mu[3] = {lwd[0] * p.inv_ixx, lwd[1] * p.inv_iyy, lwd[2] * p.inv_izz};
    const float c1[3] = {Iw[1] * mu[2] - Iw[2] * mu[1], Iw[2] * mu[0] - Iw[0] * mu[2], Iw[0] * mu[1] - Iw[1] * mu[0]};
    const float c2[3] = {mu[1] * s.w[2] - mu[2] * s.w[1], mu[2] * s.w[0] - mu[0] * s.w[2], mu[0] * s.w[1] - mu[1] * s.w[0]};
    lw[0] -= c1[0] + p.ixx * c2[0];
    lw[1] -= c1[1] + p.iyy * c2[1];
    lw[2] -= c1[2] + p.izz * c2[2];
    // acceleration from the world thrust F = R e_z T (with floor friction on the floor)
    float lF[3];
    if (!on_floor) {
        for (int k = 0; k < 3; ++k) lF[k] = la[k] * p.inv_m;
    } else {
        const float lf0 = la[0] * p.inv_m, lf1 = la[1] * p.inv_m;  // a_z = 0 on the floor
        if (still) {
            if (keep > 0.0f) {  // f = F_xy (1 - ffric / nf), ffric = mu (m g - F_z)
                const float q = (F0 * lf0 + F1 * lf1) * __frcp_rn(nf);
                lF[0] = keep * lf0 + ffric * F0 * q * __frcp_rn(nf * nf);
                lF[1] = keep * lf1 + ffric * F1 * q * __frcp_rn(nf * nf);
                lF[2] = c.mu * q;
            } else {
                lF[0] = lF[1] = lF[2] = 0.0f;
            }
        } else {  // f = F_xy - ffric v / |v|
            lF[0] = lf0;
            lF[1] = lf1;
            const float q = vh[0] * lf0 + vh[1] * lf1;
            lF[2] = c.mu * q;
            lv[0] -= ffric * inv_nv * (lf0 - vh[0] * q);
            lv[1] -= ffric * inv_nv * (lf1 - vh[1] * q);
        }
    }
    const float lT = lF[0] * s.R[2] + lF[1] * s.R[5] + lF[2] * s.R[8];
    lR[2] += T * lF[0];
    lR[5] += T * lF[1];
    lR[8] += T * lF[2];
    // motors (as in the smooth form)
    const float gx = mu[0] * sa, gy = mu[1] * sa, gz = mu[2] * c.kappa;
    const float lf[4] = {lT + gx - gy - gz, lT + gx + gy + gz, lT - gx + gy - gz, lT - gx - gy + gz};
    for (int r = 0; r < 4; ++r) {
        const float luf1 = luf[r] + 2.f * p.fmax * uf1[r] * lf[r];
        const float leps1 = leps[r] + lf[r];
        leps[r] = (c.flags & QS_F_MOTOR_NOISE) ? c.alpha_nd * leps1 : leps1;
        luf[r] = (1.f - p.alag) * luf1;
        lu[r] += p.alag * luf1;
    }
}

// The collision pass of a control step (S9, S10) as the step kernels run it:
// positions and pre-collision velocities staged in shared memory (sx, sv:
// [3][nt]). Every thread of the CTA calls it.
// Returns whether any drone of the group responded (the same value in every
// thread of the group).
__device__ __forceinline__ bool discrete_collisions(const Consts& c, Drone& s, const Prm& p, uint32_t tick, int d,
                                                    bool act, float* sx, float* sv, int nt, int sbase, int lane, int N,
                                                    int lt, int bid, int bn) {
    if (act) {
        sx[lt] = s.x[0];
        sx[nt + lt] = s.x[1];
        sx[2 * nt + lt] = s.x[2];
        sv[lt] = s.v[0];
        sv[nt + lt] = s.v[1];
        sv[2 * nt + lt] = s.v[2];
    }
    group_sync(bid, bn);
    float dvs[3] = {0.f, 0.f, 0.f};
    bool responded = false;
    if (act && N > 1) {
        uint32_t ev = 0;
        uint64_t best[QS_MAX_K];
        float az = 0.f;
        bool dwh = false;
        responded = pair_scan(c, s, p.thr, lane, N, sbase, sx, sv, nt, 0, true, true, ev, best, dvs, false, az, dwh);
    }
    const bool any = group_sync_or(bid, bn, responded);
    if (responded) apply_response(c, s, tick, d, dvs);
    return any;
}

// ---------------------------------------------------------------- event-time pair contacts
// With QS_F_EVENT_TIME a colliding, approaching pair (i, j) is taken to have
// touched sigma_ij before the end of the control step: running the pair's
// relative motion back, r(s) = r - u s with r = x_i - x_j, u = v_i - v_j, the
// separation equals the contact distance (key = thr) at
//   sigma = -c0 / (sqrt(b^2 - a c0) - b),  a = |u|^2, b = u . r (< 0), c0 = key - thr (< 0),
// at most the step's duration. The exchange with j acts on drone i's
// position from then on, the decay and the perturbation from its earliest
// contact sigma* = max_j sigma_ij:
//   x_i' = x_i + alpha_c sum_j v~_ij sigma_ij + D_i sigma*,  D_i = v_i' - v_i - alpha_c sum_j v~_ij.
// Derivatives of sigma (implicit function, p = r - u sigma the separation at
// contact): d sigma / d r = -p / (a sigma - b), d sigma / d u = sigma p / (a sigma - b).
struct PairEt {
    float n[3], w[3], vn, inv, sig, p[3], den;
    bool free;
};

__device__ __forceinline__ PairEt pair_et(const float dx[3], float key, float thr, const float rv[3], float app,
                                          float Tc) {
    PairEt q;
    q.inv = key > 0.0f ? rsqrtf(key) : 0.0f;
    q.n[0] = key > 0.0f ? -dx[0] * q.inv : 0.0f;
    q.n[1] = key > 0.0f ? -dx[1] * q.inv : 0.0f;
    q.n[2] = key > 0.0f ? -dx[2] * q.inv : 1.0f;
    for (int k = 0; k < 3; ++k) q.w[k] = -rv[k];  // v_j - v_i
    q.vn = dot3(q.w[0], q.w[1], q.w[2], q.n[0], q.n[1], q.n[2]);
    const float a = dot3(rv[0], rv[1], rv[2], rv[0], rv[1], rv[2]);
    const float c0 = __fsub_rn(key, thr);
    const float raw = -c0 / __fsub_rn(sqrtf(fmaxf(cross_c(app, app, a, c0), 0.0f)), app);
    q.free = raw > 0.0f && raw < Tc;
    q.sig = fminf(fmaxf(raw, 0.0f), Tc);
    for (int k = 0; k < 3; ++k) q.p[k] = __fmaf_rn(-rv[k], q.sig, -dx[k]);  // r - u sigma
    q.den = __fmaf_rn(a, q.sig, -app);
    return q;
}

// The event-time collision pass of a control step (forward); returns whether
// any drone of the group responded (the same value in every thread of it).
__device__ __forceinline__ bool discrete_collisions_et(const Consts& c, Drone& s, const Prm& p, uint32_t tick, int d,
                                                       bool act, float* sx, float* sv, int nt, int sbase, int lane,
                                                       int N, int lt, int bid, int bn) {
    if (act) {
        sx[lt] = s.x[0];
        sx[nt + lt] = s.x[1];
        sx[2 * nt + lt] = s.x[2];
        sv[lt] = s.v[0];
        sv[nt + lt] = s.v[1];
        sv[2 * nt + lt] = s.v[2];
    }
    group_sync(bid, bn);
    float dvs[3] = {0.f, 0.f, 0.f}, dxs[3] = {0.f, 0.f, 0.f}, smax = 0.f;
    bool responded = false;
    if (act && N > 1) {
        const float Tc = c.substeps * c.dt;
        for (int j = 0; j < N; ++j) {
            if (j == lane) continue;
            const int tj = sbase + j;
            float dx[3];
            const float key = pair_key(s.x[0], s.x[1], s.x[2], sx[tj], sx[nt + tj], sx[2 * nt + tj], dx[0], dx[1], dx[2]);
            if (!(key < p.thr)) continue;
            const float rv[3] = {s.v[0] - sv[tj], s.v[1] - sv[nt + tj], s.v[2] - sv[2 * nt + tj]};
            const float app = -dot3(rv[0], rv[1], rv[2], dx[0], dx[1], dx[2]);
            if (!(app < 0.0f)) continue;
            const PairEt q = pair_et(dx, key, p.thr, rv, app, Tc);
            for (int k = 0; k < 3; ++k) {
                dvs[k] = fmaf(q.vn, q.n[k], dvs[k]);
                dxs[k] = fmaf(q.vn * q.sig, q.n[k], dxs[k]);
            }
            smax = fmaxf(smax, q.sig);
            responded = true;
        }
    }
    const bool any = group_sync_or(bid, bn, responded);
    if (responded) {
        float n[6];
        six_normals(c, tick, (uint32_t)d, TAG_COLL, 0, n);
        for (int k = 0; k < 3; ++k) {
            const float v0 = s.v[k];
            s.v[k] = __fmul_rn(c.alpha_c, __fmaf_rn(c.sig_cv, n[k], __fadd_rn(s.v[k], dvs[k])));
            comp_add_prod(s.w[k], s.wlo[k], c.sig_cw, n[3 + k]);
            const float Dk = __fmaf_rn(-c.alpha_c, dvs[k], __fsub_rn(s.v[k], v0));
            s.x[k] = fmaf(Dk, smax, fmaf(c.alpha_c, dxs[k], s.x[k]));
        }
    }
    return any;
}

// Adjoint of the collision pass: xs, vs the pre-collision position and
// velocity of the thread's drone (as staged: sx, sv), sl the lambda of every
// drone's post-collision velocity. For a responding drone i,
//   v_i' = alpha_c (v_i + sum_j ((v_j - v_i) . n_ij) n_ij + eps),
//   n_ij = (x_i - x_j) / d_ij,
// so lambda_v_i = alpha_c (lambda_v_i' + sum_j n n^T (lambda_v_j' - lambda_v_i'))
// and lambda_x_i += sum_j alpha_c / d P ((n . q) (v_j - v_i) + vn q) with
// q = lambda_v_i' - lambda_v_j', P = I - n n^T, vn = (v_j - v_i) . n
// (the partner relation is symmetric, so every partner also responded).
__device__ __forceinline__ void collision_vjp(const Consts& c, const float xs[3], const float vs[3], float thr,
                                              const float* sx, const float* sv, const float* sl, int nt, int sbase,
                                              int lane, int N, float lx[3], float lv[3]) {
    const float l0[3] = {lv[0], lv[1], lv[2]};
    float acc_v[3] = {0.f, 0.f, 0.f}, acc_x[3] = {0.f, 0.f, 0.f};
    bool responded = false;
    for (int j = 0; j < N; ++j) {
        if (j == lane) continue;
        const int tj = sbase + j;
        float dx, dy, dz;
        const float key = pair_key(xs[0], xs[1], xs[2], sx[tj], sx[nt + tj], sx[2 * nt + tj], dx, dy, dz);
        if (!(key < thr)) continue;
        const float rv0 = vs[0] - sv[tj], rv1 = vs[1] - sv[nt + tj], rv2 = vs[2] - sv[2 * nt + tj];
        if (!(-dot3(rv0, rv1, rv2, dx, dy, dz) < 0.0f)) continue;  // approaching
        responded = true;
        float n[3] = {0.f, 0.f, 1.f}, inv = 0.f;
        if (key > 0.0f) {
            inv = rsqrtf(key);
            n[0] = -dx * inv;
            n[1] = -dy * inv;
            n[2] = -dz * inv;
        }
        const float q[3] = {l0[0] - sl[tj], l0[1] - sl[nt + tj], l0[2] - sl[2 * nt + tj]};
        const float nq = n[0] * q[0] + n[1] * q[1] + n[2] * q[2];
        for (int k = 0; k < 3; ++k) acc_v[k] -= n[k] * nq;
        if (key > 0.0f) {
            const float dv[3] = {-rv0, -rv1, -rv2};  // v_j - v_i
            const float vn = dv[0] * n[0] + dv[1] * n[1] + dv[2] * n[2];
            float y[3];
            for (int k = 0; k < 3; ++k) y[k] = nq * dv[k] + vn * q[k];
            const float ny = n[0] * y[0] + n[1] * y[1] + n[2] * y[2];
            for (int k = 0; k < 3; ++k) acc_x[k] += (y[k] - ny * n[k]) * inv;
        }
    }
    if (responded) {
        for (int k = 0; k < 3; ++k) {
            lv[k] = c.alpha_c * (l0[k] + acc_v[k]);
            lx[k] += c.alpha_c * acc_x[k];
        }
    }
}

// lambda x += d loss / d x of step t's term |x - g|^2 (scaled by dl), with
// explicit roundings: the same bits whether or not the collision reverse runs.
__device__ __forceinline__ void loss_term(float dl, const float x[3], const float g[3], float lx[3]) {
    const float s2 = __fmul_rn(dl, 2.f);
    for (int k = 0; k < 3; ++k) lx[k] = __fmaf_rn(s2, __fsub_rn(x[k], g[k]), lx[k]);
}

// Adjoint of the event-time collision pass together with step t's loss term,
// which the pass's position correction feeds: on entry lx, lv hold lambda of
// the post-collision x and v without that term, on return lambda of the
// pre-collision x and v. sc: the pre-collision state. Every thread of the
// group calls it. For a responding drone i (notation of discrete_collisions_et):
//  - the exchange terms alpha_c v~_ij . (lambda v'_i - lambda v'_j) as in
//    collision_vjp, and alpha_c sigma_ij v~_ij . (lambda x'_i - lambda x'_j);
//  - the decay: lambda v_i += (alpha_c - 1) sigma* lambda x'_i;
//  - through sigma_ij: lambda (x_i, v_i) += W_ij (d sigma / d r, d sigma / d u) with
//    W_ij = alpha_c vn (n . (lambda x'_i - lambda x'_j)) + [j is i's earliest]
//    lambda x'_i . D_i + [i is j's earliest] lambda x'_j . D_j.
// The partners' lambdas, lambda x' . D and earliest partners are exchanged
// through shared memory (sl, slx, sq, sarg: [3][nt], [3][nt], [nt], [nt]).
__device__ __forceinline__ void collision_vjp_et(const Consts& c, const Drone& sc, const Prm& p, uint32_t tick, int d,
                                                 bool act, float* sx, float* sv, float* sl, float* slx, float* sq,
                                                 int* sarg, int nt, int sbase, int lane, int N, int lt, int bid, int bn,
                                                 float dl, const float g[3], float lx[3], float lv[3]) {
    const float Tc = c.substeps * c.dt, ac = c.alpha_c;
    if (act) {
        sx[lt] = sc.x[0];
        sx[nt + lt] = sc.x[1];
        sx[2 * nt + lt] = sc.x[2];
        sv[lt] = sc.v[0];
        sv[nt + lt] = sc.v[1];
        sv[2 * nt + lt] = sc.v[2];
    }
    group_sync(bid, bn);
    float dvs[3] = {0.f, 0.f, 0.f}, dxs[3] = {0.f, 0.f, 0.f}, smax = 0.f, Dv[3] = {0.f, 0.f, 0.f};
    int m = -1;
    bool responded = false;
    if (act && N > 1) {
        for (int j = 0; j < N; ++j) {
            if (j == lane) continue;
            const int tj = sbase + j;
            float dx[3];
            const float key = pair_key(sc.x[0], sc.x[1], sc.x[2], sx[tj], sx[nt + tj], sx[2 * nt + tj], dx[0], dx[1],
                                       dx[2]);
            if (!(key < p.thr)) continue;
            const float rv[3] = {sc.v[0] - sv[tj], sc.v[1] - sv[nt + tj], sc.v[2] - sv[2 * nt + tj]};
            const float app = -dot3(rv[0], rv[1], rv[2], dx[0], dx[1], dx[2]);
            if (!(app < 0.0f)) continue;
            const PairEt q = pair_et(dx, key, p.thr, rv, app, Tc);
            for (int k = 0; k < 3; ++k) {
                dvs[k] = fmaf(q.vn, q.n[k], dvs[k]);
                dxs[k] = fmaf(q.vn * q.sig, q.n[k], dxs[k]);
            }
            if (q.sig > smax || m < 0) {
                if (q.sig > smax) smax = q.sig;
                if (q.sig >= smax) m = j;
            }
            responded = true;
        }
    }
    float xp[3] = {sc.x[0], sc.x[1], sc.x[2]}, qd = 0.f;
    if (responded) {
        float n[6];
        six_normals(c, tick, (uint32_t)d, TAG_COLL, 0, n);
        for (int k = 0; k < 3; ++k) {
            const float v1 = __fmul_rn(ac, __fmaf_rn(c.sig_cv, n[k], __fadd_rn(sc.v[k], dvs[k])));
            Dv[k] = __fmaf_rn(-ac, dvs[k], __fsub_rn(v1, sc.v[k]));
            xp[k] = fmaf(Dv[k], smax, fmaf(ac, dxs[k], sc.x[k]));
        }
    }
    if (act) loss_term(dl, xp, g, lx);  // loss of step t at the post-collision position
    if (act) {
        if (responded) qd = lx[0] * Dv[0] + lx[1] * Dv[1] + lx[2] * Dv[2];
        sl[lt] = lv[0];
        sl[nt + lt] = lv[1];
        sl[2 * nt + lt] = lv[2];
        slx[lt] = lx[0];
        slx[nt + lt] = lx[1];
        slx[2 * nt + lt] = lx[2];
        sq[lt] = qd;
        sarg[lt] = responded ? m : -1;
    }
    group_sync(bid, bn);
    if (responded) {
        const float l0[3] = {lv[0], lv[1], lv[2]}, x0[3] = {lx[0], lx[1], lx[2]};
        float acc_v[3] = {0.f, 0.f, 0.f}, acc_x[3] = {0.f, 0.f, 0.f}, gx[3] = {0.f, 0.f, 0.f}, gv[3] = {0.f, 0.f, 0.f};
        for (int j = 0; j < N; ++j) {
            if (j == lane) continue;
            const int tj = sbase + j;
            float dx[3];
            const float key = pair_key(sc.x[0], sc.x[1], sc.x[2], sx[tj], sx[nt + tj], sx[2 * nt + tj], dx[0], dx[1],
                                       dx[2]);
            if (!(key < p.thr)) continue;
            const float rv[3] = {sc.v[0] - sv[tj], sc.v[1] - sv[nt + tj], sc.v[2] - sv[2 * nt + tj]};
            const float app = -dot3(rv[0], rv[1], rv[2], dx[0], dx[1], dx[2]);
            if (!(app < 0.0f)) continue;
            const PairEt q = pair_et(dx, key, p.thr, rv, app, Tc);
            const float qv[3] = {l0[0] - sl[tj], l0[1] - sl[nt + tj], l0[2] - sl[2 * nt + tj]};
            const float qx[3] = {x0[0] - slx[tj], x0[1] - slx[nt + tj], x0[2] - slx[2 * nt + tj]};
            const float nq = q.n[0] * qv[0] + q.n[1] * qv[1] + q.n[2] * qv[2];
            const float nQ = q.n[0] * qx[0] + q.n[1] * qx[1] + q.n[2] * qx[2];
            for (int k = 0; k < 3; ++k) acc_v[k] -= q.n[k] * (nq + q.sig * nQ);
            if (key > 0.0f) {
                float y[3];
                for (int k = 0; k < 3; ++k) y[k] = (nq + q.sig * nQ) * q.w[k] + q.vn * (qv[k] + q.sig * qx[k]);
                const float ny = q.n[0] * y[0] + q.n[1] * y[1] + q.n[2] * y[2];
                for (int k = 0; k < 3; ++k) acc_x[k] += (y[k] - ny * q.n[k]) * q.inv;
            }
            if (q.free) {
                float W = ac * q.vn * nQ;
                if (m == j) W += qd;
                if (sarg[tj] == lane) W += sq[tj];
                const float f = W / q.den;
                for (int k = 0; k < 3; ++k) {
                    gx[k] -= f * q.p[k];
                    gv[k] += f * q.sig * q.p[k];
                }
            }
        }
        for (int k = 0; k < 3; ++k) {
            lv[k] = ac * (l0[k] + acc_v[k]) + (ac - 1.f) * smax * x0[k] + gv[k];
            lx[k] = x0[k] + ac * acc_x[k] + gx[k];
        }
    }
    group_sync(bid, bn);
}

template <bool ET>
__global__ void __launch_bounds__(ADJ_BLOCK_MAX) k_diffd_fwd(const Consts c, const Dev dv, const Tile* __restrict__ tiles,
                                                             const int* __restrict__ perm, const DiffArgs a) {
    extern __shared__ float sm[];
    const int nb = blockDim.x >> 1, grp = threadIdx.x >= nb ? 1 : 0, lt = threadIdx.x - grp * nb;
    const Tile tile = tile_at(dv, tiles, blockIdx.x, nb);
    const int W = tile.W, nt = nb;
    const int slot = lt / W, lane = lt - slot * W;
    const SlotGeo geo = slot_geometry(dv, perm, tile, slot, W, nt);
    const int e = geo.e, d0 = geo.d0, N = geo.N;
    const bool act = lane < N;
    const int d = d0 + lane, sbase = slot * W;
    const size_t D = dv.D;
    const bool coll = (c.flags & QS_F_COLLISIONS) != 0;
    const bool ahead = (c.flags & QS_F_MOTOR_NOISE) && c.substeps <= FWD_SUB;
    float* nbase = sm + 9 * nb;  // [2][FWD_SUB][4][nb] motor normals
    const uint32_t tick0 = act ? dv.tick[e] : 0u;
    if (grp == 1) {
        fwd_noise_group(c, nbase, nb, lt, act, ahead, tick0, d, a.T);
        return;
    }
    Drone s;
    Prm p;
    float g[3] = {0.f, 0.f, 0.f};
    if (act) {
        read_x0(s, a.x0, d);
        p = load_prm(c, dv.prm, dv.E, e);
        g[0] = dv.goal[e];
        g[1] = dv.goal[dv.E + e];
        g[2] = dv.goal[2 * dv.E + e];
    }
    const float zero3[3] = {0.f, 0.f, 0.f};
    float L = 0.f;
    for (int t = 0; t < a.T; ++t) {
        __syncthreads();  // step t's motor normals ready (group 1)
        if (act && t % a.C == 0) {
            float4 q[NPLANE];
            pack(s, q);
            float4* ck = a.ckpt + (size_t)(t / a.C) * NPLANE * D;
            for (int pl = 0; pl < NPLANE; ++pl) ck[(size_t)pl * D + d] = q[pl];
        }
        float fh[4] = {0.f, 0.f, 0.f, 0.f}, u[4] = {0.f, 0.f, 0.f, 0.f}, msk[4];
        if (act) {
            command4(c, a.act, D, t, d, fh, u, msk);
            for (int sub = 0; sub < c.substeps; ++sub) {
                float n[4];
                if (ahead)
                    for (int r = 0; r < 4; ++r) n[r] = *fwd_normals(nbase, nb, t & 1, sub, r, lt);
                substep<ET, 0>(s, p, c, u, tick0 + t, d, sub, zero3, ahead ? n : nullptr);
            }
        }
        if (coll && ET) discrete_collisions_et(c, s, p, tick0 + t, d, act, sm, sm + 3 * nt, nt, sbase, lane, N, lt, 1, nb);
        else if (coll) discrete_collisions(c, s, p, tick0 + t, d, act, sm, sm + 3 * nt, nt, sbase, lane, N, lt, 1, nb);
        if (act) {
            const float dx = s.x[0] - g[0], dy = s.x[1] - g[1], dz = s.x[2] - g[2];
            L += dx * dx + dy * dy + dz * dz + 1e-3f * (fh[0] * fh[0] + fh[1] * fh[1] + fh[2] * fh[2] + fh[3] * fh[3]);
        }
    }
    if (act) {
        a.loss[d] = L;
        if (!finite_state(s)) atomicOr(dv.status, 1);
    }
}

// Adjoint of the discrete-contact rollout, pipelined over checkpoint segments
// like k_diff_bwd: group 0 recomputes segment s - 1 (every substep input and
// each step's pre-collision state) into one scratch buffer while group 1
// reverses segment s from the other.
template <bool ET>
__global__ void __launch_bounds__(ADJ_BLOCK_MAX) k_diffd_bwd(const Consts c, const Dev dv, const Tile* __restrict__ tiles,
                                                             const int* __restrict__ perm, const DiffArgs a) {
    extern __shared__ float sm[];
    const int nb = blockDim.x >> 1, grp = threadIdx.x >= nb ? 1 : 0, lt = threadIdx.x - grp * nb, bid = 1 + grp;
    const Tile tile = tile_at(dv, tiles, blockIdx.x, nb);
    const int W = tile.W, nt = nb;
    const int slot = lt / W, lane = lt - slot * W;
    const SlotGeo geo = slot_geometry(dv, perm, tile, slot, W, nt);
    const int e = geo.e, d0 = geo.d0, N = geo.N;
    const bool act = lane < N;
    const int d = d0 + lane, sbase = slot * W;
    const size_t D = dv.D;
    const bool coll = (c.flags & QS_F_COLLISIONS) != 0;
    float* sx = sm + grp * 6 * nb;       // [3][nb] positions of the group
    float* sv = sx + 3 * nb;             // [3][nb] velocities of the group
    float* sl = sm + 12 * nb;            // [3][nb] lambda of the post-collision velocity (group 1)
    float* slx = sm + 15 * nb;           // event time: [3][nb] lambda of the post-collision position,
    float* sq = sm + 18 * nb;            //   [nb] lambda x' . D, [nb] earliest partner (group 1)
    int* sarg = reinterpret_cast<int*>(sm + 19 * nb);
    // [2][RFLAG_WORDS] bit q: some drone of the group responded to a collision
    // in step tb + q of the segment recomputed into that buffer (steps beyond
    // RFLAG_BITS are taken as responding); the reverse skips the collision
    // adjoint of a step without responses, which is then the identity
    uint32_t* rflag = reinterpret_cast<uint32_t*>(sm + 23 * nb);
    const int S = c.substeps, S1 = c.substeps + 1;  // saved states per step: each substep's input, then the pre-collision state
    const size_t sbuf = (size_t)a.C * S1 * NSUB * D;  // floats of one scratch buffer
    Prm p;
    float g[3] = {0.f, 0.f, 0.f};
    uint32_t tick0 = 0;
    float dl = 0.f;
    if (act) {
        p = load_prm(c, dv.prm, dv.E, e);
        g[0] = dv.goal[e];
        g[1] = dv.goal[dv.E + e];
        g[2] = dv.goal[2 * dv.E + e];
        tick0 = dv.tick[e];
        dl = a.dloss[d];
    }
    float lx[3] = {0.f, 0.f, 0.f}, lv[3] = {0.f, 0.f, 0.f}, lR[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float lw[3] = {0.f, 0.f, 0.f}, luf[4] = {0.f, 0.f, 0.f, 0.f}, leps[4] = {0.f, 0.f, 0.f, 0.f};
    const float zero3[3] = {0.f, 0.f, 0.f};
    const int nseg = (a.T + a.C - 1) / a.C;
    for (int it = 0; it <= nseg; ++it) {
        if (grp == 0 && it < nseg) {
            // recompute segment nseg - 1 - it
            const int seg = nseg - 1 - it, tb = seg * a.C, te = min(a.T, tb + a.C);
            float* scr = a.scratch + (size_t)(it & 1) * sbuf;
            uint32_t* fl = rflag + (it & 1) * RFLAG_WORDS;
            if (lt == 0)
                for (int w = 0; w < RFLAG_WORDS; ++w) fl[w] = 0u;
            Drone s;
            if (act) {
                float4 q[NPLANE];
                const float4* ck = a.ckpt + (size_t)seg * NPLANE * D;
                for (int pl = 0; pl < NPLANE; ++pl) q[pl] = ck[(size_t)pl * D + d];
                unpack(s, q);
            }
            for (int t = tb; t < te; ++t) {
                float fh[4] = {0.f, 0.f, 0.f, 0.f}, u[4] = {0.f, 0.f, 0.f, 0.f}, msk[4];
                if (act) {
                    command4(c, a.act, D, t, d, fh, u, msk);
                    for (int sub = 0; sub < S; ++sub) {
                        save_sub(scr, D, (t - tb) * S1 + sub, d, s);
                        substep<ET, 0>(s, p, c, u, tick0 + t, d, sub, zero3);
                    }
                    save_sub(scr, D, (t - tb) * S1 + S, d, s);
                }
                bool any = false;
                if (coll && ET)
                    any = discrete_collisions_et(c, s, p, tick0 + t, d, act, sx, sv, nt, sbase, lane, N, lt, bid, nb);
                else if (coll)
                    any = discrete_collisions(c, s, p, tick0 + t, d, act, sx, sv, nt, sbase, lane, N, lt, bid, nb);
                if (lt == 0 && any && t - tb < RFLAG_BITS) fl[(t - tb) >> 5] |= 1u << ((t - tb) & 31);
            }
        } else if (grp == 1 && it >= 1) {
            // reverse through segment nseg - it, recomputed in the previous round
            const int seg = nseg - it, tb = seg * a.C, te = min(a.T, tb + a.C);
            const float* scr = a.scratch + (size_t)((it - 1) & 1) * sbuf;
            const uint32_t* fl = rflag + ((it - 1) & 1) * RFLAG_WORDS;
            for (int t = te - 1; t >= tb; --t) {
                const int q = t - tb;  // the same in every thread of the group
                const bool any = q >= RFLAG_BITS || ((fl[q >> 5] >> (q & 31)) & 1u);
                float fh[4] = {0.f, 0.f, 0.f, 0.f}, u[4] = {0.f, 0.f, 0.f, 0.f}, msk[4] = {0.f, 0.f, 0.f, 0.f};
                Drone sc;
                if (act) {
                    command4(c, a.act, D, t, d, fh, u, msk);
                    load_sub(scr, D, (t - tb) * S1 + S, d, sc);
                    // loss of step t: |x(t) - g|^2 + 1e-3 |f^|^2 (the collision pass leaves x
                    // unchanged; the event-time pass moves it and adds the term itself)
                    if (!(ET && coll && any)) loss_term(dl, sc.x, g, lx);
                }
                if (coll && ET && any) {
                    collision_vjp_et(c, sc, p, tick0 + t, d, act, sx, sv, sl, slx, sq, sarg, nt, sbase, lane, N, lt, bid,
                                     nb, dl, g, lx, lv);
                } else if (coll && any) {
                    if (act) {
                        sx[lt] = sc.x[0];
                        sx[nt + lt] = sc.x[1];
                        sx[2 * nt + lt] = sc.x[2];
                        sv[lt] = sc.v[0];
                        sv[nt + lt] = sc.v[1];
                        sv[2 * nt + lt] = sc.v[2];
                        sl[lt] = lv[0];
                        sl[nt + lt] = lv[1];
                        sl[2 * nt + lt] = lv[2];
                    }
                    group_sync(bid, nb);
                    if (act && N > 1) collision_vjp(c, sc.x, sc.v, p.thr, sx, sv, sl, nt, sbase, lane, N, lx, lv);
                    group_sync(bid, nb);
                }
                float lu[4] = {0.f, 0.f, 0.f, 0.f};
                if (act) {
                    for (int sub = S - 1; sub >= 0; --sub) {
                        Drone si;
                        float eps1[4], vo[3];
                        load_sub(scr, D, (t - tb) * S1 + sub, d, si);
                        load_eps(scr, D, (t - tb) * S1 + sub + 1, d, eps1);
                        if (ET) load_v(scr, D, (t - tb) * S1 + sub + 1, d, vo);
                        discrete_substep_vjp<ET>(si, p, c, u, eps1, vo, lx, lv, lR, lw, luf, leps, lu);
                    }
                    float ga[4];
                    for (int r = 0; r < 4; ++r) {
                        const float du = u[r] > 0.f ? 0.5f * rcp_approx(u[r]) : 0.f;
                        ga[r] = msk[r] * (lu[r] * du + dl * 2e-3f * fh[r]);
                    }
                    reinterpret_cast<float4*>(a.grad_act + (size_t)t * D * 4)[d] = make_float4(ga[0], ga[1], ga[2], ga[3]);
                }
            }
        }
        __syncthreads();  // hand over: buffer it & 1 recomputed; buffer (it - 1) & 1 free again
    }
    if (grp == 1 && act) {
        float* gx = a.grad_x0 + (size_t)d * QS_STATE_DIM;
        for (int k = 0; k < 3; ++k) gx[k] = lx[k];
        for (int k = 0; k < 3; ++k) gx[3 + k] = lv[k];
        for (int k = 0; k < 9; ++k) gx[6 + k] = lR[k];
        for (int k = 0; k < 3; ++k) gx[15 + k] = lw[k];
        for (int k = 0; k < 4; ++k) gx[18 + k] = luf[k];
        for (int k = 0; k < 4; ++k) gx[22 + k] = leps[k];
        for (int k = 0; k < 4; ++k) gx[26 + k] = 0.f;  // f^_prev does not enter the loss
    }
}

cudaError_t launch_diff(int backward, const Consts& c, const Dev& dv, const Tile* tiles, int n_tiles, int block,
                        const int* perm, const float* x0, const float* act, float* loss, const float* dloss,
                        float* grad_act, float* grad_x0, void* workspace, int T, int C, cudaStream_t st) {
    DiffArgs a;
    a.x0 = x0;
    a.act = act;
    a.loss = loss;
    a.dloss = dloss;
    a.grad_act = grad_act;
    a.grad_x0 = grad_x0;
    a.T = T;
    a.C = C;
    const int nck = (T + C - 1) / C;
    a.ckpt = reinterpret_cast<float4*>(workspace);
    a.scratch = reinterpret_cast<float*>(reinterpret_cast<char*>(workspace) + (size_t)nck * NPLANE * dv.D * sizeof(float4));
    // forward: two groups of `block` threads (integration, motor normals ahead);
    // backward: two (recompute, reverse) with up to 23 planes of `block` floats
    // (positions and velocities of both groups, the reverse's lambdas of the
    // post-collision velocity and, with event-time contacts, position, its
    // lambda x' . D and earliest partner: 20 planes)
    const size_t smem = sizeof(float) * (9 + 2 * FWD_SUB * 4) * block,
                 smem2 = sizeof(float) * 23 * block + sizeof(uint32_t) * 2 * RFLAG_WORDS;
    if (2 * block > ADJ_BLOCK_MAX) return cudaErrorInvalidValue;
    if (c.flags & QS_F_SMOOTH) {
        if (backward) k_diff_bwd<<<n_tiles, 2 * block, smem2, st>>>(c, dv, tiles, perm, a);
        else k_diff_fwd<<<n_tiles, 2 * block, smem, st>>>(c, dv, tiles, perm, a);
    } else if (c.flags & QS_F_EVENT_TIME) {
        if (backward) k_diffd_bwd<true><<<n_tiles, 2 * block, smem2, st>>>(c, dv, tiles, perm, a);
        else k_diffd_fwd<true><<<n_tiles, 2 * block, smem, st>>>(c, dv, tiles, perm, a);
    } else {
        if (backward) k_diffd_bwd<false><<<n_tiles, 2 * block, smem2, st>>>(c, dv, tiles, perm, a);
        else k_diffd_fwd<false><<<n_tiles, 2 * block, smem, st>>>(c, dv, tiles, perm, a);
    }
    return cudaGetLastError();
}

}  // namespace qsk
