// qs_device.cuh -- device-side physics of the QuadSwarm step in binary32.
//
// One drone's state lives in registers (struct Drone); the functions below
// follow the paper's step (Sec. III-A .. III-E) in the order the step kernel
// calls them. Random numbers come from Philox4x32-10 (Salmon et al., SC'11)
// keyed by the seed, with counter (env step, drone or env id,
// tag << 16 | substream << 8 | block, 0).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "qs_internal.h"

namespace qsk {

// ---------------------------------------------------------------- Philox4x32-10
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t k0, uint32_t k1) {
    uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = 0u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, x0), lo0 = 0xD2511F53u * x0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, x2), lo1 = 0xCD9E8D57u * x2;
        const uint32_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
    return make_uint4(x0, x1, x2, x3);
}

// Same generator with the ten round keys precomputed (the Weyl schedule is the
// same for every thread): each round is two 32x32->64 multiplies and two
// three-input XORs.
__device__ __forceinline__ uint4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, const uint32_t rk[20]) {
    uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = 0u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        const uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ rk[2 * r];
        const uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ rk[2 * r + 1];
        x1 = (uint32_t)p1;
        x3 = (uint32_t)p0;
        x0 = y0;
        x2 = y2;
    }
    return make_uint4(x0, x1, x2, x3);
}

__device__ __forceinline__ uint32_t ctr_word(uint32_t tag, uint32_t sub, uint32_t blk) {
    return (tag << 16) | (sub << 8) | blk;
}

// (2k+1)/2^24 with k the top 23 bits: inside (0,1), exact in binary32. Formed
// from the bits of 1 + k 2^-23 (k as the mantissa) minus 1 - 2^-24, a
// difference that is exact (the operands lie within a factor of two), so no
// integer-to-float conversion is needed.
__device__ __forceinline__ float u01(uint32_t r) {
    return __fsub_rn(__uint_as_float(0x3F800000u | (r >> 9)), 0.99999994039535522f);
}

// Square root by the hardware approximation (PTX sqrt.approx.ftz.f32): a
// couple of instructions where the correctly rounded sqrtf takes a longer
// sequence with a special-case branch. Its relative error (measured on GB300
// over the command range by tests/test_gpu_closed_forms.py) is a few units in
// the last place at most, far inside every tolerance of the values it feeds:
// the Box-Muller radius, the rotor-speed command sqrt(f^) and the reward's
// norms. The .ftz form takes a subnormal argument (below 2^-126) as zero and
// so skips the scaling the plain form wraps around the hardware operation;
// the roots it then returns as 0 are below 1.1e-19. (The three .ftz forms here
// measured 4.6% faster in the batched step at 1,048,576 envs, same bits on
// every argument these paths see.)
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Reciprocal by the hardware approximation (PTX rcp.approx.ftz.f32, about one
// unit in the last place), where the correctly rounded __frcp_rn carries a
// longer sequence with a special-case branch. Its arguments (masses and
// inertias, 1 + c, distances, logistic denominators) are never subnormal.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// exp(x) = 2^(x log2 e) and ln(x) = log2(x) ln 2 on the hardware base-2
// approximations (PTX ex2.approx.ftz.f32, lg2.approx.ftz.f32): a scaling and
// one hardware operation, without the argument checks of the library forms.
// A result or argument below 2^-126 is taken as zero. The logarithm's error
// stays inside the bound the Box-Muller normals are tested against
// (2^-21.41 absolute on [0.5, 2]); the exponential feeds the smooth contact
// penalties, where the differentiable rollout's tests bound it.
__device__ __forceinline__ float exp_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__fmul_rn(x, 1.44269504088896341f)));
    return y;
}
__device__ __forceinline__ float log_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return __fmul_rn(y, 0.693147180559945309f);
}

// Reciprocal square root by the hardware approximation (PTX
// rsqrt.approx.ftz.f32) for arguments known to be at least 1.
__device__ __forceinline__ float rsqrt_approx_ge1(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Box-Muller: two N(0,1) from two uniforms, (rho cos 2 pi u1, rho sin 2 pi u1),
// rho = sqrt(-2 ln u0). The angle is evaluated as 2 pi (u1 - 1/2) + pi, i.e.
// cos(2 pi u1) = -cos(theta), sin(2 pi u1) = -sin(theta) with theta in (-pi, pi),
// where the hardware sine/cosine is accurate to ~4e-7 absolute. The radius
// takes the hardware logarithm (log_approx; within 2^-21.41 absolute on
// [0.5, 2] and 3 units in the last place elsewhere, the bound of __logf),
// clamped at zero where a u0 just below 1 rounds ln u0 up to a positive
// value. The error of a normal is then at most dy / (2 rho) with
// dy = 2^-20.41 max(1, rho^2 / 2), and never above sqrt(dy) ~ 8.5e-4 (radii
// near zero, whose normals are near zero too): below 2e-6 for rho > 0.2, i.e.
// for 98% of the draws. Against the library logf (about one unit in the last
// place, with a longer instruction sequence) the batched step at 1,048,576
// envs runs 7% faster (six transforms per quadrotor-step).
__device__ __forceinline__ float2 box_muller(float u0, float u1) {
    const float rho = sqrt_approx(fmaxf(-2.0f * log_approx(u0), 0.0f));
    float s, c;  // hardware sine and cosine (.ftz: the angle is never subnormal)
    const float th = 6.28318530717958648f * (u1 - 0.5f);
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(th));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(th));
    return make_float2(-rho * c, -rho * s);
}

// Six N(0,1) draws of a collision or wall perturbation (blocks 0 and 1).
__device__ __forceinline__ void six_normals(const Consts& c, uint32_t tick, uint32_t id, uint32_t tag, uint32_t sub,
                                            float n[6]) {
    const uint4 a = philox_rk(tick, id, ctr_word(tag, sub, 0), c.rk);
    const uint4 b = philox_rk(tick, id, ctr_word(tag, sub, 1), c.rk);
    const float2 p0 = box_muller(u01(a.x), u01(a.y));
    const float2 p1 = box_muller(u01(a.z), u01(a.w));
    const float2 p2 = box_muller(u01(b.x), u01(b.y));
    n[0] = p0.x; n[1] = p0.y; n[2] = p1.x; n[3] = p1.y; n[4] = p2.x; n[5] = p2.y;
}

// ---------------------------------------------------------------- per-env parameters
struct Prm {
    float m, ixx, iyy, izz, t2w, tau, arm, fmax, alag, ans, inv_m, inv_ixx, inv_iyy, inv_izz, thr, prox;
};

// The per-env constants a kernel forms from the randomised values as it loads
// them: motor-noise scale a_ns = ans_frac m g / 4, the inverses of m and the
// inertia diagonal (hardware reciprocals, about one unit in the last place),
// the collision threshold fl32((l + l)^2) and the proximity radius
// prox_factor * l. derive() stores the same values, so a kernel that loads
// them and one that forms them agree bit for bit.
__device__ __forceinline__ void complete_prm(const Consts& c, Prm& p) {
    p.ans = c.ans_frac * p.m * c.g * 0.25f;
    p.inv_m = rcp_approx(p.m);
    p.inv_ixx = rcp_approx(p.ixx);
    p.inv_iyy = rcp_approx(p.iyy);
    p.inv_izz = rcp_approx(p.izz);
    const float r = __fadd_rn(p.arm, p.arm);
    p.thr = __fmul_rn(r, r);
    p.prox = c.prox_factor * p.arm;
}

// Derived constants of the randomised values: f_max = m g t2w / 4 (max thrust
// per rotor), alpha_lag = 1 - exp(-dt / tau_m) (first-order lag whose 2%
// settling time is tau_m ln 50), and complete_prm()'s.
__device__ __forceinline__ void derive(const Consts& c, const float p7[QS_PARAM_DIM], float out[NPRM_DEV]) {
    for (int k = 0; k < QS_PARAM_DIM; ++k) out[k] = p7[k];
    Prm q;
    q.m = p7[P_M];
    q.ixx = p7[P_IXX];
    q.iyy = p7[P_IYY];
    q.izz = p7[P_IZZ];
    q.arm = p7[P_ARM];
    complete_prm(c, q);
    out[P_FMAX] = 0.25f * q.m * c.g * p7[P_T2W];
    out[P_ALAG] = -expm1f(-c.dt / p7[P_TAU]);
    out[P_ANS] = q.ans;
    out[P_INVM] = q.inv_m;
    out[P_INVIXX] = q.inv_ixx;
    out[P_INVIYY] = q.inv_iyy;
    out[P_INVIZZ] = q.inv_izz;
    out[P_THR] = q.thr;
    out[P_PROX] = q.prox;
}

// The 7 planes a step reads (m, inertia diagonal, arm, f_max, alpha_lag: 28 B
// per env); the rest is formed by complete_prm(). t2w and tau_m enter only
// through f_max and alpha_lag and are not loaded.
__device__ __forceinline__ Prm load_prm(const Consts& c, const float* __restrict__ prm, int E, int e) {
    Prm p;
    p.m = __ldg(prm + P_M * E + e);
    p.ixx = __ldg(prm + P_IXX * E + e);
    p.iyy = __ldg(prm + P_IYY * E + e);
    p.izz = __ldg(prm + P_IZZ * E + e);
    p.arm = __ldg(prm + P_ARM * E + e);
    p.fmax = __ldg(prm + P_FMAX * E + e);
    p.alag = __ldg(prm + P_ALAG * E + e);
    p.t2w = 0.f;
    p.tau = 0.f;
    complete_prm(c, p);
    return p;
}

__device__ __forceinline__ Prm prm_from(const float v[NPRM_DEV]) {
    Prm p;
    p.m = v[P_M]; p.ixx = v[P_IXX]; p.iyy = v[P_IYY]; p.izz = v[P_IZZ]; p.t2w = v[P_T2W]; p.tau = v[P_TAU];
    p.arm = v[P_ARM]; p.fmax = v[P_FMAX]; p.alag = v[P_ALAG]; p.ans = v[P_ANS]; p.inv_m = v[P_INVM];
    p.inv_ixx = v[P_INVIXX]; p.inv_iyy = v[P_INVIYY]; p.inv_izz = v[P_INVIZZ]; p.thr = v[P_THR];
    p.prox = v[P_PROX];
    return p;
}

// Domain randomisation of one env (7 scale factors U(lo,hi)) and its goal
// (uniform in the room); three Philox blocks at (tick, e, tag).
__device__ __forceinline__ void draw_env(const Consts& c, uint32_t k0, uint32_t k1, uint32_t tick, uint32_t tag,
                                         int e, float p7[QS_PARAM_DIM], float goal[3]) {
    const uint4 a = philox(tick, (uint32_t)e, ctr_word(tag, 0, 0), k0, k1);
    const uint4 b = philox(tick, (uint32_t)e, ctr_word(tag, 0, 1), k0, k1);
    const uint4 d = philox(tick, (uint32_t)e, ctr_word(tag, 0, 2), k0, k1);
    const float u[10] = {u01(a.x), u01(a.y), u01(a.z), u01(a.w), u01(b.x), u01(b.y), u01(b.z), u01(b.w),
                         u01(d.x), u01(d.y)};
    const bool dr = (c.flags & QS_F_DR) != 0;
    for (int k = 0; k < QS_PARAM_DIM; ++k)
        p7[k] = dr ? __fmul_rn(c.nominal[k], __fmaf_rn(__fsub_rn(c.dr_hi, c.dr_lo), u[k], c.dr_lo)) : c.nominal[k];
    goal[0] = __fmaf_rn(__fmul_rn(2.0f, c.room_hx), u[7], -c.room_hx);
    goal[1] = __fmaf_rn(__fmul_rn(2.0f, c.room_hy), u[8], -c.room_hy);
    goal[2] = __fmul_rn(c.room_h, u[9]);
}

// ---------------------------------------------------------------- drone state
// w + wlo is the body rate carried at about twice binary32 precision: adding
// the per-substep increment dt * dw/dt (~1e-2) onto |w| up to 40 rad/s would
// otherwise lose up to ulp(40)/2 per substep, an error that the attitude
// integrates (Kahan's compensated summation keeps the lost low-order bits).
struct Drone {
    float x[3], v[3], R[9], w[3], uf[4], eps[4], fp[4], wlo[3];
};

__device__ __forceinline__ void unpack(Drone& s, const float4 q[NPLANE]) {
    const float* f = reinterpret_cast<const float*>(q);
    for (int k = 0; k < 3; ++k) s.x[k] = f[k];
    for (int k = 0; k < 3; ++k) s.v[k] = f[3 + k];
    for (int k = 0; k < 9; ++k) s.R[k] = f[6 + k];
    for (int k = 0; k < 3; ++k) s.w[k] = f[15 + k];
    for (int k = 0; k < 4; ++k) s.uf[k] = f[18 + k];
    for (int k = 0; k < 4; ++k) s.eps[k] = f[22 + k];
    for (int k = 0; k < 4; ++k) s.fp[k] = f[26 + k];
    for (int k = 0; k < 3; ++k) s.wlo[k] = f[32 + k];
}

__device__ __forceinline__ void pack(const Drone& s, float4 q[NPLANE]) {
    float* f = reinterpret_cast<float*>(q);
    for (int k = 0; k < 3; ++k) f[k] = s.x[k];
    for (int k = 0; k < 3; ++k) f[3 + k] = s.v[k];
    for (int k = 0; k < 9; ++k) f[6 + k] = s.R[k];
    for (int k = 0; k < 3; ++k) f[15 + k] = s.w[k];
    for (int k = 0; k < 4; ++k) f[18 + k] = s.uf[k];
    for (int k = 0; k < 4; ++k) f[22 + k] = s.eps[k];
    for (int k = 0; k < 4; ++k) f[26 + k] = s.fp[k];
    f[30] = 0.0f;
    f[31] = 0.0f;
    for (int k = 0; k < 3; ++k) f[32 + k] = s.wlo[k];
    f[35] = 0.0f;
}

// ---------------------------------------------------------------- debug index checks
// The debug build (-DQS_DEBUG_CHECKS, libquadswarm_gpu_debug.so) checks the
// indices a kernel derives from its launch geometry (the env of a slot, its
// first drone and size, the slot's lanes, saved-state entries, the env of a
// drone) against the buffers they address. A failed check sets bit 1 of the
// status word (QS_ERR_INDEX at the next qs_sync) and the thread drops the work
// that would use the index, so nothing is accessed out of range and no
// barrier is skipped. The release build compiles the checks out.
constexpr int32_t STATUS_NONFINITE = 1, STATUS_INDEX = 2;
#ifdef QS_DEBUG_CHECKS
__device__ __forceinline__ bool qs_check(int32_t* status, bool ok) {
    if (!ok) atomicOr(status, STATUS_INDEX);
    return ok;
}
#else
__device__ __forceinline__ bool qs_check(int32_t*, bool) { return true; }
#endif

// ---------------------------------------------------------------- slot geometry
// A tile of `lanes` drone lanes holds lanes / W consecutive slots of the
// permutation. With uniform geometry (dv.uni_n > 0: every env has uni_n
// drones, one width class W, envs in slot order) tile i is slots
// [i per, i per + per) and env e starts at drone e uni_n, so a kernel derives
// both from its tile index instead of reading the tile table, the permutation
// and the env offsets: three dependent loads before the first state load. The
// host turns it on only after checking every tile table against this rule.
__device__ __forceinline__ Tile tile_at(const Dev& dv, const Tile* __restrict__ tiles, int i, int lanes) {
    if (dv.uni_n) {
        const int per = lanes >> dv.uni_wlog, first = i * per;
        return Tile{first, min(per, dv.E - first), 1 << dv.uni_wlog, 1};
    }
    return tiles[i];
}

// The env in slot j of the permutation.
__device__ __forceinline__ int slot_env(const Dev& dv, const int* __restrict__ perm, int j) {
    return dv.uni_n ? j : perm[j];
}

// The first drone of env e (e = E: the drone count).
__device__ __forceinline__ int env_first(const Dev& dv, int e) { return dv.uni_n ? e * dv.uni_n : dv.env_off[e]; }

// Slot `slot` of a tile: its env, first drone and size; ok when the slot
// exists (and, in the debug build, when the slot lies in the permutation, its
// env in [0, E), the env's drones in [0, D) and within the slot's W lanes,
// and the slot's lanes within the nt threads of the group).
struct SlotGeo {
    int e, d0, N;
    bool ok;
};

__device__ __forceinline__ SlotGeo slot_geometry(const Dev& dv, const int* __restrict__ perm, const Tile& tile, int slot,
                                                 int W, int nt) {
    SlotGeo g{0, 0, 0, slot < tile.count};
    if (g.ok) g.ok = qs_check(dv.status, tile.first + slot >= 0 && tile.first + slot < dv.E);
    if (g.ok) {
        g.e = slot_env(dv, perm, tile.first + slot);
        g.ok = qs_check(dv.status, g.e >= 0 && g.e < dv.E);
    }
    if (g.ok) {
        g.d0 = env_first(dv, g.e);
        g.N = env_first(dv, g.e + 1) - g.d0;
        g.ok = qs_check(dv.status,
                        g.d0 >= 0 && g.N >= 1 && g.N <= W && g.d0 + g.N <= dv.D && (slot + 1) * W <= nt);
        if (!g.ok) g.d0 = g.N = 0;
    }
    return g;
}

// The step's arithmetic is written with explicit roundings (__fmul_rn,
// __fadd_rn, __fmaf_rn): the compiler fuses a multiply and an add into one
// rounding only inside a basic block, so with implicit contraction the same
// source could round differently in the per-call, rollout, warp-specialised
// and server kernels that inline it; with explicit roundings every kernel
// gives the same bits by construction.
// a0 b0 + a1 b1 + a2 b2 as fma(a2, b2, fma(a1, b1, a0 b0)).
__device__ __forceinline__ float dot3(float a0, float a1, float a2, float b0, float b1, float b2) {
    return __fmaf_rn(a2, b2, __fmaf_rn(a1, b1, __fmul_rn(a0, b0)));
}
// a b - c d as fma(-c, d, a b).
__device__ __forceinline__ float cross_c(float a, float b, float c, float d) {
    return __fmaf_rn(-c, d, __fmul_rn(a, b));
}

// hi + lo <- hi + lo + a b, keeping the rounding error of the sum in lo
// (Kahan); the product enters with the low word in one rounding.
__device__ __forceinline__ void comp_add_prod(float& hi, float& lo, float a, float b) {
    const float y = __fmaf_rn(a, b, lo);
    const float t = __fadd_rn(hi, y);
    lo = __fsub_rn(y, __fsub_rn(t, hi));
    hi = t;
}

__device__ __forceinline__ void load_drone(Drone& s, const float4* __restrict__ st, int D, int d) {
    float4 q[NPLANE];
#pragma unroll
    for (int p = 0; p < NPLANE; ++p) q[p] = st[(size_t)p * D + d];
    unpack(s, q);
}

__device__ __forceinline__ void store_drone(const Drone& s, float4* __restrict__ st, int D, int d) {
    float4 q[NPLANE];
    pack(s, q);
#pragma unroll
    for (int p = 0; p < NPLANE; ++p) st[(size_t)p * D + d] = q[p];
}

// Initial drone state (Sec. III-A with DR): position uniform in the room,
// velocity and body rates uniform in [-1,1], orientation from a uniform unit
// quaternion (Shoemake 1992), motors at hover (u_f^2 = 1/t2w), noise zero.
__device__ __forceinline__ void draw_drone(const Consts& c, uint32_t k0, uint32_t k1, uint32_t tick, uint32_t tag,
                                           int d, float t2w, Drone& s) {
    const uint4 a = philox(tick, (uint32_t)d, ctr_word(tag, 0, 0), k0, k1);
    const uint4 b = philox(tick, (uint32_t)d, ctr_word(tag, 0, 1), k0, k1);
    const uint4 q = philox(tick, (uint32_t)d, ctr_word(tag, 0, 2), k0, k1);
    s.x[0] = __fmaf_rn(__fmul_rn(2.0f, c.room_hx), u01(a.x), -c.room_hx);
    s.x[1] = __fmaf_rn(__fmul_rn(2.0f, c.room_hy), u01(a.y), -c.room_hy);
    s.x[2] = __fmul_rn(c.room_h, u01(a.z));
    s.v[0] = __fmaf_rn(2.0f, u01(a.w), -1.0f);
    s.v[1] = __fmaf_rn(2.0f, u01(b.x), -1.0f);
    s.v[2] = __fmaf_rn(2.0f, u01(b.y), -1.0f);
    const float u6 = u01(b.z), u7 = u01(b.w), u8 = u01(q.x);
    const float ra = sqrtf(1.0f - u6), rb = sqrtf(u6);
    float s7, c7, s8, c8;
    sincospif(2.0f * u7, &s7, &c7);
    sincospif(2.0f * u8, &s8, &c8);
    const float qx = ra * s7, qy = ra * c7, qz = rb * s8, qw = rb * c8;
    s.R[0] = __fmaf_rn(-2.0f, __fmaf_rn(qz, qz, __fmul_rn(qy, qy)), 1.0f);
    s.R[1] = __fmul_rn(2.0f, cross_c(qx, qy, qz, qw));
    s.R[2] = __fmul_rn(2.0f, __fmaf_rn(qy, qw, __fmul_rn(qx, qz)));
    s.R[3] = __fmul_rn(2.0f, __fmaf_rn(qz, qw, __fmul_rn(qx, qy)));
    s.R[4] = __fmaf_rn(-2.0f, __fmaf_rn(qz, qz, __fmul_rn(qx, qx)), 1.0f);
    s.R[5] = __fmul_rn(2.0f, cross_c(qy, qz, qx, qw));
    s.R[6] = __fmul_rn(2.0f, cross_c(qx, qz, qy, qw));
    s.R[7] = __fmul_rn(2.0f, __fmaf_rn(qx, qw, __fmul_rn(qy, qz)));
    s.R[8] = __fmaf_rn(-2.0f, __fmaf_rn(qy, qy, __fmul_rn(qx, qx)), 1.0f);
    s.w[0] = -1.0f + 2.0f * u01(q.y);
    s.w[1] = -1.0f + 2.0f * u01(q.z);
    s.w[2] = -1.0f + 2.0f * u01(q.w);
    s.wlo[0] = s.wlo[1] = s.wlo[2] = 0.0f;
    const float hov = 1.0f / t2w;
    const float uh = sqrtf(hov);
    for (int r = 0; r < 4; ++r) {
        s.uf[r] = uh;
        s.eps[r] = 0.0f;
        s.fp[r] = hov;
    }
}

// ---------------------------------------------------------------- event bits
constexpr uint32_t EV_HIT_FLOOR = QS_EV_HIT_FLOOR, EV_ON_FLOOR = QS_EV_ON_FLOOR, EV_HIT_WALL = QS_EV_HIT_WALL,
                   EV_HIT_CEIL = QS_EV_HIT_CEIL, EV_HIT_QUAD = QS_EV_HIT_QUAD;

// S1 command map: clip(a, 0, 1), or (clip(a, -1, 1) + 1) / 2 (paper's form).
__device__ __forceinline__ float command(const Consts& c, float a) {
    if (c.flags & QS_F_ACTION_SYMMETRIC) return 0.5f * (fminf(fmaxf(a, -1.0f), 1.0f) + 1.0f);
    return fminf(fmaxf(a, 0.0f), 1.0f);
}

// softplus_beta(u) = log(1 + exp(beta u)) / beta. Below z = beta u = -16 it
// equals exp(z) / beta to binary32 precision (log1p(x) = x - x^2/2 + ...,
// x < 1.2e-7), which the hardware exponential gives in a few instructions;
// contact penalties far from any contact take that path.
// ib = 1 / beta (Consts::inv_beta). The smooth-contact arithmetic is written
// with explicit roundings (__fmul_rn, __fadd_rn, __fmaf_rn) so that no kernel's
// compiler fuses it differently: every kernel that steps the smooth form
// gives the same bits.
__device__ __forceinline__ float softplus_b(float u, float beta, float ib) {
    const float z = __fmul_rn(beta, u);
    if (z < -16.0f) return __fmul_rn(exp_approx(z), ib);
    return __fmul_rn(__fadd_rn(fmaxf(z, 0.0f), log1pf(exp_approx(-fabsf(z)))), ib);
}

// Pairs farther apart than 2 l + 88 / beta have softplus_beta(2 l - d) below
// exp(-88) / beta: their penalty and its derivatives vanish in binary32
// sums of order-g accelerations, so they are skipped. The squared distance
// beyond which a pair is skipped (formed once per drone, outside the pair loop):
__device__ __forceinline__ float pair_far_d2(float arm, float inv_beta) {
    const float r = 2.f * arm + 88.f * inv_beta;
    return r * r;
}

// Smooth pair acceleration of the thread's drone from the slot's positions in
// shared memory (sx[3][nt]); j == lane and coincident drones contribute 0.
__device__ __forceinline__ void pair_acc(const Consts& c, const float x[3], const float* sx, int nt, int sbase, int lane,
                                         int N, float arm, float out[3]) {
    out[0] = out[1] = out[2] = 0.f;
    const float kcg = __fmul_rn(c.kc, c.g), far2 = pair_far_d2(arm, c.inv_beta);
    for (int j = 0; j < N; ++j) {
        if (j == lane) continue;
        const int tj = sbase + j;
        const float r0 = x[0] - sx[tj], r1 = x[1] - sx[nt + tj], r2 = x[2] - sx[2 * nt + tj];
        const float d2 = __fmaf_rn(r2, r2, __fmaf_rn(r1, r1, __fmul_rn(r0, r0)));
        if (d2 == 0.f || d2 > far2) continue;
        const float d = sqrtf(d2);
        const float psi = __fmul_rn(__fmul_rn(kcg, softplus_b(__fsub_rn(2.f * arm, d), c.beta, c.inv_beta)), __frcp_rn(d));
        out[0] = fmaf(psi, r0, out[0]);
        out[1] = fmaf(psi, r1, out[1]);
        out[2] = fmaf(psi, r2, out[2]);
    }
}

// R <- polar(R + dt R [w]x) for a rotation R. In closed form the polar factor
// of I + dt [w]x is the rotation about w by atan(dt |w|), i.e.
// Q = I + a [w]x + b [w]x^2 with c = 1/sqrt(1 + dt^2 |w|^2), a = dt c,
// b = dt^2 c^2 / (1 + c); row_i(R [w]x) = row_i(R) x w. One Bjorck step
// R <- R (3I - R^T R) / 2 then removes the binary32 drift of R itself.
__device__ __forceinline__ void rotate_polar(float R[9], const float w[3], float dt) {
    const float n2 = dot3(w[0], w[1], w[2], w[0], w[1], w[2]);
    const float q = __fmaf_rn(__fmul_rn(dt, dt), n2, 1.0f);
    float cc = rsqrt_approx_ge1(q);  // q >= 1
    cc = __fmul_rn(cc, __fmaf_rn(__fmul_rn(__fmul_rn(-0.5f, q), cc), cc, 1.5f));  // one Newton step: ~1 ulp
    const float a = __fmul_rn(dt, cc);
    const float b = __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(dt, dt), cc), cc), rcp_approx(__fadd_rn(1.0f, cc)));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float r0 = R[3 * i], r1 = R[3 * i + 1], r2 = R[3 * i + 2];
        const float t0 = cross_c(r1, w[2], r2, w[1]), t1 = cross_c(r2, w[0], r0, w[2]), t2 = cross_c(r0, w[1], r1, w[0]);
        const float q0 = cross_c(t1, w[2], t2, w[1]), q1 = cross_c(t2, w[0], t0, w[2]), q2 = cross_c(t0, w[1], t1, w[0]);
        R[3 * i] = __fmaf_rn(b, q0, __fmaf_rn(a, t0, r0));
        R[3 * i + 1] = __fmaf_rn(b, q1, __fmaf_rn(a, t1, r1));
        R[3 * i + 2] = __fmaf_rn(b, q2, __fmaf_rn(a, t2, r2));
    }
    // one Bjorck step: S = R^T R; R <- R (1.5 I - 0.5 S)
    float S[6];  // 00 01 02 11 12 22
    S[0] = dot3(R[0], R[3], R[6], R[0], R[3], R[6]);
    S[1] = dot3(R[0], R[3], R[6], R[1], R[4], R[7]);
    S[2] = dot3(R[0], R[3], R[6], R[2], R[5], R[8]);
    S[3] = dot3(R[1], R[4], R[7], R[1], R[4], R[7]);
    S[4] = dot3(R[1], R[4], R[7], R[2], R[5], R[8]);
    S[5] = dot3(R[2], R[5], R[8], R[2], R[5], R[8]);
    const float A00 = __fmaf_rn(-0.5f, S[0], 1.5f), A11 = __fmaf_rn(-0.5f, S[3], 1.5f), A22 = __fmaf_rn(-0.5f, S[5], 1.5f);
    const float A01 = __fmul_rn(-0.5f, S[1]), A02 = __fmul_rn(-0.5f, S[2]), A12 = __fmul_rn(-0.5f, S[4]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float r0 = R[3 * i], r1 = R[3 * i + 1], r2 = R[3 * i + 2];
        R[3 * i] = dot3(r0, r1, r2, A00, A01, A02);
        R[3 * i + 1] = dot3(r0, r1, r2, A01, A11, A12);
        R[3 * i + 2] = dot3(r0, r1, r2, A02, A12, A22);
    }
}

// One physics substep of one drone (S1 .. S8). fh: this control step's
// normalised commands; u = sqrt(fh). pacc: smooth-mode pair acceleration
// (zero otherwise). Returns the substep's event bits.
__device__ __forceinline__ void motor_normals(const Consts& c, uint32_t tick, int d, int sub, float n[4]) {
    const uint4 q = philox_rk(tick, (uint32_t)d, ctr_word(TAG_MOTOR, (uint32_t)sub, 0), c.rk);
    const float2 n01 = box_muller(u01(q.x), u01(q.y));
    const float2 n23 = box_muller(u01(q.z), u01(q.w));
    n[0] = n01.x;
    n[1] = n01.y;
    n[2] = n23.x;
    n[3] = n23.y;
}

// nrm: this substep's four motor-noise normals when already drawn elsewhere
// (nullptr: draw them here). ET: event-time contacts (QS_F_EVENT_TIME, the
// differentiable rollout's variant): a floor, wall or ceiling contact is
// resolved at its crossing time on the substep's straight path x0 + v1 s.
// SMC: the contact form, 0 discrete, 1 smooth (QS_F_SMOOTH) or -1 read from
// the flags; a kernel that knows it compiles only that branch.
template <bool ET = false, int SMC = -1>
__device__ __forceinline__ uint32_t substep(Drone& s, const Prm& p, const Consts& c, const float u[4], uint32_t tick,
                                            int d, int sub, const float pacc[3], const float* nrm = nullptr) {
    const bool smooth = SMC < 0 ? (c.flags & QS_F_SMOOTH) != 0 : SMC > 0;
    uint32_t ev = 0;
    const float dt = c.dt, g = c.g;
    // S1 first-order motor lag on the normalised rotor speed
#pragma unroll
    for (int r = 0; r < 4; ++r) s.uf[r] = fmaf(p.alag, u[r] - s.uf[r], s.uf[r]);
    // S2 AR(1) motor noise and per-rotor thrust f = f_max uf^2 + eps
    if (c.flags & QS_F_MOTOR_NOISE) {
        float n[4];
        if (nrm) {
            n[0] = nrm[0];
            n[1] = nrm[1];
            n[2] = nrm[2];
            n[3] = nrm[3];
        } else {
            motor_normals(c, tick, d, sub, n);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) s.eps[r] = fmaf(c.alpha_nd, s.eps[r], p.ans * n[r]);
    }
    float f[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) f[r] = fmaf(p.fmax * s.uf[r], s.uf[r], s.eps[r]);
    // S3 X layout: rotors at (+-l, +-l)/sqrt(2); thrust along body z; yaw
    // torque kappa * sum s_r f_r with spins (-1, +1, -1, +1)
    const float T = (f[0] + f[1]) + (f[2] + f[3]);
    const float sa = p.arm * 0.70710678118654752f;
    const float tx = sa * ((f[0] + f[1]) - (f[2] + f[3]));
    const float ty = sa * ((f[1] + f[2]) - (f[0] + f[3]));
    const float tz = c.kappa * ((f[1] + f[3]) - (f[0] + f[2]));
    // S4 world thrust F = R (0,0,T), a = F/m + g
    const float F0 = s.R[2] * T, F1 = s.R[5] * T, F2 = s.R[8] * T;
    float a0 = F0 * p.inv_m, a1 = F1 * p.inv_m, a2 = fmaf(F2, p.inv_m, -g);
    bool on_floor = false, moving = false;
    if (smooth) {  // explicit roundings (see softplus_b)
        const float kcg = __fmul_rn(c.kc, g);
        const float b = c.beta, ib = c.inv_beta;
        const float pz = __fsub_rn(softplus_b(-s.x[2], b, ib), softplus_b(__fsub_rn(s.x[2], c.room_h), b, ib));
        const float px = __fsub_rn(softplus_b(__fsub_rn(-c.room_hx, s.x[0]), b, ib),
                                   softplus_b(__fsub_rn(s.x[0], c.room_hx), b, ib));
        const float py = __fsub_rn(softplus_b(__fsub_rn(-c.room_hy, s.x[1]), b, ib),
                                   softplus_b(__fsub_rn(s.x[1], c.room_hy), b, ib));
        a2 = __fadd_rn(__fmaf_rn(kcg, pz, a2), pacc[2]);
        a0 = __fadd_rn(__fmaf_rn(kcg, px, a0), pacc[0]);
        a1 = __fadd_rn(__fmaf_rn(kcg, py, a1), pacc[1]);
    } else if ((c.flags & QS_F_FLOOR) && s.x[2] <= 0.0f) {
        const float mg = __fmul_rn(p.m, g);
        if (F2 < mg) {
            // resting on the floor: friction mu (m g - F_z) against the motion
            on_floor = true;
            ev |= EV_ON_FLOOR;
            const float ffric = __fmul_rn(c.mu, __fsub_rn(mg, F2));
            float fx = F0, fy = F1;
            if (s.v[0] == 0.0f && s.v[1] == 0.0f) {
                const float nf = sqrtf(__fmaf_rn(fy, fy, __fmul_rn(fx, fx)));
                const float keep = nf > ffric ? __fmul_rn(__fsub_rn(nf, ffric), __frcp_rn(nf)) : 0.0f;
                fx = __fmul_rn(fx, keep);
                fy = __fmul_rn(fy, keep);
            } else {
                const float inv_nv = rsqrtf(__fmaf_rn(s.v[1], s.v[1], __fmul_rn(s.v[0], s.v[0])));
                fx = __fmaf_rn(-__fmul_rn(ffric, s.v[0]), inv_nv, fx);
                fy = __fmaf_rn(-__fmul_rn(ffric, s.v[1]), inv_nv, fy);
                moving = true;
            }
            a0 = __fmul_rn(fx, p.inv_m);
            a1 = __fmul_rn(fy, p.inv_m);
            a2 = 0.0f;
            s.v[2] = 0.0f;
        }
    }
    // S5 Euler's equation, diagonal inertia
    const float Iw0 = __fmul_rn(p.ixx, s.w[0]), Iw1 = __fmul_rn(p.iyy, s.w[1]), Iw2 = __fmul_rn(p.izz, s.w[2]);
    const float wd0 = __fmul_rn(__fsub_rn(tx, cross_c(s.w[1], Iw2, s.w[2], Iw1)), p.inv_ixx);
    const float wd1 = __fmul_rn(__fsub_rn(ty, cross_c(s.w[2], Iw0, s.w[0], Iw2)), p.inv_iyy);
    const float wd2 = __fmul_rn(__fsub_rn(tz, cross_c(s.w[0], Iw1, s.w[1], Iw0)), p.inv_izz);
    // S6 semi-implicit Euler, body rates bounded by omega_max
    const float vx0 = s.v[0], vy0 = s.v[1];
    const float x0[3] = {s.x[0], s.x[1], s.x[2]};  // substep start (event-time contacts)
    s.v[0] = fmaf(a0, dt, s.v[0]);
    s.v[1] = fmaf(a1, dt, s.v[1]);
    s.v[2] = fmaf(a2, dt, s.v[2]);
    if (on_floor && moving && __fmaf_rn(s.v[1], vy0, __fmul_rn(s.v[0], vx0)) < 0.0f) {
        s.v[0] = 0.0f;
        s.v[1] = 0.0f;
    }
    s.x[0] = fmaf(s.v[0], dt, s.x[0]);
    s.x[1] = fmaf(s.v[1], dt, s.x[1]);
    s.x[2] = fmaf(s.v[2], dt, s.x[2]);
    const float wd[3] = {wd0, wd1, wd2};
#pragma unroll
    for (int k = 0; k < 3; ++k) comp_add_prod(s.w[k], s.wlo[k], wd[k], dt);
    // body rates past omega_max are rare: one test on the largest first
    if (fmaxf(fmaxf(fabsf(s.w[0]), fabsf(s.w[1])), fabsf(s.w[2])) > c.omega_max) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (fabsf(s.w[k]) > c.omega_max) {
                s.w[k] = copysignf(c.omega_max, s.w[k]);
                s.wlo[k] = 0.0f;
            }
        }
    }
    rotate_polar(s.R, s.w, dt);

    if (smooth) {
        if (s.x[2] < 0.0f) ev |= EV_HIT_FLOOR;
        if (s.x[2] > c.room_h) ev |= EV_HIT_CEIL;
        if (fabsf(s.x[0]) > c.room_hx || fabsf(s.x[1]) > c.room_hy) ev |= EV_HIT_WALL;
        return ev;
    }
    // S7 floor hit: momenta to zero, upright attitude keeping the heading
    if ((c.flags & QS_F_FLOOR) && s.x[2] <= 0.0f && s.v[2] < 0.0f) {
        ev |= EV_HIT_FLOOR;
        if (ET) {  // crossing at tau = -z0 / v_z; at rest from then on
            const float tau = fminf(fmaxf(-x0[2] / s.v[2], 0.0f), dt);
            s.x[0] = fmaf(s.v[0], tau, x0[0]);
            s.x[1] = fmaf(s.v[1], tau, x0[1]);
        }
        s.x[2] = 0.0f;
        for (int k = 0; k < 3; ++k) {
            s.v[k] = 0.0f;
            s.w[k] = 0.0f;
            s.wlo[k] = 0.0f;
        }
        float cs, sn;
        const float h2 = __fmaf_rn(s.R[3], s.R[3], __fmul_rn(s.R[0], s.R[0]));
        if (h2 >= 1e-12f) {
            const float ih = rsqrtf(h2);
            cs = s.R[0] * ih;
            sn = s.R[3] * ih;
        } else {
            const float ih = rsqrtf(__fmaf_rn(s.R[4], s.R[4], __fmul_rn(s.R[1], s.R[1])));
            cs = s.R[4] * ih;
            sn = -s.R[1] * ih;
        }
        s.R[0] = cs; s.R[1] = -sn; s.R[2] = 0.0f;
        s.R[3] = sn; s.R[4] = cs;  s.R[5] = 0.0f;
        s.R[6] = 0.0f; s.R[7] = 0.0f; s.R[8] = 1.0f;
    }
    // S8 walls and ceiling: a drone past a boundary is put back onto it; if it
    // was moving outward its normal velocity is removed and
    // v <- alpha_c (v + eps_v), w <- w + eps_w
    // (a drone inside the room, the common case, passes one test)
    if ((c.flags & QS_F_WALLS) &&
        (fabsf(s.x[0]) > c.room_hx || fabsf(s.x[1]) > c.room_hy || s.x[2] > c.room_h)) {
        bool wall = false, ceil = false, held[3] = {false, false, false};
        const float v1[3] = {s.v[0], s.v[1], s.v[2]};
        float tau = dt;  // earliest boundary crossing (event-time contacts)
        if (s.x[0] > c.room_hx) {
            if (s.v[0] > 0.0f) { s.v[0] = 0.0f; wall = true; if (ET) tau = fminf(tau, (c.room_hx - x0[0]) / v1[0]); }
            s.x[0] = c.room_hx;
            held[0] = true;
        } else if (s.x[0] < -c.room_hx) {
            if (s.v[0] < 0.0f) { s.v[0] = 0.0f; wall = true; if (ET) tau = fminf(tau, (-c.room_hx - x0[0]) / v1[0]); }
            s.x[0] = -c.room_hx;
            held[0] = true;
        }
        if (s.x[1] > c.room_hy) {
            if (s.v[1] > 0.0f) { s.v[1] = 0.0f; wall = true; if (ET) tau = fminf(tau, (c.room_hy - x0[1]) / v1[1]); }
            s.x[1] = c.room_hy;
            held[1] = true;
        } else if (s.x[1] < -c.room_hy) {
            if (s.v[1] < 0.0f) { s.v[1] = 0.0f; wall = true; if (ET) tau = fminf(tau, (-c.room_hy - x0[1]) / v1[1]); }
            s.x[1] = -c.room_hy;
            held[1] = true;
        }
        if (s.x[2] > c.room_h) {
            if (s.v[2] > 0.0f) { s.v[2] = 0.0f; ceil = true; if (ET) tau = fminf(tau, (c.room_h - x0[2]) / v1[2]); }
            s.x[2] = c.room_h;
            held[2] = true;
        }
        if (wall || ceil) {
            float n[6];
            six_normals(c, tick, (uint32_t)d, TAG_WALL, (uint32_t)sub, n);
            for (int k = 0; k < 3; ++k) {
                s.v[k] = c.alpha_c * fmaf(c.sig_cv, n[k], s.v[k]);
                comp_add_prod(s.w[k], s.wlo[k], c.sig_cw, n[3 + k]);
            }
            if (ET) {  // pre-contact velocity until tau, post-contact for the rest
                tau = fmaxf(tau, 0.0f);
                for (int k = 0; k < 3; ++k)
                    if (!held[k]) s.x[k] = fmaf(s.v[k], dt - tau, fmaf(v1[k], tau, x0[k]));
            }
            ev |= (wall ? EV_HIT_WALL : 0u) | (ceil ? EV_HIT_CEIL : 0u);
        }
    }
    return ev;
}

// Canonical binary32 pair key |x_j - x_i|^2, evaluated without contraction in
// a fixed order so that both members of a pair, and any other implementation
// of the same sequence, obtain the same bits.
__device__ __forceinline__ float pair_key(float xi0, float xi1, float xi2, float xj0, float xj1, float xj2,
                                          float& dx, float& dy, float& dz) {
    dx = __fsub_rn(xj0, xi0);
    dy = __fsub_rn(xj1, xi1);
    dz = __fsub_rn(xj2, xi2);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Inserts cand into the ascending list best[0..K).
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

// The same with the list length KN fixed at compile time (no test of k < K).
template <int KN>
__device__ __forceinline__ void topk_insert_n(uint64_t best[QS_MAX_K], uint64_t cand) {
#pragma unroll
    for (int k = 0; k < KN; ++k) {
        if (cand < best[k]) {
            const uint64_t t = best[k];
            best[k] = cand;
            cand = t;
        }
    }
}

// Compare-exchange of two (key, index) words: a <- min, b <- max.
__device__ __forceinline__ void cmp_swap(uint64_t& a, uint64_t& b) {
    const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

// Sorts k[0..8) ascending with Floyd's 19-comparator network for 8 inputs
// (Knuth, The Art of Computer Programming vol. 3, Sec. 5.3.4), depth 6:
// the words are distinct (the low half is the partner index), so the result
// is the same order an insertion sort gives.
static_assert(QS_MAX_K == 8, "the sorting network holds QS_MAX_K words");
__device__ __forceinline__ void sort8(uint64_t k[8]) {
    cmp_swap(k[0], k[2]); cmp_swap(k[1], k[3]); cmp_swap(k[4], k[6]); cmp_swap(k[5], k[7]);
    cmp_swap(k[0], k[4]); cmp_swap(k[1], k[5]); cmp_swap(k[2], k[6]); cmp_swap(k[3], k[7]);
    cmp_swap(k[0], k[1]); cmp_swap(k[2], k[3]); cmp_swap(k[4], k[5]); cmp_swap(k[6], k[7]);
    cmp_swap(k[2], k[4]); cmp_swap(k[3], k[5]);
    cmp_swap(k[1], k[4]); cmp_swap(k[3], k[6]);
    cmp_swap(k[1], k[2]); cmp_swap(k[3], k[4]); cmp_swap(k[5], k[6]);
}

// One partner j of the pair pass: its canonical key |x_j - x_i|^2, the
// collision flag and Jacobi term (S9, S10) and the downwash term (S10b).
__device__ __forceinline__ float pair_partner(const Consts& c, const Drone& s, float thr, int tj, const float* sx,
                                              const float* sv, int nt, bool coll, bool flag_coll, uint32_t& ev,
                                              float dvs[3], const bool dw, float& dw_az, bool& dw_hit,
                                              bool& responded) {
    float dx, dy, dz;
    const float key = pair_key(s.x[0], s.x[1], s.x[2], sx[tj], sx[nt + tj], sx[2 * nt + tj], dx, dy, dz);
    // downwash: j overlaps this drone from above (horizontal distance below
    // l_i + l_j, height difference in (0, dw_h))
    if (dw && __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) < thr && dz > 0.0f && dz < c.dw_h) {
        dw_az = __fmaf_rn(-c.dw_k1, __fmaf_rn(c.dw_k2, dz, c.dw_b1), dw_az);
        dw_hit = true;
    }
    if (flag_coll && key < thr) {
        ev |= EV_HIT_QUAD;
        if (coll) {
            // approaching iff (v_i - v_j) . (x_i - x_j) < 0
            const float rv0 = s.v[0] - sv[tj], rv1 = s.v[1] - sv[nt + tj], rv2 = s.v[2] - sv[2 * nt + tj];
            const float app = -dot3(rv0, rv1, rv2, dx, dy, dz);
            if (app < 0.0f) {
                float n0 = 0.f, n1 = 0.f, n2 = 1.f;
                if (key > 0.0f) {
                    const float inv = rsqrtf(key);
                    n0 = -dx * inv;
                    n1 = -dy * inv;
                    n2 = -dz * inv;
                }
                const float vn = -dot3(rv0, rv1, rv2, n0, n1, n2);  // (v_j - v_i) . n
                dvs[0] = fmaf(vn, n0, dvs[0]);
                dvs[1] = fmaf(vn, n1, dvs[1]);
                dvs[2] = fmaf(vn, n2, dvs[2]);
                responded = true;
            }
        }
    }
    return key;
}

// S9 + S11 for the thread's drone (slot-local index `lane`) against the slot's
// staged positions / pre-collision velocities (planes of stride nt): collision
// flag, the Jacobi sum of ((v_j - v_i).n) n over colliding approaching
// partners (S10), and the sorted neighbour list. Swarms of at most 8 (width
// classes up to 8, so the test is uniform over a tile) keep every partner's
// (key, index) word in registers and sort them with a network of 19
// compare-exchanges; larger swarms insert each partner into the list of the
// K nearest so far (with K = 6 a list of compile-time length).
__device__ __forceinline__ bool pair_scan(const Consts& c, const Drone& s, float thr, int lane, int N, int sbase,
                                          const float* sx, const float* sv, int nt, int keff, bool coll, bool flag_coll,
                                          uint32_t& ev, uint64_t best[QS_MAX_K], float dvs[3], const bool dw,
                                          float& dw_az, bool& dw_hit) {
    bool responded = false;
    if (N <= 8) {
        uint64_t kk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            kk[j] = ~0ull;
            if (j < N && j != lane) {
                const float key = pair_partner(c, s, thr, sbase + j, sx, sv, nt, coll, flag_coll, ev, dvs, dw, dw_az,
                                               dw_hit, responded);
                kk[j] = ((uint64_t)__float_as_uint(key) << 32) | (uint32_t)j;
            }
        }
        if (keff > 0) {
            sort8(kk);
#pragma unroll
            for (int k = 0; k < QS_MAX_K; ++k) best[k] = k < keff ? kk[k] : ~0ull;
        }
        return responded;
    }
    if (keff == 6) {  // the paper's K (N > 8 here, so keff = K): the list length fixed
        for (int j = 0; j < N; ++j) {
            if (j == lane) continue;
            const float key = pair_partner(c, s, thr, sbase + j, sx, sv, nt, coll, flag_coll, ev, dvs, dw, dw_az,
                                           dw_hit, responded);
            topk_insert_n<6>(best, ((uint64_t)__float_as_uint(key) << 32) | (uint32_t)j);
        }
        return responded;
    }
    for (int j = 0; j < N; ++j) {
        if (j == lane) continue;
        const float key = pair_partner(c, s, thr, sbase + j, sx, sv, nt, coll, flag_coll, ev, dvs, dw, dw_az, dw_hit,
                                       responded);
        if (keff > 0) topk_insert(best, keff, ((uint64_t)__float_as_uint(key) << 32) | (uint32_t)j);
    }
    return responded;
}

// S10: v <- alpha_c (v + sum + eps_v), w <- w + eps_w for a responding drone.
__device__ __forceinline__ void apply_response(const Consts& c, Drone& s, uint32_t tick, int d, const float dvs[3]) {
    float n[6];
    six_normals(c, tick, (uint32_t)d, TAG_COLL, 0, n);
    s.v[0] = __fmul_rn(c.alpha_c, __fmaf_rn(c.sig_cv, n[0], __fadd_rn(s.v[0], dvs[0])));
    s.v[1] = __fmul_rn(c.alpha_c, __fmaf_rn(c.sig_cv, n[1], __fadd_rn(s.v[1], dvs[1])));
    s.v[2] = __fmul_rn(c.alpha_c, __fmaf_rn(c.sig_cv, n[2], __fadd_rn(s.v[2], dvs[2])));
    comp_add_prod(s.w[0], s.wlo[0], c.sig_cw, n[3]);
    comp_add_prod(s.w[1], s.wlo[1], c.sig_cw, n[4]);
    comp_add_prod(s.w[2], s.wlo[2], c.sig_cw, n[5]);
}

// Sensor noise of the observation (Sec. III-C): U(-s,s) on x and v, N(0,s^2)
// on w; three Philox blocks of the OBS stream, substream `sub`.
__device__ __forceinline__ void obs_noise(const Consts& c, uint32_t tick, int d, uint32_t sub, float ex[3], float ev[3],
                                          float ew[3]) {
    const uint4 a = philox_rk(tick, (uint32_t)d, ctr_word(TAG_OBS, sub, 0), c.rk);
    const uint4 b = philox_rk(tick, (uint32_t)d, ctr_word(TAG_OBS, sub, 1), c.rk);
    const uint4 q = philox_rk(tick, (uint32_t)d, ctr_word(TAG_OBS, sub, 2), c.rk);
    ex[0] = (2.0f * u01(a.x) - 1.0f) * c.obs_sx;
    ex[1] = (2.0f * u01(a.y) - 1.0f) * c.obs_sx;
    ex[2] = (2.0f * u01(a.z) - 1.0f) * c.obs_sx;
    ev[0] = (2.0f * u01(a.w) - 1.0f) * c.obs_sv;
    ev[1] = (2.0f * u01(b.x) - 1.0f) * c.obs_sv;
    ev[2] = (2.0f * u01(b.y) - 1.0f) * c.obs_sv;
    const float2 n01 = box_muller(u01(b.z), u01(b.w));
    const float2 n2 = box_muller(u01(q.x), u01(q.y));
    ew[0] = n01.x * c.obs_sw;
    ew[1] = n01.y * c.obs_sw;
    ew[2] = n2.x * c.obs_sw;
}

// Every state component feeds the position within a substep (motor state ->
// thrust -> acceleration -> velocity -> position; rotation -> thrust
// direction) and the body rates feed the rotation, so a non-finite value
// anywhere shows up in x or w by the end of the control step.
__device__ __forceinline__ bool finite_state(const Drone& s) {
    return isfinite((s.x[0] + s.x[1]) + (s.x[2] + s.w[0]) + (s.w[1] + s.w[2]));
}

}  // namespace qsk
