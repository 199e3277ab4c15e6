// qs_scenario.cuh -- training scenarios (Sec. III-D) on the device.
//
// Each env carries a scenario record drawn at every reset: the scenario type
// (uniform over the handle's enabled set), two goal formations, the step at
// which a dynamic scenario switches, two centres (or the Lissajous
// amplitudes), Lissajous frequencies and phases, and a 32-bit seed for the
// evader's waypoints and the swap permutation. The goal of every drone at any
// control step is a closed-form function of the record, the drone's index in
// its swarm, the swarm size and the step, so the step kernel evaluates it in
// registers and no per-drone goal array exists.
//
// Records are double-buffered per env ([2][QS_NSCN][E] planes, selector
// scn_sel[e]): an auto-reset writes the next episode's record into the other
// buffer, so lanes of the same env that are still evaluating the terminal
// step's goal never read a half-written record.
#pragma once
#include "qs_device.cuh"

namespace qsk {

// floor(top24(r) * n / 2^24): an exact uniform integer choice in [0, n).
__device__ __forceinline__ uint32_t pick(uint32_t r, uint32_t n) {
    return (uint32_t)(((uint64_t)(r >> 8) * n) >> 24);
}

// Smallest m >= 1 with m^2 >= n (p = 2) or m^3 >= n (p = 3), n <= 2^16.
__device__ __forceinline__ int root_ceil(int n, int p) {
    const float x = (float)n;
    int m = (int)(p == 2 ? sqrtf(x) : cbrtf(x));
    m = max(m, 1);
    while ((p == 2 ? m * m : m * m * m) < n) ++m;
    while (m > 1 && (p == 2 ? (m - 1) * (m - 1) : (m - 1) * (m - 1) * (m - 1)) >= n) --m;
    return m;
}

// Offset from the formation's centre of goal slot k (0 <= k < n) of a
// formation of n goals with spacing s (QS_FORM_*):
//   circle    n goals evenly on a horizontal circle of radius min(s n / 2 pi, rmax);
//   grid      a horizontal square grid of side ceil(sqrt n), filled row by row,
//             centred on its occupied rows;
//   sphere    the Fibonacci lattice: heights 1 - (2k+1)/n, azimuth advancing by
//             the golden angle, radius s sqrt(n / 4 pi) (area s^2 per goal);
//   cylinder  L rings (L the smallest with 4 L^2 >= n) of ceil(n / L) goals,
//             each ring's radius that of a circle of that many goals, rings s
//             apart and centred on the occupied ones;
//   cube      a cubic grid of side ceil(cbrt n) filled along x, y, then z,
//             centred on its occupied layers.
__device__ __forceinline__ void formation_offset(const Consts& c, int form, int k, int n, float s, float out[3]) {
    out[0] = out[1] = out[2] = 0.0f;
    if (form == QS_FORM_CIRCLE) {
        const float r = fminf(s * (float)n * 0.159154943091895336f, c.form_rmax);
        float sn, cs;
        sincospif(2.0f * (float)k / (float)n, &sn, &cs);
        out[0] = r * cs;
        out[1] = r * sn;
    } else if (form == QS_FORM_GRID) {
        const int m = root_ceil(n, 2), rows = (n + m - 1) / m;
        const int row = k / m;
        out[0] = s * ((float)(k - row * m) - 0.5f * (float)(m - 1));
        out[1] = s * ((float)row - 0.5f * (float)(rows - 1));
    } else if (form == QS_FORM_SPHERE) {
        const float r = s * sqrtf((float)n * 0.0795774715459476679f);
        const float a = (float)(2 * k + 1) / (float)n;  // 1 - z
        const float rho = sqrtf(a * (2.0f - a));         // sqrt(1 - z^2) without cancellation
        const uint32_t turn = (uint32_t)k * c.golden_q32;  // modulo 2^32 = one turn
        float sn, cs;
        sincospif(2.0f * ((float)turn * 2.3283064365386963e-10f), &sn, &cs);
        out[0] = r * rho * cs;
        out[1] = r * rho * sn;
        out[2] = r * (1.0f - a);
    } else if (form == QS_FORM_CYLINDER) {
        int L = max(1, (int)(0.5f * sqrtf((float)n)));
        while (4 * L * L < n) ++L;
        while (L > 1 && 4 * (L - 1) * (L - 1) >= n) --L;
        const int m = (n + L - 1) / L, used = (n + m - 1) / m;
        const int layer = k / m, idx = k - layer * m;
        const float r = fminf(s * (float)m * 0.159154943091895336f, c.form_rmax);
        float sn, cs;
        sincospif(2.0f * (float)idx / (float)m, &sn, &cs);
        out[0] = r * cs;
        out[1] = r * sn;
        out[2] = s * ((float)layer - 0.5f * (float)(used - 1));
    } else if (form == QS_FORM_CUBE) {
        const int m = root_ceil(n, 3), m2 = m * m, layers = (n + m2 - 1) / m2;
        const int l = k / m2, rem = k - l * m2, j = rem / m, i = rem - j * m;
        out[0] = s * ((float)i - 0.5f * (float)(m - 1));
        out[1] = s * ((float)j - 0.5f * (float)(m - 1));
        out[2] = s * ((float)l - 0.5f * (float)(layers - 1));
    }
}

// A coordinate uniform in [-h + m, h - m] (a room half-width h, clearance m)
// and a height uniform in [m, h - m], with explicit roundings so that every
// kernel that draws a record gives the same bits.
__device__ __forceinline__ float in_box(float h, float m, float u) {
    return __fmaf_rn(__fmul_rn(2.0f, __fsub_rn(h, m)), u, __fadd_rn(-h, m));
}
__device__ __forceinline__ float in_height(float h, float m, float u) {
    return __fmaf_rn(__fsub_rn(h, __fmul_rn(2.0f, m)), u, m);
}

// Scenario record of env e after a reset: five Philox blocks at (tick, e,
// tag << 16 | block) under key (k0, k1). Type uniform over the enabled ones;
// formations uniform over the five; switch step uniform in [T/4, 3T/4] (T the
// episode length, at least 1); centres uniform in the room shrunk by the
// clearance on every face; Lissajous centre within 1 m per axis of the room's
// middle, amplitudes U(0.5, 1) times the half-extent the clearance leaves,
// frequencies U(0.5, 1.5) times the base, phases U(0, 1) turns. With only the
// single goal enabled the record is all zero.
__device__ __forceinline__ void draw_scenario(const Consts& c, uint32_t k0, uint32_t k1, uint32_t tick, uint32_t tag,
                                              int e, float rec[QS_NSCN]) {
#pragma unroll
    for (int k = 0; k < QS_NSCN; ++k) rec[k] = 0.0f;
    const uint32_t mask = c.scn_mask;
    if ((mask & ~1u) == 0u) return;
    const uint4 b0 = philox(tick, (uint32_t)e, (tag << 16) | 0u, k0, k1);
    const uint4 b1 = philox(tick, (uint32_t)e, (tag << 16) | 1u, k0, k1);
    const uint4 b2 = philox(tick, (uint32_t)e, (tag << 16) | 2u, k0, k1);
    uint32_t idx = pick(b0.x, (uint32_t)__popc(mask));
    int type = 0;
    for (int t = 0; t < QS_NSCN_TYPES; ++t) {
        if (!((mask >> t) & 1u)) continue;
        if (idx == 0u) {
            type = t;
            break;
        }
        --idx;
    }
    rec[QS_R_TYPE] = (float)type;
    rec[QS_R_F0] = (float)pick(b0.y, QS_NFORM);
    rec[QS_R_F1] = (float)pick(b0.z, QS_NFORM);
    int lo = c.episode_steps / 4, hi = 3 * c.episode_steps / 4;
    lo = max(lo, 1);
    hi = max(hi, lo);
    rec[QS_R_TSW] = (float)(lo + (int)pick(b0.w, (uint32_t)(hi - lo + 1)));
    rec[QS_R_SEED_LO] = (float)(b1.w & 0xffffu);
    rec[QS_R_SEED_HI] = (float)(b1.w >> 16);
    const float m = c.scn_m, hx = c.room_hx, hy = c.room_hy, hz = c.room_h;
    if (type == QS_SCN_PURSUIT_LISSAJOUS) {
        const uint4 b3 = philox(tick, (uint32_t)e, (tag << 16) | 3u, k0, k1);
        const uint4 b4 = philox(tick, (uint32_t)e, (tag << 16) | 4u, k0, k1);
        rec[QS_R_C0 + 0] = -1.0f + 2.0f * u01(b1.x);
        rec[QS_R_C0 + 1] = -1.0f + 2.0f * u01(b1.y);
        rec[QS_R_C0 + 2] = 0.5f * hz - 1.0f + 2.0f * u01(b1.z);
        rec[QS_R_C1 + 0] = (hx - m) * (0.5f + 0.5f * u01(b2.x));
        rec[QS_R_C1 + 1] = (hy - m) * (0.5f + 0.5f * u01(b2.y));
        rec[QS_R_C1 + 2] = (0.5f * hz - m) * (0.5f + 0.5f * u01(b2.z));
        rec[QS_R_FREQ + 0] = c.liss_f * (0.5f + u01(b3.x));
        rec[QS_R_FREQ + 1] = c.liss_f * (0.5f + u01(b3.y));
        rec[QS_R_FREQ + 2] = c.liss_f * (0.5f + u01(b3.z));
        rec[QS_R_PHASE + 0] = u01(b4.x);
        rec[QS_R_PHASE + 1] = u01(b4.y);
        rec[QS_R_PHASE + 2] = u01(b4.z);
    } else {
        rec[QS_R_C0 + 0] = in_box(hx, m, u01(b1.x));
        rec[QS_R_C0 + 1] = in_box(hy, m, u01(b1.y));
        rec[QS_R_C0 + 2] = in_height(hz, m, u01(b1.z));
        rec[QS_R_C1 + 0] = in_box(hx, m, u01(b2.x));
        rec[QS_R_C1 + 1] = in_box(hy, m, u01(b2.y));
        rec[QS_R_C1 + 2] = in_height(hz, m, u01(b2.z));
    }
}

// Writes rec into buffer `sel` of env e's record planes.
__device__ __forceinline__ void store_scenario(const Dev& dv, int sel, int e, const float rec[QS_NSCN]) {
    float* base = dv.scn + (size_t)sel * QS_NSCN * dv.E + e;
#pragma unroll
    for (int k = 0; k < QS_NSCN; ++k) base[(size_t)k * dv.E] = rec[k];
}

// Plane k of env e's active record (a plain load: the record may have been
// written earlier in the same launch by another thread of the CTA).
__device__ __forceinline__ float scn_at(const Dev& dv, int sel, int e, int k) {
    return dv.scn[((size_t)sel * QS_NSCN + k) * dv.E + e];
}

__device__ __forceinline__ uint32_t scn_seed(const Dev& dv, int sel, int e) {
    return (uint32_t)scn_at(dv, sel, e, QS_R_SEED_LO) | ((uint32_t)scn_at(dv, sel, e, QS_R_SEED_HI) << 16);
}

// Swap key of drone slot j: first word of the Philox block at (seed, j, SWAP << 16).
__device__ __forceinline__ uint32_t swap_key(const Consts& c, uint32_t seed, int j) {
    return philox_rk(seed, (uint32_t)j, TAG_SWAP << 16, c.rk).x;
}

// Evader waypoint j >= -1, uniform in the room shrunk by the clearance.
__device__ __forceinline__ void waypoint(const Consts& c, uint32_t seed, int j, float w[3]) {
    const uint4 r = philox_rk(seed, (uint32_t)(j + 1), TAG_WAYPOINT << 16, c.rk);
    const float m = c.scn_m;
    w[0] = in_box(c.room_hx, m, u01(r.x));
    w[1] = in_box(c.room_hy, m, u01(r.y));
    w[2] = in_height(c.room_h, m, u01(r.z));
}

// True when env e's drones need the swap permutation at step tau.
__device__ __forceinline__ bool swap_active(const Dev& dv, int sel, int e, int tau) {
    return (int)scn_at(dv, sel, e, QS_R_TYPE) == QS_SCN_SWAP && tau >= (int)scn_at(dv, sel, e, QS_R_TSW);
}

// Goal of local drone i (of N) of env e at control step tau of its episode
// (single goal: the env's goal genv). `slot` is the drone's goal slot after a
// swap (the rank of its swap key among the env's keys, ties to the lower
// index); it is read only by an active swap.
//   static          formation F0 around centre 0
//   dynamic goals   from the switch step on, formation F1 around centre 1
//   swap goals      from the switch step on, drone i takes goal slot `slot`
//   shrink/expand   F0 scaled by 1 - (1 - se_min)(1 - cos(2 pi tau / P)) / 2
//   swarm vs swarm  the first ceil(N/2) drones are group 0, the rest group 1,
//                   each a formation of its own size: group g around centre g
//                   in F0, from the switch step on around the other centre in F1
//   Lissajous       c + A sin(2 pi (f tau T + phase)) per axis, T = substeps dt
//   Bezier          through the waypoints, one per S control steps: on segment
//                   q = floor(tau / S) the cubic from W_q to W_q+1 with inner
//                   control points W_q + (W_q+1 - W_q-1)/6 and
//                   W_q+1 - (W_q+2 - W_q)/6, at u = (tau - qS)/S
__device__ __forceinline__ void scenario_goal(const Consts& c, const Dev& dv, int sel, int e, int i, int N, int tau,
                                              int slot, const float genv[3], float g[3]) {
    const int type = (int)scn_at(dv, sel, e, QS_R_TYPE);
    if (type == QS_SCN_SINGLE || type >= QS_NSCN_TYPES) {
        g[0] = genv[0];
        g[1] = genv[1];
        g[2] = genv[2];
        return;
    }
    const bool sw = tau >= (int)scn_at(dv, sel, e, QS_R_TSW);
    if (type == QS_SCN_PURSUIT_LISSAJOUS) {
        const float T = c.dt * (float)c.substeps;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float fT = scn_at(dv, sel, e, QS_R_FREQ + k) * T;
            const float p = fmaf(fT, (float)tau, scn_at(dv, sel, e, QS_R_PHASE + k));
            g[k] = fmaf(scn_at(dv, sel, e, QS_R_C1 + k), sinpif(2.0f * (p - floorf(p))), scn_at(dv, sel, e, QS_R_C0 + k));
        }
        return;
    }
    if (type == QS_SCN_PURSUIT_BEZIER) {
        const int S = c.bez_seg, q = tau / S;
        const float u = (float)(tau - q * S) / (float)S, v = 1.0f - u;
        const uint32_t seed = scn_seed(dv, sel, e);
        float wm[3], w0[3], w1[3], w2[3];
        waypoint(c, seed, q - 1, wm);
        waypoint(c, seed, q, w0);
        waypoint(c, seed, q + 1, w1);
        waypoint(c, seed, q + 2, w2);
        const float b0 = __fmul_rn(__fmul_rn(v, v), v), b1 = __fmul_rn(__fmul_rn(__fmul_rn(3.0f, v), v), u),
                    b2 = __fmul_rn(__fmul_rn(__fmul_rn(3.0f, v), u), u), b3 = __fmul_rn(__fmul_rn(u, u), u);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float p1 = __fmaf_rn(__fsub_rn(w1[k], wm[k]), 1.0f / 6.0f, w0[k]);
            const float p2 = __fmaf_rn(-__fsub_rn(w2[k], w0[k]), 1.0f / 6.0f, w1[k]);
            g[k] = __fmaf_rn(b3, w1[k], __fmaf_rn(b2, p2, __fmaf_rn(b1, p1, __fmul_rn(b0, w0[k]))));
        }
        return;
    }
    // formations
    int form = (int)scn_at(dv, sel, e, QS_R_F0), k = i, n = N, cen = QS_R_C0;
    float lam = 1.0f;
    if (type == QS_SCN_DYNAMIC && sw) {
        form = (int)scn_at(dv, sel, e, QS_R_F1);
        cen = QS_R_C1;
    } else if (type == QS_SCN_SWAP && sw) {
        k = slot;
    } else if (type == QS_SCN_SHRINK_EXPAND) {
        lam = __fmaf_rn(-__fmul_rn(__fsub_rn(1.0f, c.se_min), 0.5f), __fsub_rn(1.0f, cospif(2.0f * (float)tau / c.se_period)),
                        1.0f);
    } else if (type == QS_SCN_SWARM_VS_SWARM) {
        const int n0 = (N + 1) >> 1, grp = i >= n0 ? 1 : 0;
        k = i - grp * n0;
        n = grp ? N - n0 : n0;
        if (sw) form = (int)scn_at(dv, sel, e, QS_R_F1);
        cen = (grp ^ (sw ? 1 : 0)) ? QS_R_C1 : QS_R_C0;
    }
    float off[3];
    formation_offset(c, form, k, n, c.form_s, off);
#pragma unroll
    for (int q = 0; q < 3; ++q) g[q] = fmaf(lam, off[q], scn_at(dv, sel, e, cen + q));
}

// A drone's goal carried in registers across the steps of a rollout, valid
// for episode steps from <= tau < until (until = -1: empty). Static goals hold
// for the whole episode; dynamic, swap and swarm-vs-swarm goals before and
// from the switch step; the moving ones (shrink & expand, pursuit) for one
// step. Keeps the per-step goal work, which diverges across the envs of a
// warp, to the steps where a goal changes.
struct GoalCache {
    float g[3];
    int from, until;
};

__device__ __forceinline__ bool goal_cached(const GoalCache& gc, int tau) { return tau >= gc.from && tau < gc.until; }

__device__ __forceinline__ void goal_cache_set(GoalCache& gc, const Dev& dv, int sel, int e, int tau, const float g[3]) {
    const int type = (int)scn_at(dv, sel, e, QS_R_TYPE);
    const int tsw = (int)scn_at(dv, sel, e, QS_R_TSW);
    int from = tau, until = tau + 1;
    if (type == QS_SCN_SINGLE || type == QS_SCN_STATIC || type >= QS_NSCN_TYPES) {
        from = 0;
        until = 0x7fffffff;
    } else if (type == QS_SCN_DYNAMIC || type == QS_SCN_SWAP || type == QS_SCN_SWARM_VS_SWARM) {
        from = tau < tsw ? 0 : tsw;
        until = tau < tsw ? tsw : 0x7fffffff;
    }
    gc.g[0] = g[0];
    gc.g[1] = g[1];
    gc.g[2] = g[2];
    gc.from = from;
    gc.until = until;
}

}  // namespace qsk
