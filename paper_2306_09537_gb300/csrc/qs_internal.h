// qs_internal.h -- host/device shared definitions of libquadswarm_gpu.so.
// Not part of the public ABI (include/qs.h is).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "qs.h"

namespace qsk {

// Per-env parameter planes in device memory, [NPRM_DEV][E] (plane-major so
// that consecutive single-drone envs read them coalesced).
enum PrmIdx {
    P_M, P_IXX, P_IYY, P_IZZ, P_T2W, P_TAU, P_ARM,  // the 7 randomised values
    P_FMAX, P_ALAG, P_ANS, P_INVM, P_INVIXX, P_INVIYY, P_INVIZZ, P_THR, P_PROX,
    NPRM_DEV
};

// Philox stream tags (counter word 2 = tag << 16 | substream << 8 | block).
enum Tag : uint32_t {
    TAG_RESET_ENV = 1, TAG_RESET_DRONE = 2, TAG_MOTOR = 3, TAG_OBS = 4, TAG_COLL = 5, TAG_WALL = 6,
    TAG_AUTO_ENV = 7, TAG_AUTO_DRONE = 8, TAG_DOWNWASH = 9, TAG_SCN = 10, TAG_AUTO_SCN = 11, TAG_WAYPOINT = 12,
    TAG_SWAP = 13
};

// Number of float4 planes of the drone state: the 30 public floats fill
// planes 0..7 (2 pad); plane 8 holds the low-order parts of the body rates
// (compensated accumulation, see Drone::wlo) and 1 pad.
constexpr int NPLANE = 9;
constexpr int NPLANE_PUBLIC = 8;

// Model constants, passed by value to every kernel.
struct Consts {
    float dt, g, kappa, mu, alpha_nd, alpha_c, sig_cv, sig_cw;
    float obs_sx, obs_sv, obs_sw;
    float room_hx, room_hy, room_h;
    float beta, kc, omega_max, ans_frac, prox_factor, dr_lo, dr_hi;
    float inv_beta;  // 1 / beta, rounded once on the host
    float dw_k1, dw_k2, dw_b1, dw_h, dw_sa, dw_sw;  // downwash
    // scenarios: enabled mask, goal spacing, circle radius cap, clearance,
    // shrink/expand minimum and period, Lissajous base frequency, Bezier
    // segment steps, golden angle as a 32-bit turn fraction
    uint32_t scn_mask;
    float form_s, form_rmax, scn_m, se_min, se_period, liss_f;
    int bez_seg;
    uint32_t golden_q32;
    float nominal[QS_PARAM_DIM];
    float w[QS_NW];
    uint32_t flags, key0, key1;
    uint32_t rk[20];  // Philox round keys (k0, k1) of rounds 0..9 for key (key0, key1)
    int substeps, K, episode_steps, obs_dim;
};

// Whether a handle runs the general instance of the step kernels (scenario
// goals, downwash or smooth contacts, each decided at run time) rather than
// the common one that compiles them out.
inline bool extended_instance(const Consts& c) {
    return (c.scn_mask & ~1u) != 0 || (c.flags & (QS_F_DOWNWASH | QS_F_SMOOTH)) != 0;
}

// Fills c.rk from c.key0 / c.key1 (Weyl increments 0x9E3779B9, 0xBB67AE85).
inline void set_round_keys(Consts& c) {
    uint32_t k0 = c.key0, k1 = c.key1;
    for (int r = 0; r < 10; ++r) {
        c.rk[2 * r] = k0;
        c.rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Device buffers owned by a handle.
struct Dev {
    float4* st;              // [NPLANE][D] drone state planes
    float* prm;              // [NPRM_DEV][E]
    float* goal;             // [3][E]
    int32_t* ep;             // [E] control steps into the episode
    uint32_t* tick;          // [E] Philox step counter
    const int32_t* env_off;  // [E+1]
    const int32_t* env_of;   // [D]
    uint32_t* ev;            // [D] event bits of the last step
    int16_t* knn;            // [K][D] neighbour local indices (QS_F_RECORD_KNN)
    int32_t* status;         // device error word (bit 0: non-finite state; bit 1: a debug-build index check failed)
    float* scn;              // [2][QS_NSCN][E] scenario records, double-buffered (null: single goal only)
    uint8_t* scn_sel;        // [E] active buffer of each env's record
    int D, E;
    // uniform geometry (every env uni_n drones, width class 1 << uni_wlog, slots
    // in env order): tiles, envs and first drones follow from the tile index
    // (tile_at); 0 when the swarm sizes differ
    int uni_n = 0, uni_wlog = 0;
};

// A launch covers "tiles": consecutive slots (envs of one width class W) of
// the permutation `perm`; a tile is one CTA of `block` threads = block / W slots.
struct Tile {
    int first;  // first slot (index into perm)
    int count;  // slots in this tile
    int W;      // width class of its slots
    int pad;    // 1: the tile's envs are consecutive, so its drones are contiguous
};

struct ClassPlan {
    int W;         // lanes per env slot (power of two >= N of its envs)
    int block;     // threads per CTA (32 drone lanes per tile when ws)
    int ws;        // warp-specialised per-call step (W <= 32)
    int n_tiles;
    int tile_off;  // offset of this class's tiles in the tile array
};

// Per-step input/output pointers; strides let one call address step t of a
// [T][...] rollout buffer.
struct StepIO {
    const float* act;  // [D][4]
    float* obs;        // [D][obs_dim] or null
    float* rew;        // [D] or null
    uint8_t* done;     // [E] or null
};

// [T][...] buffers of a rollout (outputs nullable).
struct RolloutIO {
    const float* act;  // [T][D][4]
    float* obs;        // [T][D][obs_dim]
    float* rew;        // [T][D]
    uint8_t* done;     // [T][E]
};

// kernels (qs_step.cu)
cudaError_t launch_step(const Consts& c, const Dev& dv, const ClassPlan& cp, const Tile* tiles, const int* perm,
                        const StepIO& io, int observe_only, cudaStream_t s);
// Persistent launch over n_tiles tiles (any classes) of `block` threads;
// steps t0 .. t0+nsteps-1 of the io buffers. grid <= 0: one CTA per tile.
// single: every env of the handle holds one drone (the single-drone instance).
cudaError_t launch_rollout(const Consts& c, const Dev& dv, const Tile* tiles, int n_tiles, int block, const int* perm,
                           int* counter, const RolloutIO& io, int t0, int nsteps, int grid, bool single,
                           cudaStream_t s);
// Warp-specialised rollout: one CTA of 64P threads per tile of 32P drone
// lanes, P = 1 (every class at most 32 wide) or 2 (at most 64 wide).
cudaError_t launch_rollout_ws(const Consts& c, const Dev& dv, const Tile* tiles, int n_tiles, int P, const int* perm,
                              const RolloutIO& io, int t0, int nsteps, cudaStream_t s);
// Resident step server (k_serve): commands, outputs and the handshake words
// live in page-locked host memory mapped into the device. Codes of the go
// word besides a step count: the host ends the launch; the server retired.
constexpr int SERVE_STOP = -1, SERVE_IDLE = -2;
struct ServeIO {
    const float* act;            // [n_slots][D][4]
    float* obs;                  // [D][obs_dim] or null
    float* rew;                  // [D] or null
    uint8_t* done;               // [E] or null
    unsigned long long* go;      // low half: steps posted by the host (or a stop code); high half: command slot
    int* fin;                    // steps completed
    unsigned long long* count;   // device: CTAs finished since the launch began
    unsigned long long* relay;   // device: the value of go CTA 0 last acted on
    int n_slots;
    long long idle_ns;           // the server retires after this long without a posted step
};
// One cooperative launch of n_tiles warp-specialised CTAs (64P threads) that
// runs global steps k0, k0 + 1, ... as the host posts them.
cudaError_t launch_serve(const Consts& c, const Dev& dv, const Tile* tiles, int n_tiles, int P, const int* perm,
                         const ServeIO& io, int k0, cudaStream_t s);
// CTAs of the server the device keeps resident at once.
int serve_resident_ctas(const Consts& c, int P);
// CTAs of the warp-specialised rollout (64P threads) the device keeps
// resident at once.
int rollout_ws_resident_ctas(const Consts& c, int P);
// CTAs of `block` threads the device keeps resident at once for the k_rollout
// instance launch_rollout picks (extended: extended_instance(); single: one
// drone per env).
int rollout_grid(int block, bool extended, bool single);

// differentiable rollout (qs_adjoint.cu)
size_t diff_workspace_bytes(int D, int T, int C, int substeps);
cudaError_t launch_diff(int backward, const Consts& c, const Dev& dv, const Tile* tiles, int n_tiles, int block,
                        const int* perm, const float* x0, const float* act, float* loss, const float* dloss,
                        float* grad_act, float* grad_x0, void* workspace, int T, int C, cudaStream_t s);

// kernels (qs_kernels.cu)
// out [n][4] = Philox4x32-10 of ctr [n][3] (word 3 zero) under (key0, key1);
// variant 0: precomputed round keys, 1: inline key schedule.
cudaError_t launch_philox(const uint32_t* ctr, uint32_t key0, uint32_t key1, int variant, uint32_t* out, long long n,
                          cudaStream_t s);
cudaError_t launch_reset(const Consts& c, const Dev& dv, uint32_t key0, uint32_t key1, const uint8_t* mask,
                         cudaStream_t s);
cudaError_t launch_get_state(const Dev& dv, float* state, float* params, float* goals, int32_t* ep,
                             uint32_t* tick, cudaStream_t s);
cudaError_t launch_set_state(const Consts& c, const Dev& dv, const float* state, const float* params,
                             const float* goals, const int32_t* ep, const uint32_t* tick, cudaStream_t s);
cudaError_t launch_get_events(const Dev& dv, int K, uint32_t* events, int16_t* knn, cudaStream_t s);
cudaError_t launch_scenario_io(const Dev& dv, float* out, const float* in, cudaStream_t s);
cudaError_t launch_goals(const Consts& c, const Dev& dv, float* goals, cudaStream_t s);
// Debug build: one index check of `index` against the drone count (see
// qs_debug_check_selftest).
cudaError_t launch_check_selftest(const Dev& dv, int index, cudaStream_t s);

}  // namespace qsk
