// qs_api.cu -- the C ABI of libquadswarm_gpu.so (declared in include/qs.h):
// argument validation, device memory of a handle, launch plans per swarm
// width class, and the host-buffer step.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "qs.h"
#include "qs_internal.h"

using namespace qsk;

static thread_local std::string g_create_error;

struct qs_env {
    qs_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int D = 0, E = 0, K = 0, obs_dim = 0;
    Consts c{};
    Dev dv{};
    std::vector<int32_t> env_off_h;
    std::vector<ClassPlan> plan;
    std::vector<int> class_first_slot;  // first slot of each class in perm
    std::vector<int> class_slots;       // slots per class
    std::vector<int> perm_h;            // envs grouped by width class (host copy of d_perm)
    Tile* d_tiles = nullptr;
    int* d_perm = nullptr;
    void* arena = nullptr;
    // rollout: one tile table over all classes (costliest first), launch shape
    Tile* d_rtiles = nullptr;
    int n_rtiles = 0;
    // differentiable rollout: small CTAs (one or two warps), one tile each
    Tile* d_dtiles = nullptr;
    int n_dtiles = 0;
    // warp-specialised rollout: tiles of 32 ws_p drone lanes (every class <= 32 ws_p wide)
    Tile* d_wtiles = nullptr;
    int n_wtiles = 0;
    int ws_p = 0;  // 1 or 2 dynamics warps per CTA; 0: a class is wider than 64
    int diff_block = 32;
    int rollout_block = 128;  // or QS_BLOCK_WARP_SPECIALISED
    bool single_drone = false;  // every env holds one drone (the single-drone rollout instance)
    int rollout_fuse = 0;   // control steps per launch (0: all T in one launch)
    int rollout_grid = 0;   // resident CTAs for rollout_block
    int use_graph = 1;
    int* d_counter = nullptr;
    cudaGraphExec_t graph = nullptr;
    struct {
        int T, fuse, block;
        const void *a, *o, *r, *d;
    } graph_key{};
    // device staging of qs_step_host (one allocation, made on first use)
    char* stage = nullptr;
    size_t st_obs = 0, st_rew = 0, st_done = 0;
    int32_t* status_h = nullptr;  // host view of the status word (qs_sync)
    bool status_mapped = false;   // the device status word is page-locked host memory
    // resident step server (qs_serve_*): while it runs its launch occupies the stream
    bool serving = false;
    unsigned long long* serve_words = nullptr;  // page-locked, mapped: [0] go (slot << 32 | steps), [1] fin (low half)
    unsigned long long* serve_dev = nullptr;    // device: [0] CTAs finished since the launch began, [1] relay word
    ServeIO serve_io{};
    int serve_k = 0;                             // steps completed since qs_serve_begin
    std::string err;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

qs_status fail(qs_env* h, qs_status s, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return s;
}

// Calls that use the handle's stream or state are refused while a resident
// server occupies the stream.
qs_status busy(qs_env* h, const char* who) {
    return fail(h, QS_ERR_ARG, std::string(who) + ": the handle is serving (call qs_serve_end first)");
}

qs_status cuda_fail(qs_env* h, cudaError_t e, const char* where) {
    return fail(h, QS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int width_class(int n) {
    int w = 1;
    while (w < n) w <<= 1;
    return w;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

void build_consts(qs_env* h) {
    const qs_config& f = h->cfg;
    const qs_params& p = f.params;
    Consts& c = h->c;
    c.dt = f.dt;
    c.g = p.gravity;
    c.kappa = p.kappa;
    c.mu = p.mu;
    c.alpha_nd = p.alpha_nd;
    c.alpha_c = p.alpha_c;
    c.sig_cv = p.coll_sigma_v;
    c.sig_cw = p.coll_sigma_w;
    c.obs_sx = p.obs_sigma_x;
    c.obs_sv = p.obs_sigma_v;
    c.obs_sw = p.obs_sigma_w;
    c.room_hx = p.room_hx;
    c.room_hy = p.room_hy;
    c.room_h = p.room_h;
    c.beta = p.smooth_beta;
    c.inv_beta = 1.0f / p.smooth_beta;
    c.kc = p.smooth_kc;
    c.omega_max = p.omega_max;
    c.ans_frac = p.alpha_ns_frac;
    c.prox_factor = p.prox_factor;
    c.dr_lo = p.dr_lo;
    c.dr_hi = p.dr_hi;
    c.dw_k1 = p.dw_k1;
    c.dw_k2 = p.dw_k2;
    c.dw_b1 = p.dw_b1;
    c.dw_h = p.dw_height;
    c.dw_sa = p.dw_sigma_a;
    c.dw_sw = p.dw_sigma_w;
    c.scn_mask = f.scenarios & ((1u << QS_NSCN_TYPES) - 1u);
    c.form_s = p.form_spacing;
    c.form_rmax = p.form_rmax;
    c.scn_m = p.scn_margin;
    c.se_min = p.se_min;
    c.se_period = p.se_period;
    c.liss_f = p.liss_f;
    c.bez_seg = (int)p.bez_seg;
    // golden angle (3 - sqrt 5) / 2 turns as a 32-bit fixed-point fraction
    c.golden_q32 = (uint32_t)std::floor(4294967296.0 * (3.0 - std::sqrt(5.0)) / 2.0);
    const float nom[QS_PARAM_DIM] = {p.mass, p.ixx, p.iyy, p.izz, p.t2w, p.tau_m, p.arm};
    for (int k = 0; k < QS_PARAM_DIM; ++k) c.nominal[k] = nom[k];
    for (int k = 0; k < QS_NW; ++k) c.w[k] = p.w[k];
    c.flags = f.flags;
    c.substeps = f.substeps;
    c.K = f.k_neighbors;
    c.episode_steps = f.episode_steps;
    c.obs_dim = 18 + 6 * f.k_neighbors;
    c.key0 = (uint32_t)(f.seed & 0xffffffffu);
    c.key1 = (uint32_t)(f.seed >> 32);
    set_round_keys(c);
}

// Tiles of one class: `slots` consecutive slots starting at `first`, each CTA
// takes block / W of them.
void build_tiles(qs_env* h, std::vector<Tile>& tiles) {
    tiles.clear();
    for (size_t ci = 0; ci < h->plan.size(); ++ci) {
        ClassPlan& cp = h->plan[ci];
        const int per = cp.block / cp.W;
        cp.tile_off = (int)tiles.size();
        cp.n_tiles = 0;
        for (int s = 0; s < h->class_slots[ci]; s += per) {
            const int first = h->class_first_slot[ci] + s, count = std::min(per, h->class_slots[ci] - s);
            int contig = 1;
            for (int i = 1; i < count; ++i) contig &= h->perm_h[first + i] == h->perm_h[first] + i;
            tiles.push_back(Tile{first, count, cp.W, contig});
            ++cp.n_tiles;
        }
    }
}

// Rollout tiles: every class cut into tiles of rollout_block threads, widest
// class first (its tiles cost the most: the pair pass is O(N^2)), so that the
// persistent CTAs take the long tiles before the short ones.
void build_rollout_tiles(qs_env* h, std::vector<Tile>& tiles, int block) {
    tiles.clear();
    for (int ci = (int)h->plan.size() - 1; ci >= 0; --ci) {
        const int W = h->plan[ci].W;
        const int per = block / W;
        for (int s = 0; s < h->class_slots[ci]; s += per)
            tiles.push_back(Tile{h->class_first_slot[ci] + s, std::min(per, h->class_slots[ci] - s), W, 0});
    }
}

// Tiles of the warp-specialised rollout: 32P drone lanes per CTA (P = 1 when
// every class is at most 32 wide, 2 when at most 64), slots of one class
// each; none when a class is wider than 64.
void build_ws_tiles(qs_env* h, std::vector<Tile>& tiles) {
    tiles.clear();
    int maxW = 1;
    for (const ClassPlan& cp : h->plan) maxW = std::max(maxW, cp.W);
    h->ws_p = maxW <= 32 ? 1 : maxW <= 64 ? 2 : 0;
    if (!h->ws_p) return;
    for (size_t ci = 0; ci < h->plan.size(); ++ci) {
        const int W = h->plan[ci].W, per = 32 * h->ws_p / W;
        for (int s = 0; s < h->class_slots[ci]; s += per) {
            const int first = h->class_first_slot[ci] + s, count = std::min(per, h->class_slots[ci] - s);
            int contig = 1;
            for (int i = 1; i < count; ++i) contig &= h->perm_h[first + i] == h->perm_h[first] + i;
            tiles.push_back(Tile{first, count, W, contig});
        }
    }
}

void drop_graph(qs_env* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_key = {};
}

// One wave of warp-specialised CTAs: 8 two-warp CTAs of 32 drones per SM.
long ws_wave(int n_sm) { return (long)n_sm * 8 * 32; }

// The warp-specialised step wins while a class is latency-bound: up to about
// one wave of its CTAs. Swarms of 17..32 keep it only up to two CTAs per SM:
// their dynamics warps' pair pass (31 partners a drone) is heavy in issue
// slots, and once more CTAs share an SM the noise warps' work competes for
// those slots instead of filling idle ones (measured on GB300 at K = 6,
// warp-specialised vs one env per 32-thread CTA: 8,192 drones 16.99 vs 17.13
// us, 16,384 18.77 vs 17.83, 32,768 25.04 vs 21.26; swarms of 16 stay level
// or ahead up to 32,768).
bool use_ws(int W, int slots, int n_sm) {
    const long threads = (long)slots * W;
    return W <= 32 && threads <= (W > 16 ? (long)n_sm * 64 : ws_wave(n_sm));
}

// Default launch shape of the general per-call kernel: 64 threads per CTA (or
// W) for classes beyond a wave (small CTAs interleave their load, compute and
// store phases best: measured at 262,144 and 1,048,576 single-drone envs);
// else enough CTAs to cover 2 CTAs per SM when the class has the threads for
// it, 32..256 threads per CTA.
int default_block(int W, int slots, int n_sm) {
    const long threads = (long)slots * W;
    if (threads > ws_wave(n_sm)) return std::max(64, W);
    if (W >= 32) return W;  // one env per CTA (32-wide: 21.3 vs 22.7 us for 64-thread CTAs at 32,768 drones)
    int b = 256;
    while (b > 32 && b > W && threads / b < 2 * n_sm) b >>= 1;
    return std::max(b, std::max(W, 32));
}

bool rollout_is_ws(const qs_env* h) { return h->rollout_block == QS_BLOCK_WARP_SPECIALISED; }

// Whether a tile table of `lanes` lanes per tile cuts E envs of width W into
// consecutive runs of lanes / W slots from slot 0 (the rule tile_at computes).
bool follows_uniform_rule(const Tile* t, size_t n, int E, int W, int lanes) {
    const int per = lanes / W;
    if (per < 1 || per * W != lanes || (long)n * per < E) return false;
    for (size_t i = 0; i < n; ++i) {
        const int first = (int)i * per;
        if (t[i].first != first || t[i].count != std::min(per, E - first) || t[i].W != W) return false;
    }
    return true;
}

// Uniform geometry: one width class, every env the same size, envs in slot
// order, and every tile table the kernels read following the computed rule
// for the block it is launched with.
void set_uniform(qs_env* h, const std::vector<Tile>& tiles, const std::vector<Tile>& rtiles, int rblock,
                 const std::vector<Tile>& dtiles, const std::vector<Tile>& wtiles) {
    h->dv.uni_n = 0;
    h->dv.uni_wlog = 0;
    if (h->plan.size() != 1 || h->E < 1) return;
    const int N = h->env_off_h[1], W = h->plan[0].W;
    for (int e = 0; e <= h->E; ++e)
        if (h->env_off_h[e] != e * N) return;
    for (int e = 0; e < h->E; ++e)
        if (h->perm_h[e] != e) return;
    const ClassPlan& cp = h->plan[0];
    if (!follows_uniform_rule(tiles.data() + cp.tile_off, cp.n_tiles, h->E, W, cp.block) ||
        !follows_uniform_rule(rtiles.data(), rtiles.size(), h->E, W, rblock) ||
        !follows_uniform_rule(dtiles.data(), dtiles.size(), h->E, W, h->diff_block) ||
        (!wtiles.empty() && !follows_uniform_rule(wtiles.data(), wtiles.size(), h->E, W, 32 * h->ws_p)))
        return;
    int wlog = 0;
    while ((1 << wlog) < W) ++wlog;
    h->dv.uni_n = N;
    h->dv.uni_wlog = wlog;
}

qs_status upload_tiles(qs_env* h) {
    std::vector<Tile> tiles, rtiles, dtiles, wtiles;
    build_tiles(h, tiles);
    const int rblock = rollout_is_ws(h) ? 128 : h->rollout_block;  // the persistent kernel's tiles stay available
    build_rollout_tiles(h, rtiles, rblock);
    build_ws_tiles(h, wtiles);
    int maxW = 1;
    for (const ClassPlan& cp : h->plan) maxW = std::max(maxW, cp.W);
    h->diff_block = std::max(32, maxW);  // many small CTAs: the adjoint is latency-bound
    build_rollout_tiles(h, dtiles, h->diff_block);
    set_uniform(h, tiles, rtiles, rblock, dtiles, wtiles);
    drop_graph(h);
    if (h->d_tiles) cudaFree(h->d_tiles);
    h->d_tiles = nullptr;
    h->d_rtiles = nullptr;
    h->d_dtiles = nullptr;
    h->d_wtiles = nullptr;
    const size_t n0 = tiles.size(), n1 = rtiles.size(), n2 = dtiles.size(), n = n0 + n1 + n2 + wtiles.size();
    cudaError_t e = cudaMalloc(&h->d_tiles, sizeof(Tile) * std::max<size_t>(n, 1));
    if (e != cudaSuccess) return fail(h, QS_ERR_OOM, "tile table allocation failed");
    tiles.insert(tiles.end(), rtiles.begin(), rtiles.end());
    tiles.insert(tiles.end(), dtiles.begin(), dtiles.end());
    tiles.insert(tiles.end(), wtiles.begin(), wtiles.end());
    e = cudaMemcpy(h->d_tiles, tiles.data(), sizeof(Tile) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "tile table upload");
    h->d_rtiles = h->d_tiles + n0;
    h->n_rtiles = (int)n1;
    h->d_dtiles = h->d_tiles + n0 + n1;
    h->n_dtiles = (int)n2;
    h->d_wtiles = h->d_tiles + n0 + n1 + n2;
    h->n_wtiles = (int)wtiles.size();
    h->single_drone = maxW == 1;
    h->rollout_grid = rollout_grid(rblock, extended_instance(h->c), h->single_drone);
    return QS_OK;
}

// Enqueues the rollout of T steps: ceil(T / fuse) persistent launches.
qs_status enqueue_rollout(qs_env* h, int T, const RolloutIO& io) {
    const int fuse = h->rollout_fuse > 0 ? h->rollout_fuse : T;
    for (int t0 = 0; t0 < T; t0 += fuse) {
        const int n = std::min(fuse, T - t0);
        cudaError_t e = rollout_is_ws(h)
                            ? launch_rollout_ws(h->c, h->dv, h->d_wtiles, h->n_wtiles, h->ws_p, h->d_perm, io, t0, n,
                                                h->stream)
                            : launch_rollout(h->c, h->dv, h->d_rtiles, h->n_rtiles, h->rollout_block, h->d_perm,
                                             h->d_counter, io, t0, n, h->rollout_grid, h->single_drone, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "rollout launch");
    }
    return QS_OK;
}


// One control step of every env. A handle with several width classes steps
// them all in one launch of the rollout kernels with T = 1 (the same bits as
// the per-class kernels; measured on GB300 with sizes 1..64: 4096 envs 90.8
// -> 35.5 us, 65,536 envs 271 -> 207 us); one class keeps its per-call kernel.
qs_status do_step(qs_env* h, const float* act, float* obs, float* rew, uint8_t* done) {
    if (h->plan.size() > 1) return enqueue_rollout(h, 1, RolloutIO{act, obs, rew, done});
    StepIO io{act, obs, rew, done};
    for (const ClassPlan& cp : h->plan) {
        cudaError_t e = launch_step(h->c, h->dv, cp, h->d_tiles, h->d_perm, io, 0, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
    }
    return QS_OK;
}

// (Re)starts the resident server at step serve_k: go = fin = serve_k, the CTA
// counter zeroed and the relay word at serve_k before the cooperative launch.
qs_status serve_launch(qs_env* h) {
    const unsigned long long go = (unsigned long long)(unsigned int)h->serve_k;  // slot 0
    __atomic_store_n(h->serve_words, go, __ATOMIC_SEQ_CST);
    *(volatile int*)(h->serve_words + 1) = h->serve_k;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    const unsigned long long init[2] = {0ull, go};
    cudaError_t e = cudaMemcpy(h->serve_dev, init, sizeof init, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_serve(h->c, h->dv, h->d_wtiles, h->n_wtiles, h->ws_p, h->d_perm, h->serve_io, h->serve_k, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "resident server launch");
    h->serving = true;
    return QS_OK;
}

}  // namespace

extern "C" {

void qs_config_default(qs_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->size = sizeof(qs_config);
    cfg->n_envs = 1;
    cfg->swarm_sizes = nullptr;
    cfg->n_per_env = 1;
    cfg->k_neighbors = 6;
    cfg->substeps = 2;
    cfg->dt = 0.005f;
    cfg->episode_steps = 1500;
    cfg->seed = 1;
    cfg->flags = QS_F_DR | QS_F_MOTOR_NOISE | QS_F_OBS_NOISE | QS_F_COLLISIONS | QS_F_FLOOR | QS_F_WALLS;
    qs_params& p = cfg->params;
    p.mass = 0.028f;
    p.arm = 0.046f;
    p.ixx = 1.657e-5f;
    p.iyy = 1.666e-5f;
    p.izz = 2.926e-5f;
    p.t2w = 2.0f;
    p.kappa = 0.006f;
    p.tau_m = 0.04f;
    p.gravity = 9.81f;
    p.mu = 0.3f;
    p.alpha_nd = 0.9f;
    p.alpha_ns_frac = 0.02f;
    p.alpha_c = 0.8f;
    p.coll_sigma_v = 0.2f;
    p.coll_sigma_w = 0.5f;
    p.obs_sigma_x = 5e-3f;
    p.obs_sigma_v = 1e-2f;
    p.obs_sigma_w = 1.75e-4f;
    p.room_hx = 5.0f;
    p.room_hy = 5.0f;
    p.room_h = 10.0f;
    p.dr_lo = 0.8f;
    p.dr_hi = 1.2f;
    p.smooth_beta = 200.0f;
    p.smooth_kc = 20.0f;
    p.prox_factor = 4.0f;
    p.omega_max = 40.0f;
    p.dw_k1 = 2.4525f;
    p.dw_k2 = -2.0f;
    p.dw_b1 = 1.0f;
    p.dw_height = 0.5f;
    p.dw_sigma_a = 0.1f;
    p.dw_sigma_w = 1.0f;
    cfg->scenarios = 0;
    p.form_spacing = 0.5f;
    p.form_rmax = 4.0f;
    p.scn_margin = 1.5f;
    p.se_min = 0.5f;
    p.se_period = 400.0f;
    p.liss_f = 0.1f;
    p.bez_seg = 300.0f;
    p.w[QS_W_POS] = -1.0f;
    p.w[QS_W_SPIN] = -0.1f;
    p.w[QS_W_HIT_FLOOR] = -1.0f;
    p.w[QS_W_HIT_WALL] = -1.0f;
    p.w[QS_W_HIT_CEIL] = -1.0f;
    p.w[QS_W_HIT_QUAD] = -1.0f;
}

qs_status qs_create(const qs_config* cfg, void* cuda_stream, qs_env** out) {
    if (!out) return fail(nullptr, QS_ERR_ARG, "qs_create: out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, QS_ERR_ARG, "qs_create: cfg is NULL");
    if (cfg->size != sizeof(qs_config)) return fail(nullptr, QS_ERR_ARG, "qs_create: cfg->size mismatch (ABI version)");
    if (cfg->n_envs < 1) return fail(nullptr, QS_ERR_ARG, "qs_create: n_envs must be >= 1");
    if (cfg->k_neighbors < 0) return fail(nullptr, QS_ERR_ARG, "qs_create: k_neighbors must be >= 0");
    if (cfg->k_neighbors > QS_MAX_K) return fail(nullptr, QS_ERR_UNSUPPORTED, "qs_create: k_neighbors > 8");
    if (cfg->substeps < 1 || cfg->substeps > 255) return fail(nullptr, QS_ERR_ARG, "qs_create: substeps must be 1..255");
    if (!(cfg->dt > 0.0f)) return fail(nullptr, QS_ERR_ARG, "qs_create: dt must be > 0");
    if (cfg->episode_steps < 1) return fail(nullptr, QS_ERR_ARG, "qs_create: episode_steps must be >= 1");
    const qs_params& pp = cfg->params;
    if (cfg->scenarios >> QS_NSCN_TYPES) return fail(nullptr, QS_ERR_ARG, "qs_create: unknown scenario bits");
    if ((cfg->scenarios & ~1u) &&
        !(pp.form_spacing > 0.0f && pp.form_rmax > 0.0f && pp.se_period > 0.0f && pp.bez_seg >= 1.0f &&
          pp.scn_margin >= 0.0f && pp.liss_f >= 0.0f))
        return fail(nullptr, QS_ERR_ARG, "qs_create: scenario constants out of range");
    if (!(pp.mass > 0 && pp.arm > 0 && pp.ixx > 0 && pp.iyy > 0 && pp.izz > 0 && pp.t2w > 0 && pp.tau_m > 0 &&
          pp.dr_lo > 0 && pp.dr_hi >= pp.dr_lo && pp.omega_max > 0 && pp.prox_factor > 0))
        return fail(nullptr, QS_ERR_ARG, "qs_create: physical parameters must be positive");

    qs_env* h = new (std::nothrow) qs_env();
    if (!h) return fail(nullptr, QS_ERR_OOM, "qs_create: host allocation failed");
    h->cfg = *cfg;
    h->cfg.swarm_sizes = nullptr;
    h->stream = (cudaStream_t)cuda_stream;
    h->E = cfg->n_envs;
    h->K = cfg->k_neighbors;
    h->obs_dim = 18 + 6 * h->K;
    std::vector<int32_t> sizes(h->E);
    for (int e = 0; e < h->E; ++e) sizes[e] = cfg->swarm_sizes ? cfg->swarm_sizes[e] : cfg->n_per_env;
    h->env_off_h.assign(h->E + 1, 0);
    std::vector<int32_t> env_of;
    for (int e = 0; e < h->E; ++e) {
        if (sizes[e] < 1) {
            delete h;
            return fail(nullptr, QS_ERR_ARG, "qs_create: swarm sizes must be >= 1");
        }
        if (sizes[e] > QS_MAX_SWARM) {
            delete h;
            return fail(nullptr, QS_ERR_UNSUPPORTED, "qs_create: swarm size > 128");
        }
        h->env_off_h[e + 1] = h->env_off_h[e] + sizes[e];
        if (h->env_off_h[e + 1] > (1 << 30)) {
            delete h;
            return fail(nullptr, QS_ERR_UNSUPPORTED, "qs_create: too many drones");
        }
        for (int i = 0; i < sizes[e]; ++i) env_of.push_back(e);
    }
    h->D = h->env_off_h[h->E];
    cudaGetDevice(&h->device);
    build_consts(h);

    int n_sm = 152;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, h->device);
    // envs grouped by width class (stable order inside a class)
    std::vector<int> perm;
    for (int W = 1; W <= QS_MAX_SWARM; W <<= 1) {
        int first = (int)perm.size();
        for (int e = 0; e < h->E; ++e)
            if (width_class(sizes[e]) == W) perm.push_back(e);
        int n = (int)perm.size() - first;
        if (n > 0) {
            // latency-bound classes: warp-specialised per-call step on tiles of 32 drone lanes
            const int ws = use_ws(W, n, n_sm) ? 1 : 0;
            h->plan.push_back(ClassPlan{W, ws ? 32 : default_block(W, n, n_sm), ws, 0, 0});
            h->class_first_slot.push_back(first);
            h->class_slots.push_back(n);
        }
    }
    // default rollout shape: warp-specialised while every class is at most 32
    // wide, its CTAs (one per 32 drone lanes) fit one wave on the device
    // (latency-bound; a second wave would run the whole horizon again) and
    // neither scenarios nor downwash lengthen the dynamics warp's step (then
    // its noise warp would idle at the barriers); else the persistent kernel,
    // whose work counter also balances uneven swarm sizes. Measured on GB300
    // (warp-specialised vs persistent, us per step): plain 8192 x 1 2.66 vs
    // 3.47, 28,672 x 1 3.75 vs 3.90, 30,720 x 1 (past the 29,184 lanes of
    // one wave) 5.89 vs 3.90; swarm 2048 x 8 4.81 vs 6.67, 4096 x 8 9.46 vs
    // 7.81; with every scenario type 1.9e9 vs 2.0e9 quadrotor-steps/s;
    // uneven sizes up to 64 (two-warp pairs per CTA) 1.86e9 vs 1.80e9, close
    // enough to leave to the autotuner.
    {
        int maxW = 1;
        long ws_ctas = 0;
        for (size_t ci = 0; ci < h->plan.size(); ++ci) {
            maxW = std::max(maxW, h->plan[ci].W);
            const int per = std::max(1, 32 / h->plan[ci].W);
            ws_ctas += (h->class_slots[ci] + per - 1) / per;
        }
        const bool ext = (h->c.scn_mask & ~1u) != 0 || (h->c.flags & QS_F_DOWNWASH) != 0;
        if (maxW <= 32 && !ext && ws_ctas <= rollout_ws_resident_ctas(h->c, 1))
            h->rollout_block = QS_BLOCK_WARP_SPECIALISED;
    }

    // one arena for the state
    const size_t D = h->D, E = h->E;
    const bool rec = (cfg->flags & QS_F_RECORD_KNN) && h->K > 0;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = (off + 255) & ~size_t(255);
        off = o + bytes;
        return o;
    };
    const size_t o_st = take(sizeof(float4) * NPLANE * D), o_prm = take(sizeof(float) * NPRM_DEV * E),
                 o_goal = take(sizeof(float) * 3 * E), o_ep = take(sizeof(int32_t) * E),
                 o_tick = take(sizeof(uint32_t) * E), o_off = take(sizeof(int32_t) * (E + 1)),
                 o_of = take(sizeof(int32_t) * D), o_ev = take(sizeof(uint32_t) * D),
                 o_knn = take(rec ? sizeof(int16_t) * h->K * D : 0), o_status = take(sizeof(int32_t)),
                 o_perm = take(sizeof(int) * E), o_cnt = take(sizeof(int)),
                 o_scn = take(sizeof(float) * 2 * QS_NSCN * E), o_sel = take(E);
    cudaError_t ce = cudaMalloc(&h->arena, off);
    if (ce != cudaSuccess) {
        delete h;
        return fail(nullptr, QS_ERR_OOM, std::string("qs_create: device allocation failed: ") + cudaGetErrorString(ce));
    }
    char* base = (char*)h->arena;
    h->dv.st = (float4*)(base + o_st);
    h->dv.prm = (float*)(base + o_prm);
    h->dv.goal = (float*)(base + o_goal);
    h->dv.ep = (int32_t*)(base + o_ep);
    h->dv.tick = (uint32_t*)(base + o_tick);
    h->dv.env_off = (const int32_t*)(base + o_off);
    h->dv.env_of = (const int32_t*)(base + o_of);
    h->dv.ev = (uint32_t*)(base + o_ev);
    h->dv.knn = rec ? (int16_t*)(base + o_knn) : nullptr;
    h->dv.status = (int32_t*)(base + o_status);
    {
        // where the device can update page-locked host memory atomically (a
        // coherent host link), the status word lives there: kernels set it in
        // place and qs_sync reads it after its wait, with no copy
        int native = 0;
        void* dptr = nullptr;
        if (cudaDeviceGetAttribute(&native, cudaDevAttrHostNativeAtomicSupported, h->device) == cudaSuccess && native &&
            cudaHostAlloc((void**)&h->status_h, sizeof(int32_t), cudaHostAllocMapped) == cudaSuccess) {
            if (cudaHostGetDevicePointer(&dptr, h->status_h, 0) == cudaSuccess && dptr) {
                *h->status_h = 0;
                h->dv.status = (int32_t*)dptr;
                h->status_mapped = true;
            } else {
                cudaFreeHost(h->status_h);
                h->status_h = nullptr;
            }
        }
        cudaGetLastError();
    }
    h->dv.scn = (float*)(base + o_scn);
    h->dv.scn_sel = (uint8_t*)(base + o_sel);
    h->dv.D = h->D;
    h->dv.E = h->E;
    h->d_perm = (int*)(base + o_perm);
    h->d_counter = (int*)(base + o_cnt);
    bool ok = cudaMemset(h->arena, 0, off) == cudaSuccess &&
              cudaMemcpy((void*)h->dv.env_off, h->env_off_h.data(), sizeof(int32_t) * (E + 1), cudaMemcpyHostToDevice) ==
                  cudaSuccess &&
              cudaMemcpy((void*)h->dv.env_of, env_of.data(), sizeof(int32_t) * D, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(h->d_perm, perm.data(), sizeof(int) * E, cudaMemcpyHostToDevice) == cudaSuccess;
    auto release = [&]() {
        cudaFree(h->d_tiles);
        cudaFree(h->arena);
        if (h->status_h) cudaFreeHost(h->status_h);
        delete h;
    };
    if (!ok) {
        release();
        return fail(nullptr, QS_ERR_CUDA, "qs_create: initial upload failed");
    }
    h->perm_h = perm;
    qs_status s = upload_tiles(h);
    if (s != QS_OK) {
        std::string m = h->err;
        release();
        return fail(nullptr, s, m);
    }
    ce = launch_reset(h->c, h->dv, h->c.key0, h->c.key1, nullptr, h->stream);
    if (ce != cudaSuccess) {
        release();
        return fail(nullptr, QS_ERR_CUDA, std::string("qs_create: reset launch: ") + cudaGetErrorString(ce));
    }
    *out = h;
    return QS_OK;
}

qs_status qs_destroy(qs_env* h) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_destroy: NULL handle");
    DeviceGuard g(h->device);
    if (h->serving) qs_serve_end(h);
    cudaStreamSynchronize(h->stream);
    drop_graph(h);
    cudaFree(h->d_tiles);
    cudaFree(h->arena);
    cudaFree(h->stage);
    if (h->status_h) cudaFreeHost(h->status_h);
    if (h->serve_words) cudaFreeHost(h->serve_words);
    cudaFree(h->serve_dev);
    delete h;
    return QS_OK;
}

qs_status qs_get_dims(const qs_env* h, int32_t* n_drones, int32_t* n_envs, int32_t* obs_dim) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_get_dims: NULL handle");
    if (n_drones) *n_drones = h->D;
    if (n_envs) *n_envs = h->E;
    if (obs_dim) *obs_dim = h->obs_dim;
    return QS_OK;
}

qs_status qs_reset(qs_env* h, uint64_t seed, const uint8_t* env_mask_dev, float* obs_dev) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_reset: NULL handle");
    if (h->serving) return busy(h, "qs_reset");
    if (obs_dev && !aligned(obs_dev, 8)) return fail(h, QS_ERR_ARG, "qs_reset: obs_dev must be 8-byte aligned");
    DeviceGuard g(h->device);
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    if (!env_mask_dev) {
        h->c.key0 = k0;
        h->c.key1 = k1;
        set_round_keys(h->c);
        cudaError_t e = cudaMemsetAsync(h->dv.status, 0, sizeof(int32_t), h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "qs_reset");
    }
    cudaError_t e = launch_reset(h->c, h->dv, k0, k1, env_mask_dev, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qs_reset launch");
    if (obs_dev) {
        StepIO io{nullptr, obs_dev, nullptr, nullptr};
        for (const ClassPlan& cp : h->plan) {
            e = launch_step(h->c, h->dv, cp, h->d_tiles, h->d_perm, io, 1, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "qs_reset observation");
        }
    }
    return QS_OK;
}

// Event-time contacts are a model of the differentiable rollout only.
static qs_status no_event_time(qs_env* h, const char* who) {
    if (!(h->cfg.flags & QS_F_EVENT_TIME)) return QS_OK;
    return fail(h, QS_ERR_UNSUPPORTED,
                std::string(who) + ": a handle with QS_F_EVENT_TIME runs the differentiable rollout only");
}

qs_status qs_step(qs_env* h, const float* actions_dev, float* obs_dev, float* reward_dev, uint8_t* done_dev) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_step: NULL handle");
    if (h->serving) return busy(h, "qs_step");
    if (no_event_time(h, "qs_step") != QS_OK) return QS_ERR_UNSUPPORTED;
    if (!actions_dev) return fail(h, QS_ERR_ARG, "qs_step: actions_dev is NULL");
    if (!aligned(actions_dev, 16)) return fail(h, QS_ERR_ARG, "qs_step: actions_dev must be 16-byte aligned");
    if (obs_dev && !aligned(obs_dev, 8)) return fail(h, QS_ERR_ARG, "qs_step: obs_dev must be 8-byte aligned");
    DeviceGuard g(h->device);
    return do_step(h, actions_dev, obs_dev, reward_dev, done_dev);
}

// Device address of page-locked (pinned or registered) host memory that the
// device can load from and store to directly, or null for any other pointer.
void* mapped_host(const void* p, size_t align) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // an unregistered pointer is not an error here
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || !aligned(a.devicePointer, align)) return nullptr;
    return a.devicePointer;
}

qs_status qs_step_host(qs_env* h, const float* actions_host, float* obs_host, float* reward_host, uint8_t* done_host) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_step_host: NULL handle");
    if (h->serving) return busy(h, "qs_step_host");
    if (no_event_time(h, "qs_step_host") != QS_OK) return QS_ERR_UNSUPPORTED;
    if (!actions_host) return fail(h, QS_ERR_ARG, "qs_step_host: actions_host is NULL");
    DeviceGuard g(h->device);
    const size_t D = h->D, E = h->E;
    const size_t b_act = sizeof(float) * 4 * D, b_obs = sizeof(float) * h->obs_dim * D, b_rew = sizeof(float) * D,
                 b_done = E;
    // page-locked host buffers are read and written by the step kernel in place
    // (over NVLink-C2C on a Grace host); other host memory goes through device
    // staging buffers and one copy each way
    const float* a_map = (const float*)mapped_host(actions_host, 16);
    float* o_map = obs_host ? (float*)mapped_host(obs_host, 8) : nullptr;
    float* r_map = reward_host ? (float*)mapped_host(reward_host, 4) : nullptr;
    uint8_t* dn_map = done_host ? (uint8_t*)mapped_host(done_host, 1) : nullptr;
    const bool staged = !a_map || (obs_host && !o_map) || (reward_host && !r_map) || (done_host && !dn_map);
    if (staged && !h->stage) {
        h->st_obs = (b_act + 255) & ~size_t(255);
        h->st_rew = (h->st_obs + b_obs + 255) & ~size_t(255);
        h->st_done = (h->st_rew + b_rew + 255) & ~size_t(255);
        if (cudaMalloc(&h->stage, h->st_done + b_done) != cudaSuccess) {
            h->stage = nullptr;
            return fail(h, QS_ERR_OOM, "qs_step_host: staging allocation");
        }
    }
    cudaError_t e = cudaSuccess;
    const float* d_act = a_map;
    if (!d_act) {
        d_act = (float*)h->stage;
        e = cudaMemcpyAsync((void*)d_act, actions_host, b_act, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "qs_step_host: action copy");
    }
    float* d_obs = !obs_host ? nullptr : o_map ? o_map : (float*)(h->stage + h->st_obs);
    float* d_rew = !reward_host ? nullptr : r_map ? r_map : (float*)(h->stage + h->st_rew);
    uint8_t* d_done = !done_host ? nullptr : dn_map ? dn_map : (uint8_t*)(h->stage + h->st_done);
    qs_status s = do_step(h, d_act, d_obs, d_rew, d_done);
    if (s != QS_OK) return s;
    if (obs_host && !o_map && (e = cudaMemcpyAsync(obs_host, d_obs, b_obs, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "qs_step_host: observation copy");
    if (reward_host && !r_map &&
        (e = cudaMemcpyAsync(reward_host, d_rew, b_rew, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "qs_step_host: reward copy");
    if (done_host && !dn_map && (e = cudaMemcpyAsync(done_host, d_done, b_done, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "qs_step_host: done copy");
    return qs_sync(h);
}

qs_status qs_rollout(qs_env* h, int32_t T, const float* actions_dev, float* obs_dev, float* reward_dev,
                     uint8_t* done_dev) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_rollout: NULL handle");
    if (h->serving) return busy(h, "qs_rollout");
    if (no_event_time(h, "qs_rollout") != QS_OK) return QS_ERR_UNSUPPORTED;
    if (T < 1) return fail(h, QS_ERR_ARG, "qs_rollout: T must be >= 1");
    if (!actions_dev || !aligned(actions_dev, 16)) return fail(h, QS_ERR_ARG, "qs_rollout: actions_dev NULL or misaligned");
    if (obs_dev && !aligned(obs_dev, 8)) return fail(h, QS_ERR_ARG, "qs_rollout: obs_dev must be 8-byte aligned");
    DeviceGuard g(h->device);
    const RolloutIO io{actions_dev, obs_dev, reward_dev, done_dev};
    // Graph replay: the launches of one (T, buffers, shape) are captured once
    // and replayed; any change of buffers or shape re-captures. The legacy
    // default stream cannot be captured, so it launches directly.
    if (!h->use_graph || h->stream == nullptr) return enqueue_rollout(h, T, io);
    const auto& k = h->graph_key;
    if (h->graph && k.T == T && k.fuse == h->rollout_fuse && k.block == h->rollout_block && k.a == actions_dev &&
        k.o == obs_dev && k.r == reward_dev && k.d == done_dev) {
        cudaError_t e = cudaGraphLaunch(h->graph, h->stream);
        return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "rollout graph launch");
    }
    drop_graph(h);
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "rollout capture begin");
    qs_status s = enqueue_rollout(h, T, io);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->stream, &graph);
    if (s != QS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "rollout capture end");
    e = cudaGraphInstantiate(&h->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return cuda_fail(h, e, "rollout graph instantiate");
    }
    h->graph_key = {T, h->rollout_fuse, h->rollout_block, actions_dev, obs_dev, reward_dev, done_dev};
    e = cudaGraphLaunch(h->graph, h->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "rollout graph launch");
}

qs_status qs_set_rollout_shape(qs_env* h, int32_t block, int32_t fuse, int32_t use_graph) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_set_rollout_shape: NULL handle");
    if (h->serving) return busy(h, "qs_set_rollout_shape");
    int maxW = 1;
    for (const ClassPlan& cp : h->plan) maxW = std::max(maxW, cp.W);
    const bool ws = block == QS_BLOCK_WARP_SPECIALISED && maxW <= 64;
    if (!ws && (block < 32 || block > 256 || block % 32 != 0 || block < maxW))
        return fail(h, QS_ERR_ARG, "qs_set_rollout_shape: block must be 32..256, a multiple of 32, >= the widest class, "
                                   "or QS_BLOCK_WARP_SPECIALISED when every class is at most 64 wide");
    if (fuse < 0) return fail(h, QS_ERR_ARG, "qs_set_rollout_shape: fuse must be >= 0");
    DeviceGuard g(h->device);
    cudaError_t e = cudaStreamSynchronize(h->stream);  // the old tables may be in use
    if (e != cudaSuccess) return cuda_fail(h, e, "qs_set_rollout_shape");
    h->rollout_block = block;
    h->rollout_fuse = fuse;
    h->use_graph = use_graph ? 1 : 0;
    return upload_tiles(h);
}

static qs_status diff_check(qs_env* h, const char* who, int32_t T, int32_t C) {
    if (!h) return fail(nullptr, QS_ERR_ARG, std::string(who) + ": NULL handle");
    if (h->serving) return busy(h, who);
    if (h->cfg.flags & QS_F_DOWNWASH)
        return fail(h, QS_ERR_UNSUPPORTED, std::string(who) + ": the differentiable rollout has no downwash term");
    if (h->c.scn_mask & ~1u)
        return fail(h, QS_ERR_UNSUPPORTED, std::string(who) + ": the differentiable rollout uses the single goal only");
    if ((h->cfg.flags & QS_F_EVENT_TIME) && (h->cfg.flags & QS_F_SMOOTH))
        return fail(h, QS_ERR_UNSUPPORTED, std::string(who) + ": event-time contacts apply to the discrete contacts only");
    if (T < 1 || C < 1) return fail(h, QS_ERR_ARG, std::string(who) + ": T and ckpt_every must be >= 1");
    return QS_OK;
}

qs_status qs_diff_workspace_size(const qs_env* h, int32_t T, int32_t ckpt_every, size_t* bytes) {
    if (!h || !bytes) return fail(nullptr, QS_ERR_ARG, "qs_diff_workspace_size: NULL argument");
    if (T < 1 || ckpt_every < 1) return fail(nullptr, QS_ERR_ARG, "qs_diff_workspace_size: T, ckpt_every >= 1");
    *bytes = diff_workspace_bytes(h->D, T, std::min(T, ckpt_every), h->cfg.substeps);
    return QS_OK;
}

qs_status qs_diff_forward(qs_env* h, int32_t T, int32_t ckpt_every, const float* x0_dev, const float* actions_dev,
                          float* loss_dev, void* workspace_dev) {
    qs_status s = diff_check(h, "qs_diff_forward", T, ckpt_every);
    if (s != QS_OK) return s;
    if (!x0_dev || !loss_dev || !workspace_dev || !actions_dev || !aligned(actions_dev, 16) || !aligned(workspace_dev, 16))
        return fail(h, QS_ERR_ARG, "qs_diff_forward: NULL or misaligned buffer");
    DeviceGuard g(h->device);
    cudaError_t e = launch_diff(0, h->c, h->dv, h->d_dtiles, h->n_dtiles, h->diff_block, h->d_perm, x0_dev,
                                actions_dev, loss_dev, nullptr, nullptr, nullptr, workspace_dev, T,
                                std::min(T, ckpt_every), h->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "qs_diff_forward launch");
}

qs_status qs_diff_backward(qs_env* h, int32_t T, int32_t ckpt_every, const float* actions_dev, const float* dloss_dev,
                           void* workspace_dev, float* grad_actions_dev, float* grad_x0_dev) {
    qs_status s = diff_check(h, "qs_diff_backward", T, ckpt_every);
    if (s != QS_OK) return s;
    if (!dloss_dev || !workspace_dev || !actions_dev || !grad_actions_dev || !grad_x0_dev || !aligned(actions_dev, 16) ||
        !aligned(grad_actions_dev, 16) || !aligned(workspace_dev, 16))
        return fail(h, QS_ERR_ARG, "qs_diff_backward: NULL or misaligned buffer");
    DeviceGuard g(h->device);
    cudaError_t e = launch_diff(1, h->c, h->dv, h->d_dtiles, h->n_dtiles, h->diff_block, h->d_perm, nullptr,
                                actions_dev, nullptr, dloss_dev, grad_actions_dev, grad_x0_dev, workspace_dev, T,
                                std::min(T, ckpt_every), h->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "qs_diff_backward launch");
}

// ---------------------------------------------------------------------------
// Allocation-free differentiable rollout (qs_diff_grad_static).
//
// Some callers cannot allocate device memory at the point where they need a
// gradient: code that runs while a CUDA graph is being captured, real-time
// control loops that must never call cudaMalloc or cudaFree (either may
// synchronise the whole device), and plugins inside a host framework that owns
// the device's memory budget. For them the workspace of the forward + adjoint
// pass (checkpoints and recomputed substep states) lives in this fixed array
// of the library's device image instead of a caller buffer. Every GPU that
// loads the library keeps the array until the process exits.
static __device__ __align__(256) unsigned char g_diff_static[QS_DIFF_STATIC_BYTES];

namespace {
std::mutex g_static_mu;
void* g_static_addr[256] = {};  // device address of g_diff_static, per device ordinal

// Device address of the array on the current device. In host code
// g_diff_static names a host-side stand-in, not memory the GPU can use, so
// the address comes from cudaGetSymbolAddress. It is looked up again on every
// call made while the handle's stream is not capturing (a device reset or a
// released primary context moves the array); while capturing, the address
// found by the last such call on this device is used, so the first call on a
// device has to come before any capture.
qs_status static_workspace(qs_env* h, void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "qs_diff_grad_static: cudaGetDevice");
    if (dev < 0 || dev >= 256) return fail(h, QS_ERR_UNSUPPORTED, "qs_diff_grad_static: device ordinal >= 256");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(h->stream, &cs);
    if (e != cudaSuccess) return cuda_fail(h, e, "qs_diff_grad_static: cudaStreamIsCapturing");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_diff_static);
        if (e != cudaSuccess || !p) return cuda_fail(h, e, "qs_diff_grad_static: cudaGetSymbolAddress");
        g_static_addr[dev] = p;
    } else if (!g_static_addr[dev]) {
        return fail(h, QS_ERR_UNSUPPORTED,
                    "qs_diff_grad_static: the first call on a device must come before any stream capture");
    }
    *out = g_static_addr[dev];
    return QS_OK;
}
}  // namespace

qs_status qs_diff_grad_static(qs_env* h, int32_t T, int32_t ckpt_every, const float* x0_dev, const float* actions_dev,
                              const float* dloss_dev, float* loss_dev, float* grad_actions_dev, float* grad_x0_dev) {
    qs_status s = diff_check(h, "qs_diff_grad_static", T, ckpt_every);
    if (s != QS_OK) return s;
    if (!x0_dev || !actions_dev || !dloss_dev || !loss_dev || !grad_actions_dev || !grad_x0_dev ||
        !aligned(actions_dev, 16) || !aligned(grad_actions_dev, 16))
        return fail(h, QS_ERR_ARG, "qs_diff_grad_static: NULL or misaligned buffer");
    const int C = std::min(T, ckpt_every);
    const size_t need = diff_workspace_bytes(h->D, T, C, h->cfg.substeps);
    if (need > (size_t)QS_DIFF_STATIC_BYTES)
        return fail(h, QS_ERR_UNSUPPORTED,
                    "qs_diff_grad_static: this rollout needs " + std::to_string(need) + " bytes of workspace, the static "
                    "workspace holds " + std::to_string((size_t)QS_DIFF_STATIC_BYTES) +
                    "; use fewer drones, a shorter horizon or checkpoint interval, or qs_diff_forward/qs_diff_backward "
                    "with a caller workspace");
    DeviceGuard g(h->device);
    void* ws = nullptr;
    s = static_workspace(h, &ws);
    if (s != QS_OK) return s;
    // Every byte the backward pass reads is written earlier in this call (the
    // checkpoints by the forward pass, the substep states by the recompute),
    // so nothing left by a previous call needs clearing.
    cudaError_t e = launch_diff(0, h->c, h->dv, h->d_dtiles, h->n_dtiles, h->diff_block, h->d_perm, x0_dev,
                                actions_dev, loss_dev, nullptr, nullptr, nullptr, ws, T, C, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qs_diff_grad_static forward launch");
    e = launch_diff(1, h->c, h->dv, h->d_dtiles, h->n_dtiles, h->diff_block, h->d_perm, nullptr, actions_dev, nullptr,
                    dloss_dev, grad_actions_dev, grad_x0_dev, ws, T, C, h->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "qs_diff_grad_static backward launch");
}

qs_status qs_get_rollout_shape(const qs_env* h, int32_t* block, int32_t* fuse, int32_t* use_graph) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_get_rollout_shape: NULL handle");
    if (block) *block = h->rollout_block;
    if (fuse) *fuse = h->rollout_fuse;
    if (use_graph) *use_graph = h->use_graph;
    return QS_OK;
}

qs_status qs_get_state(qs_env* h, float* state_dev, float* params_dev, float* goals_dev, int32_t* ep_step_dev,
                       uint32_t* tick_dev) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_get_state: NULL handle");
    if (h->serving) return busy(h, "qs_get_state");
    DeviceGuard g(h->device);
    cudaError_t e = launch_get_state(h->dv, state_dev, params_dev, goals_dev, ep_step_dev, tick_dev, h->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "qs_get_state");
}

qs_status qs_set_state(qs_env* h, const float* state_dev, const float* params_dev, const float* goals_dev,
                       const int32_t* ep_step_dev, const uint32_t* tick_dev) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_set_state: NULL handle");
    if (h->serving) return busy(h, "qs_set_state");
    DeviceGuard g(h->device);
    cudaError_t e = launch_set_state(h->c, h->dv, state_dev, params_dev, goals_dev, ep_step_dev, tick_dev, h->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "qs_set_state");
}

qs_status qs_get_events(qs_env* h, uint32_t* events_dev, int16_t* knn_dev) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_get_events: NULL handle");
    if (h->serving) return busy(h, "qs_get_events");
    if (knn_dev && !h->dv.knn && h->K > 0)
        return fail(h, QS_ERR_ARG, "qs_get_events: neighbour lists need QS_F_RECORD_KNN at creation");
    if (!events_dev && !knn_dev) return QS_OK;
    DeviceGuard g(h->device);
    cudaError_t e = launch_get_events(h->dv, h->K, events_dev, knn_dev, h->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "qs_get_events");
}

qs_status qs_get_scenario(qs_env* h, float* records_dev) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_get_scenario: NULL handle");
    if (h->serving) return busy(h, "qs_get_scenario");
    if (!records_dev) return fail(h, QS_ERR_ARG, "qs_get_scenario: records_dev is NULL");
    DeviceGuard g(h->device);
    cudaError_t e = launch_scenario_io(h->dv, records_dev, nullptr, h->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "qs_get_scenario");
}

qs_status qs_set_scenario(qs_env* h, const float* records_dev) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_set_scenario: NULL handle");
    if (h->serving) return busy(h, "qs_set_scenario");
    if (!records_dev) return fail(h, QS_ERR_ARG, "qs_set_scenario: records_dev is NULL");
    DeviceGuard g(h->device);
    cudaError_t e = launch_scenario_io(h->dv, nullptr, records_dev, h->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "qs_set_scenario");
}

qs_status qs_get_goals(qs_env* h, float* goals_dev) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_get_goals: NULL handle");
    if (h->serving) return busy(h, "qs_get_goals");
    if (!goals_dev) return fail(h, QS_ERR_ARG, "qs_get_goals: goals_dev is NULL");
    DeviceGuard g(h->device);
    cudaError_t e = launch_goals(h->c, h->dv, goals_dev, h->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "qs_get_goals");
}

qs_status qs_sync(qs_env* h) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_sync: NULL handle");
    if (h->serving) return busy(h, "qs_sync");
    DeviceGuard g(h->device);
    if (!h->status_h && cudaHostAlloc((void**)&h->status_h, sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess) {
        h->status_h = nullptr;
        return fail(h, QS_ERR_OOM, "qs_sync: pinned status word");
    }
    cudaError_t e = cudaSuccess;
    if (!h->status_mapped) {
        // the status word follows the stream's work, so one wait covers both
        e = cudaMemcpyAsync(h->status_h, h->dv.status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "qs_sync status copy");
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qs_sync");
    const int32_t st = *(volatile int32_t*)h->status_h;
    if (st & 1) return fail(h, QS_ERR_STATE_NONFINITE, "a drone state became non-finite");
    if (st & 2) return fail(h, QS_ERR_INDEX, "a device index check of the debug build failed");
    return QS_OK;
}

int32_t qs_build_flags(void) {
#ifdef QS_DEBUG_CHECKS
    return QS_BUILD_DEBUG_CHECKS;
#else
    return 0;
#endif
}

qs_status qs_debug_check_selftest(qs_env* h, int32_t index) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_debug_check_selftest: NULL handle");
    if (h->serving) return busy(h, "qs_debug_check_selftest");
    if (!(qs_build_flags() & QS_BUILD_DEBUG_CHECKS))
        return fail(h, QS_ERR_UNSUPPORTED, "qs_debug_check_selftest: the release build has no device index checks");
    DeviceGuard g(h->device);
    cudaError_t e = launch_check_selftest(h->dv, index, h->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(h, e, "qs_debug_check_selftest");
}

qs_status qs_set_block(qs_env* h, int32_t width, int32_t block) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_set_block: NULL handle");
    if (h->serving) return busy(h, "qs_set_block");
    const bool ws = block == QS_BLOCK_WARP_SPECIALISED;
    if (ws ? width > 32 : (block < 32 || block > 256 || block % 32 != 0 || block % width != 0))
        return fail(h, QS_ERR_ARG, "qs_set_block: block must be 32..256, a multiple of 32 and of width, or "
                                   "QS_BLOCK_WARP_SPECIALISED for widths <= 32");
    for (ClassPlan& cp : h->plan) {
        if (cp.W != width) continue;
        DeviceGuard g(h->device);
        cudaError_t e = cudaStreamSynchronize(h->stream);  // the old tile table may be in use
        if (e != cudaSuccess) return cuda_fail(h, e, "qs_set_block");
        cp.ws = ws ? 1 : 0;
        cp.block = ws ? 32 : block;
        return upload_tiles(h);
    }
    return fail(h, QS_ERR_ARG, "qs_set_block: no envs of that width class");
}

qs_status qs_get_block(const qs_env* h, int32_t width, int32_t* block) {
    if (!h || !block) return fail(nullptr, QS_ERR_ARG, "qs_get_block: NULL argument");
    *block = 0;
    for (const ClassPlan& cp : h->plan)
        if (cp.W == width) *block = cp.ws ? QS_BLOCK_WARP_SPECIALISED : cp.block;
    return QS_OK;
}

qs_status qs_serve_begin(qs_env* h, const float* actions_host, int32_t n_slots, float* obs_host, float* reward_host,
                         uint8_t* done_host, int32_t idle_ms) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_serve_begin: NULL handle");
    if (h->serving) return fail(h, QS_ERR_ARG, "qs_serve_begin: the handle is already serving");
    if (no_event_time(h, "qs_serve_begin") != QS_OK) return QS_ERR_UNSUPPORTED;
    if (!actions_host) return fail(h, QS_ERR_ARG, "qs_serve_begin: actions_host is NULL");
    if (idle_ms < 1 || idle_ms > QS_SERVE_IDLE_MS_MAX)
        return fail(h, QS_ERR_ARG, "qs_serve_begin: idle_ms must be in [1, " + std::to_string(QS_SERVE_IDLE_MS_MAX) + "]");
    if (n_slots < 1) return fail(h, QS_ERR_ARG, "qs_serve_begin: n_slots must be >= 1");
    if (!h->ws_p || h->n_wtiles < 1)
        return fail(h, QS_ERR_UNSUPPORTED, "qs_serve_begin: every swarm must have at most 64 drones");
    DeviceGuard g(h->device);
    unsigned int sflags = 0;
    if (!h->stream || cudaStreamGetFlags(h->stream, &sflags) != cudaSuccess || !(sflags & cudaStreamNonBlocking)) {
        cudaGetLastError();
        return fail(h, QS_ERR_UNSUPPORTED, "qs_serve_begin: the handle's stream must be a non-blocking stream (the "
                                           "legacy default stream would wait behind the resident launch)");
    }
    int native = 0;
    if (cudaDeviceGetAttribute(&native, cudaDevAttrHostNativeAtomicSupported, h->device) != cudaSuccess || !native) {
        cudaGetLastError();
        return fail(h, QS_ERR_UNSUPPORTED, "qs_serve_begin: the device has no native atomics on host memory");
    }
    const float* a = (const float*)mapped_host(actions_host, 16);
    float* o = obs_host ? (float*)mapped_host(obs_host, 8) : nullptr;
    float* r = reward_host ? (float*)mapped_host(reward_host, 4) : nullptr;
    uint8_t* dn = done_host ? (uint8_t*)mapped_host(done_host, 1) : nullptr;
    if (!a || (obs_host && !o) || (reward_host && !r) || (done_host && !dn))
        return fail(h, QS_ERR_ARG, "qs_serve_begin: buffers must be page-locked host memory the device can map "
                                   "(actions 16-byte, observations 8-byte aligned)");
    if (serve_resident_ctas(h->c, h->ws_p) < h->n_wtiles)
        return fail(h, QS_ERR_UNSUPPORTED, "qs_serve_begin: the handle's CTAs do not fit on the device at once");
    if (!h->serve_words) {
        void* dp = nullptr;
        if (cudaHostAlloc((void**)&h->serve_words, 2 * sizeof(unsigned long long), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(&dp, h->serve_words, 0) != cudaSuccess || !dp) {
            if (h->serve_words) cudaFreeHost(h->serve_words);
            h->serve_words = nullptr;
            cudaGetLastError();
            return fail(h, QS_ERR_OOM, "qs_serve_begin: handshake words");
        }
        h->serve_io.go = (unsigned long long*)dp;
        h->serve_io.fin = (int*)((unsigned long long*)dp + 1);
    }
    if (!h->serve_dev && cudaMalloc(&h->serve_dev, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        h->serve_dev = nullptr;
        return fail(h, QS_ERR_OOM, "qs_serve_begin: CTA counter");
    }
    // drain the stream: the server must not queue behind earlier work it cannot see
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "qs_serve_begin");
    h->serve_io.act = a;
    h->serve_io.obs = o;
    h->serve_io.rew = r;
    h->serve_io.done = dn;
    h->serve_io.count = h->serve_dev;
    h->serve_io.relay = h->serve_dev + 1;
    h->serve_io.n_slots = n_slots;
    h->serve_io.idle_ns = (long long)idle_ms * 1000000;
    h->serve_k = 0;
    return serve_launch(h);
}

qs_status qs_serve_step(qs_env* h, int32_t slot) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_serve_step: NULL handle");
    if (!h->serving) return fail(h, QS_ERR_ARG, "qs_serve_step: the handle is not serving (qs_serve_begin)");
    if (slot < 0 || slot >= h->serve_io.n_slots) return fail(h, QS_ERR_ARG, "qs_serve_step: slot out of range");
    const int k = h->serve_k;
    unsigned long long* go = h->serve_words;
    // the caller's command writes happen before the post (sequentially consistent swap)
    for (int relaunches = 0;;) {
        unsigned long long cur = __atomic_load_n(go, __ATOMIC_SEQ_CST);
        const int steps = (int)(unsigned int)(cur & 0xffffffffull);
        if (steps == k) {
            const unsigned long long want = ((unsigned long long)(unsigned int)slot << 32) | (unsigned int)(k + 1);
            if (__atomic_compare_exchange_n(go, &cur, want, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST)) break;
            continue;  // the server retired meanwhile
        }
        if (steps == k + 1) break;  // posted by a call that returned QS_ERR_TIMEOUT: keep waiting for it
        if (steps != SERVE_IDLE || relaunches++ > 0) {
            h->serving = false;
            return fail(h, QS_ERR_CUDA, "qs_serve_step: the server's handshake word holds an unexpected value");
        }
        // the server retired while the host was idle; its launch ends by itself
        DeviceGuard g(h->device);
        cudaError_t e = cudaStreamSynchronize(h->stream);
        h->serving = false;
        if (e != cudaSuccess) return cuda_fail(h, e, "qs_serve_step");
        qs_status st = serve_launch(h);
        if (st != QS_OK) return st;
    }
    volatile int* fin = (volatile int*)(h->serve_words + 1);
    const auto t0 = std::chrono::steady_clock::now();
    for (unsigned long i = 1; *fin != k + 1; ++i) {
        if ((i & 4095) == 0) {
            DeviceGuard g(h->device);
            const cudaError_t q = cudaStreamQuery(h->stream);
            if (q != cudaErrorNotReady) {
                if (*fin == k + 1) break;
                h->serving = false;
                if (q == cudaSuccess) return fail(h, QS_ERR_CUDA, "qs_serve_step: the server ended before the step completed");
                return cuda_fail(h, q, "qs_serve_step");
            }
            if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(10))
                return fail(h, QS_ERR_TIMEOUT, "qs_serve_step: the step did not complete within 10 s");
        }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    h->serve_k = k + 1;
    if (h->status_mapped && (*(volatile int32_t*)h->status_h & 1))
        return fail(h, QS_ERR_STATE_NONFINITE, "a drone state became non-finite");
    return QS_OK;
}

qs_status qs_serve_end(qs_env* h) {
    if (!h) return fail(nullptr, QS_ERR_ARG, "qs_serve_end: NULL handle");
    if (!h->serving) return QS_OK;
    // from whatever step go holds (serve_k, or serve_k + 1 after a timed-out
    // post); a retired server (SERVE_IDLE) is ending its launch already
    unsigned long long cur = __atomic_load_n(h->serve_words, __ATOMIC_SEQ_CST);
    while ((int)(unsigned int)(cur & 0xffffffffull) >= 0) {
        const unsigned long long stop = (cur & ~0xffffffffull) | (unsigned long long)(unsigned int)SERVE_STOP;
        if (__atomic_compare_exchange_n(h->serve_words, &cur, stop, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST)) break;
    }
    DeviceGuard g(h->device);
    const cudaError_t e = cudaStreamSynchronize(h->stream);
    h->serving = false;
    if (e != cudaSuccess) return cuda_fail(h, e, "qs_serve_end");
    if (h->status_mapped && (*(volatile int32_t*)h->status_h & 1))
        return fail(h, QS_ERR_STATE_NONFINITE, "a drone state became non-finite");
    return QS_OK;
}

qs_status qs_philox4x32_10(const uint32_t* ctr_dev, uint32_t key0, uint32_t key1, int32_t variant, uint32_t* out_dev,
                           int64_t n, void* cuda_stream) {
    if (n < 0 || (n > 0 && (!ctr_dev || !out_dev)) || (variant != 0 && variant != 1) || (out_dev && !aligned(out_dev, 16)))
        return fail(nullptr, QS_ERR_ARG, "qs_philox4x32_10: NULL or misaligned buffer, n < 0 or variant not 0 / 1");
    const cudaError_t e = launch_philox(ctr_dev, key0, key1, variant, out_dev, (long long)n, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? QS_OK : fail(nullptr, QS_ERR_CUDA, std::string("qs_philox4x32_10: ") + cudaGetErrorString(e));
}

const char* qs_last_error(const qs_env* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
