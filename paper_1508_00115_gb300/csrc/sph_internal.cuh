// sph_internal.cuh -- library-private declarations shared by the libsph sources.
//
// Layout in HBM (all library-owned unless noted, n = particle count, cell order):
//   caller SoA (FP64 x,y,z,vx,vy,vz; FP32 m,u,h and outputs)  -- caller-owned
//   pos4[n]     float4 {x - c_cell, y - c_cell, z - c_cell, h}  cell-relative FP32
//   vel4[n]     float4 {vx, vy, vz, m} (FP32; predicted velocities inside a step)
//   thermo4[n]  float4 {rho, A = f P / rho^2, c, B}  written by the density pass
//   upred[n]    FP32 internal energy seen by the pressure (predicted inside a step)
//   ids[n]      int64 composite permutation (original index of each slot)
//   cell_start[n_cells + 1], tiles[n_tiles]  cell ranges and warp work items
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <string>
#include <vector>

#include "../../include/sph.h"

namespace sph {

constexpr float kSigma = 2.54647908947032550f;  // 8/pi, 3-D cubic-spline normalisation
constexpr float kFourPi3 = 4.18879020478639098f; // 4 pi / 3
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMinTile = 16;          // smallest tile (targets per warp work item)
constexpr int kMaxNc = 512;           // cells per side cap
constexpr int64_t kScanAuxCap = 65536; // block sums of one exclusive scan (4096 items/block)
// FP32 distance tests within kBandK * h * (h + L) of the cutoff are re-decided in
// FP64 from the absolute positions (2^-19; the FP32 error bound is ~2^-21 h(3.5L+h)).
constexpr float kBandK = 1.9073486328125e-06f;
// Box pruning keeps sources up to (1 + kPruneMargin) H^2 so that no pair the FP32 or
// FP64 test accepts is pruned.
constexpr float kPruneMargin = 2.44140625e-04f;  // 2^-12

// device counters (unsigned long long slots)
enum Counter {
    C_UNCONV = 0,     // unconverged particles after the last density pass
    C_HFLAG = 1,      // some h outgrew what the cells (leaf lists) hold
    C_DPAIRS = 2,     // density interactions
    C_FPAIRS = 3,     // force interactions
    C_DCAND = 4,      // density candidate tests
    C_FCAND = 5,      // force candidate tests
    C_FLOORS = 6,     // u floors
    C_DTARGETS = 7,   // active density targets
    C_GFLAGS = 8,     // multi-step run: OR of per-step flags (1: unconverged, 2: h beyond cells,
                      // 4: h below what the uniform grid's FP32 frame resolves, 8: a
                      // tensor-core wait of the learned-h inference ran out)
    C_SHRINK = 9,     // adaptive: leaves whose largest h fell below kTreeShrink x its build value
    C_WALKOVF = 10,   // adaptive: leaf walks whose stack overflowed
    C_LISTTOT = 11,   // adaptive: neighbour-list entries (64-bit total)
    C_TICKET = 12,    // pair kernels: next tile group to hand out (reset before each launch)
    C_BINACT = 13,    // individual time-steps: particles whose step ends at the current time
    C_BINMAX = 14,    // individual time-steps: deepest bin in use
    C_BINOVER = 15,   // individual time-steps: CFL steps below the smallest bin's step
    C_PREC = 16,      // uniform grid: a converged h below cell side / SPH_FRAME_RATIO
    C_GPAIRS = 17,    // gravity near field: pair interactions
    C_SYMGATHER = 18, // symmetric force pass: some cell needs the radius-2 stencil (gather runs instead)
    C_DSTREAM = 19,   // density: sources read from the cells / lists (before the box test)
    C_DSTAGED = 20,   // density: sources staged for the distance tests (per tile)
    C_FSTREAM = 21,   // force: sources read
    C_FSTAGED = 22,   // force: sources staged
    C_LIMCHG = 23,    // time-step limiter: bins one pass changed
    C_LIMITED = 24,   // time-step limiter: starting steps whose bin it raised
    C_WOKEN = 25,     // time-step limiter: steps cut by wake-ups
    C_TMIN = 26,      // individual time-steps: earliest step end
    C_LIMACT = 27,    // time-step limiter: particles in the active list
    C_TCERR = 28,     // learned h: a tensor-core (mbarrier) wait of the inference ran out
    C_NCOUNTERS = 29
};

// Cell grid of one periodic box (every box has side box_size; boxes are batched
// by concatenating their particle ranges and their cell numberings).
struct BoxDev {
    int p_begin, p_end;  // particle slots of the box (cell order keeps boxes contiguous)
    int cell_off;        // global id of the box's first cell
    int nc;              // cells per side
    double L64;          // cell side, box / nc
    double s;            // nc / box
    float L32;           // cell side, FP32
    float hplan;         // max h the grid was planned for
};

// Adaptive cells: a leaf's neighbour list holds every leaf whose bounding box comes
// within kTreeReach x (the larger of the two leaves' largest h at build time), so
// the lists stay exact while no h grows beyond kTreeReach x its leaf's build value.
// (A CFL step changes h by a few per cent at most; 1.15 leaves room for that and for
// Newton overshoots, and loads 1.15^3 / 1.25^3 = 0.78 of the list volume of 1.25:
// 2-3 % faster steps on clustered fields.)
constexpr float kTreeReach = 1.15f;
// ... and once many leaves' largest h fell below kTreeShrink x its build value the
// lists are worth rebuilding (they are valid, only longer than needed)
constexpr float kTreeShrink = 0.45f;

// octree node inside a top cell: a contiguous range of the sorted particles
struct TreeNode {
    int lo, hi;        // particle slots [lo, hi)
    int child;         // first child node (children are consecutive), -1 for a leaf
    int nchild;
    int top;           // global top-cell id
    int level;         // 0 = the top cell itself
    unsigned long long prefix;  // Morton prefix inside the top cell (3 bits per level)
    float hmax;        // largest h of its particles
    int parent;        // -1 for a top cell
    float bx0, by0, bz0, bx1, by1, bz1;  // bounding box, relative to the top-cell centre
};

// device-side sizes of an adaptive build that runs without host reads (the build
// inside a graph-captured step)
struct TreeCounts {
    int nl, err;
    int level_begin[18];           // nodes of level L: [level_begin[L], level_begin[L + 1])
    unsigned long long list_total;
    unsigned long long walk_ovf;   // a warp's list walk overflowed its stack
    unsigned walk_ticket[2];       // leaf tickets of the counting and the filling walk
};
// TreeCounts.err bits: the nodes did not fit (some leaves stay above leaf_max, the
// lists remain exact), the neighbour lists did not fit (the step did no pair work)
constexpr int kTreeErrNodes = 1, kTreeErrList = 2;

// adaptive cells (sph_tree.cu): arrays and their capacities
struct AdaptiveTree {
    TreeNode *nodes = nullptr;
    int *front = nullptr, *front2 = nullptr, *bounds = nullptr, *node_leaf = nullptr, *node_at = nullptr;
    uint32_t *nkids = nullptr;
    int *top_node = nullptr;   // root node of every top cell (-1: empty)
    int *leaf_of = nullptr;    // leaf of every particle slot
    int *tord = nullptr;       // slots of every leaf in ascending h (the targets of its tiles)
    int *act_ord = nullptr;    // later density passes: active slots packed per leaf (tord order)
    int *nact_leaf = nullptr;  // active targets per leaf
    int *leaf_node = nullptr;
    int2 *leaf_rng = nullptr;  // particle slots of every leaf
    double *leaf_cen = nullptr; // absolute centre of every leaf (3 per leaf)
    float4 *leaf_lo = nullptr, *leaf_hi = nullptr;  // leaf bounding box relative to its centre
                                                    // (lo.w: the leaf's largest h at the build)
    float *leaf_h = nullptr;     // largest h per leaf when the tree was built
    float *leaf_scale = nullptr; // coordinate scale of the leaf's pair arithmetic (FP32 band width)
    uint32_t *list_off = nullptr; // neighbour-list offsets, n_leaves + 1
    float4 *list = nullptr;     // {offset between leaf centres, neighbour leaf}
    uint32_t *h_u32 = nullptr;  // pinned scratch for host reads
    int *h_i32 = nullptr;
    int64_t cap_keys = 0, cap_keys2 = 0, cap_leaf_of = 0, cap_tord = 0, cap_act_ord = 0, cap_nact_leaf = 0, cap_node_at = 0, cap_top = 0, cap_nodes = 0,
            cap_front = 0, cap_front2 = 0, cap_bounds = 0, cap_nkids = 0, cap_node_leaf = 0, cap_leaf_node = 0,
            cap_leaf_rng = 0, cap_leaf_cen = 0, cap_leaf_h = 0, cap_leaf_scale = 0, cap_list_off = 0, cap_list = 0,
            cap_leaf_lo = 0, cap_leaf_hi = 0;
    int n_nodes = 0, n_leaves = 0;
    int64_t n_entries = 0;
    // graph-captured steps: counts on the device (dc) and their pinned host copy (hc),
    // fixed capacities of a frontier and of the node array, and the build mode
    TreeCounts *dc = nullptr, *hc = nullptr;
    int64_t dev_capf = 0, dev_cap_nodes = 0, dev_cap_list = 0;
    bool device_sized = false;   // build without host reads (set while a step is captured)
};

// learned initial h (sph_hpredict.cu)
struct HPredictor {
    float *params = nullptr, *adam_m = nullptr, *adam_v = nullptr;  // FP32 parameters, Adam moments
    float *norm = nullptr;        // feature / target normalisation
    uint16_t *wbf = nullptr;      // BF16 inference copy
    float *gpart = nullptr;       // per-block partial gradients
    double *stat_part = nullptr;  // normalisation sums
    float *d_loss = nullptr, *h_loss = nullptr;
    float *feats = nullptr, *h_prev = nullptr;  // features of the current state, h before the iteration
    int64_t cap = 0;
    std::vector<float> h_params = std::vector<float>(4673), h_norm = std::vector<float>(14);
    std::vector<uint16_t> h_wbf = std::vector<uint16_t>(5184);
    int64_t adam_t = 0;
    bool ready = false, norm_set = false;
    // sample collection during sph_step (caller's device buffers)
    float *col_feats = nullptr, *col_target = nullptr;
    int64_t col_cap = 0, col_n = 0;
};

struct Grid {
    int nc = 0;          // box 0 (statistics)
    int64_t n_cells = 0; // all boxes
    double L64 = 0;      // box 0
    int key_bits = 0;
};

struct Timer {
    cudaEvent_t a, b;
    int kind;  // 0 density, 1 force, 2 build, 3 gravity
};

}  // namespace sph

struct sph_ctx {
    sph_params p{};
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t n = 0, cap = 0;

    // packed particle data
    float4 *pos4 = nullptr, *vel4 = nullptr, *thermo4 = nullptr;
    // SPH_FLAG_AXIS_SWEEP: for each of the 13 half-stencil directions, every cell's
    // particles sorted by their projection on it: {projection, slot}, 13 x cap
    float2 *axis = nullptr;
    int64_t axis_cap = 0;
    float *upred = nullptr;
    float *h_lo = nullptr, *h_hi = nullptr;  // bracket of each particle's h root (density iteration)
    uint8_t *active = nullptr;
    int64_t *ids = nullptr, *ids_tmp = nullptr;
    uint64_t *ngb_hash = nullptr;
    // sort
    uint32_t *keys = nullptr, *keys_alt = nullptr, *vals = nullptr, *vals_alt = nullptr;
    uint64_t *keys64 = nullptr, *keys64_alt = nullptr;  // adaptive cells (allocated on first use)
    uint32_t *hist = nullptr;  // 256 * n_sort_tiles
    uint32_t *scan_aux = nullptr;
    int64_t hist_cap = 0;
    // permutation scratch (gather targets before the copy back)
    double *s64 = nullptr;  // 6 * cap
    float *s32 = nullptr;   // 10 * cap
    // adaptive cells (SPH_FLAG_ADAPTIVE)
    bool adaptive = false;
    int leaf_max = 64;
    bool h_guess_pending = false;  // SPH_FLAG_TREE_H_GUESS before the first build
    sph::HPredictor hp;            // learned initial h (SPH_FLAG_HPREDICT)
    sph::AdaptiveTree tree;
    // boxes and their cell grids
    int n_boxes = 1;
    std::vector<int64_t> box_off;     // host, n_boxes + 1
    int64_t *d_box_off = nullptr;     // device copy
    sph::BoxDev *d_boxes = nullptr;   // device, n_boxes
    sph::BoxDev *h_boxes = nullptr;   // pinned host mirror
    float *d_box_hmax = nullptr;      // device, n_boxes
    float *h_box_hmax = nullptr;      // pinned
    bool planned = false;             // d_boxes holds a grid plan
    // cells
    sph::Grid grid;
    int tile_w = 16;             // targets per tile: 16 (two tiles per warp) or 32
    int *cell_start = nullptr;
    int64_t cell_cap = 0;
    float *cell_hmax = nullptr;   // max h per cell (scratch of the reach passes)
    float *cell_tmp = nullptr;    // after cell_reach: max h over the 5x5x5 cell block
    int4 *tiles = nullptr;
    int64_t tile_cap = 0;
    int *n_tiles = nullptr;      // device scalar
    int4 *act_tiles = nullptr;   // tiles with an unconverged target (later density passes)
    uint32_t *tile_flag = nullptr, *tile_pos = nullptr;  // compaction by prefix sum (tile_cap each)
    int *n_act_tiles = nullptr;  // device scalar
    bool tuned = false;          // autotuner ran
    uint32_t *cell_tiles = nullptr;  // per-cell tile counts -> offsets
    // scalars
    unsigned long long *counters = nullptr;  // device
    unsigned long long *h_counters = nullptr; // pinned host mirror
    float *d_scalars = nullptr;   // [0] max h, [1] min h/vsig
    float *h_scalars = nullptr;   // pinned
    double *d_red = nullptr;      // FP64 reduction partials
    double *h_red = nullptr;      // pinned
    int64_t red_blocks = 0;
    // host-buffer stepping
    sph_particles dev_mirror{};
    int64_t mirror_cap = 0;
    void *mirror_block = nullptr;
    // inside sph_step_host: the caller's arrays, and a second stream on which each
    // result goes back to the host once the step has finished with it
    sph_particles *host_out = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev = nullptr;

    bool ids_valid = false;   // ids hold a permutation
    bool built = false;       // cells match the current positions
    bool density_valid = false;
    bool hydro_valid = false; // a, dudt, vsig match the current state
    bool predict = false;     // gather predicts v, u by half of *d_dt (inside a step)
    double *d_dt = nullptr;   // device: the step's dt
    double *h_dt = nullptr;   // pinned
    // captured multi-step graph
    cudaGraphExec_t step_exec = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream the step is captured on
    // what the captured step depends on besides device memory: reuse it while equal
    struct GraphKey {
        sph_particles parts;
        double dt;
        int64_t n, n_cells;
        int key_bits, passes, tile_w;
        uint64_t tree_sig;  // adaptive cells: arrays and capacities the captured build uses
        bool sym;           // symmetric force pass
        bool operator==(const GraphKey &o) const
        {
            return memcmp(&parts, &o.parts, sizeof parts) == 0 && dt == o.dt && n == o.n && n_cells == o.n_cells &&
                   key_bits == o.key_bits && passes == o.passes && tile_w == o.tile_w && tree_sig == o.tree_sig &&
                   sym == o.sym;
        }
    } graph_key{};
    int64_t graph_launches = 0;  // kernels in one captured step
    // sort buffers as a replay leaves them (an odd number of radix passes swaps the
    // ping-pong pair on the host while capturing; replays always end in these)
    uint32_t *g_keys = nullptr, *g_keys_alt = nullptr, *g_vals = nullptr, *g_vals_alt = nullptr;
    uint64_t *g_keys64 = nullptr, *g_keys64_alt = nullptr;

    // individual time-steps (sph_step_bins), allocated on first use: each particle's
    // bin and whether its step ends at the current time (slot order, permuted with
    // the particles), and scratch for the quantities inactive particles keep
    int8_t *bins = nullptr, *bins_tmp = nullptr;
    uint8_t *bin_active = nullptr, *bin_active_tmp = nullptr;
    int2 *bin_st = nullptr, *bin_st_tmp = nullptr;  // {start, end} of each particle's current step
    int8_t *bins_cfl = nullptr;   // SPH_FLAG_BIN_LIMITER: the bins before the limiter's passes
    int32_t *lim_cell = nullptr;  // SPH_FLAG_BIN_LIMITER: (top-level) cell of each slot
    int *lim_want = nullptr;      // SPH_FLAG_BIN_LIMITER: bins gathered by / scattered to each particle
    int *lim_list = nullptr;      // SPH_FLAG_BIN_LIMITER: the active slots
    int *lim_cmax = nullptr;      // SPH_FLAG_BIN_LIMITER: per cell largest bin, smallest sleeping bin,
                                  // then 2 x cells of changed-cell flags
    int64_t lim_cmax_cap = 0;
    float *bin_s32 = nullptr;  // 5 * cap: rho, P, c, f, curl while permuting
    int64_t bin_cap = 0;
    bool bin_mode = false;     // inside sph_step_bins: builds also permute the above
    int bin_levels = 0;        // n_bins of the running call
    int64_t bin_now = 0;       // current time in units of dt_max / 2^n_bins
    double bin_unit = 0.0;

    // a status that does not stop a compound call (sph_step, sph_steps, sph_step_bins,
    // sph_step_host): SPH_ERR_PRECISION, or SPH_ERR_NOT_CONVERGED after the pass budget,
    // from a density pass whose results were written; the call finishes and returns
    // the first such status (with its message) at the end
    int soft_rc = 0;
    std::string soft_msg;

    // symmetric force pass (SPH_FLAG_SYMMETRIC or the autotuner's choice): source-side
    // slots, 13 float4 per particle, and the source-side v_sig maxima
    bool sym_force = false;
    float4 *sym_slot = nullptr;
    unsigned *sym_vsig = nullptr;
    int64_t sym_cap = 0;

    // statistics
    sph_stats st{};
    std::vector<sph::Timer> timers;
    std::vector<sph::Timer> free_timers;
    std::string err;
};

namespace sph {

// error plumbing -------------------------------------------------------------
int fail(sph_ctx *ctx, int code, const std::string &msg);
int cuda_fail(sph_ctx *ctx, cudaError_t e, const char *what);
#define SPH_CUDA(ctx, call)                                          \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return sph::cuda_fail(ctx, e_, #call); \
    } while (0)
// after every kernel launch: count it and surface launch errors
#define SPH_LAUNCH(ctx, what)                                         \
    do {                                                              \
        (ctx)->st.kernel_launches++;                                  \
        cudaError_t e_ = cudaGetLastError();                          \
        if (e_ != cudaSuccess) return sph::cuda_fail(ctx, e_, what);  \
    } while (0)

// timing
void timer_begin(sph_ctx *ctx, int kind, cudaEvent_t *out_end);
void timer_end(sph_ctx *ctx, cudaEvent_t end);

// launch wrappers (defined in the .cu files) ---------------------------------
int plan_cells(sph_ctx *ctx, sph_particles *parts);             // sph_cells.cu (host read)
int read_box_max_h(sph_ctx *ctx, sph_particles *parts);         // sph_cells.cu (host read)
int plan_from_hmax(sph_ctx *ctx);                               // sph_cells.cu
bool plan_still_good(sph_ctx *ctx);                             // sph_cells.cu
int build_cells(sph_ctx *ctx, sph_particles *parts);            // sph_cells.cu (plan + build)
int build_planned(sph_ctx *ctx, sph_particles *parts);          // sph_cells.cu (no host read)
int box_max_h(sph_ctx *ctx, const float *h);                    // sph_cells.cu
int cell_reach(sph_ctx *ctx);  // cell_tmp = max h within two cells   // sph_cells.cu
int permute_particles(sph_ctx *ctx, sph_particles *parts, bool cell_pos);  // sph_cells.cu
int axis_sort(sph_ctx *ctx);  // SPH_FLAG_AXIS_SWEEP: per-cell orders along the 13 directions  // sph_cells.cu
int build_tree(sph_ctx *ctx, sph_particles *parts);             // sph_tree.cu
int tree_prepare_device(sph_ctx *ctx, uint64_t *sig);           // sph_tree.cu (before a capture)
int tree_read_device(sph_ctx *ctx);                             // sph_tree.cu (after replays)
int tree_cell_keys_out(sph_ctx *ctx, int32_t *dev_keys);        // sph_tree.cu
int tree_shrink_count(sph_ctx *ctx, sph_particles *parts);      // sph_tree.cu
int tree_leaf_hcur(sph_ctx *ctx, sph_particles *parts);         // sph_tree.cu (before a force pass)
int reset_h_brackets(sph_ctx *ctx);                             // sph_pairs.cu
// individual time-steps, sph_integrate.cu
int bin_permute(sph_ctx *ctx, sph_particles *parts);  // after each permutation: bins, kept state, prediction
int bin_active(sph_ctx *ctx, unsigned long long *n_active);  // active mask at ctx->bin_now (host read)
int bin_kick(sph_ctx *ctx, sph_particles *parts, bool all);  // half of each particle's own step
int bin_assign(sph_ctx *ctx, sph_particles *parts, bool all, double dt_max);  // new bins from the CFL step
int bin_max_read(sph_ctx *ctx, int *max_bin, unsigned long long *over,
                 int64_t *t_min);  // deepest bin in use, earliest step end (host read)
int bin_limit(sph_ctx *ctx, sph_particles *parts, bool all, int64_t *sweeps);  // limiter passes (host reads)
int bin_open(sph_ctx *ctx, sph_particles *parts, bool all, bool limiter);    // open steps; wake-ups
// sph_hpredict.cu
int hp_init(sph_ctx *ctx, uint64_t seed);
int hp_load(sph_ctx *ctx, const uint16_t *w_bf16, const float *f32);
int hp_save(sph_ctx *ctx, uint16_t *w_bf16, float *f32);
int hp_params(sph_ctx *ctx, float *out);
int hp_ensure(sph_ctx *ctx, int64_t n);  // feature buffers for n particles (outside graph capture)
int hp_features(sph_ctx *ctx, sph_particles *parts);
int hp_run(sph_ctx *ctx, const float *feats, const float *h_prev, float *out, int64_t n, float log_lo, float log_hi);
int hp_apply_step(sph_ctx *ctx, sph_particles *parts);
int hp_targets(sph_ctx *ctx, sph_particles *parts, float *dev_target);
int hp_collect(sph_ctx *ctx, sph_particles *parts);
int hp_train(sph_ctx *ctx, const float *X, const float *Y, int64_t n, int epochs, float lr, uint64_t seed,
             float *loss_out);
void hp_free(sph_ctx *ctx);
void free_tree(sph_ctx *ctx);                                   // sph_tree.cu
int cell_keys_out(sph_ctx *ctx, int32_t *dev_keys);             // sph_cells.cu
int run_density_pass(sph_ctx *ctx, sph_particles *parts, bool last_pass, bool active_list);  // sph_pairs.cu
int compact_active_tiles(sph_ctx *ctx);                                    // sph_pairs.cu
int compact_active_leaf_tiles(sph_ctx *ctx);  // adaptive cells: tiles of active targets only  // sph_tree.cu
int order_tiles(sph_ctx *ctx, int4 *tiles, const int *n_tiles);  // adaptive: longest-first tile groups  // sph_tree.cu
int run_force_pass(sph_ctx *ctx, sph_particles *parts, bool active_list = false);  // sph_pairs.cu
int run_gravity_pass(sph_ctx *ctx, double G, double eps, float *ax, float *ay, float *az, float *phi);  // sph_gravity.cu
int ensure_sym(sph_ctx *ctx);  // slot arrays of the symmetric force pass           // sph_pairs.cu
int sync_h(sph_ctx *ctx, sph_particles *parts);                            // sph_pairs.cu
int kick(sph_ctx *ctx, sph_particles *parts);    // by *d_dt / 2           // sph_integrate.cu
int drift(sph_ctx *ctx, sph_particles *parts);   // by *d_dt               // sph_integrate.cu
int set_dt(sph_ctx *ctx, double dt);             // *d_dt = dt (kernel)    // sph_integrate.cu
int cfl_dt_device(sph_ctx *ctx, sph_particles *parts);  // *d_dt = CFL    // sph_integrate.cu
int conserved_device(sph_ctx *ctx, sph_particles *parts);                  // sph_integrate.cu
int conserved_read(sph_ctx *ctx, sph_conserved *out);                      // sph_integrate.cu
int cfl_dt(sph_ctx *ctx, sph_particles *parts, double *dt_out);            // sph_integrate.cu
int exclusive_scan_u32(sph_ctx *ctx, const uint32_t *in, uint32_t *out, int64_t n);  // sph_cells.cu
int radix_sort64(sph_ctx *ctx, int n, int key_bits);                                   // sph_cells.cu

// FP32 pair math ---------------------------------------------------------------

// Cubic spline of support 1 (Monaghan & Lattanzio 1985): w(q) and dw/dq, zero for q >= 1.
__device__ __forceinline__ void spline(float q, float &w, float &dw)
{
    float t = fmaxf(1.f - q, 0.f);
    float t2 = t * t;
    float q2 = q * q;
    bool inner = q <= 0.5f;
    float w_in = fmaf(6.f * q2, q - 1.f, 1.f);  // 1 - 6q^2 + 6q^3
    float dw_in = q * fmaf(18.f, q, -12.f);     // -12q + 18q^2
    w = kSigma * (inner ? w_in : 2.f * t2 * t);
    dw = kSigma * (inner ? dw_in : -6.f * t2);
}

__device__ __forceinline__ float spline_dw(float q)
{
    float t = fmaxf(1.f - q, 0.f);
    float dw_in = q * fmaf(18.f, q, -12.f);
    return kSigma * (q <= 0.5f ? dw_in : -6.f * t * t);
}

// Compensated (Kahan) accumulation; __fadd_rn/__fsub_rn keep the compiler from
// contracting or reassociating the error term away.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// splitmix64 finaliser (neighbour-set fingerprint term)
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// FP64 re-decision of r_ij^2 < h^2 from absolute positions, minimal image, with the
// operation order of the plain definition (no contraction).
__device__ __forceinline__ double sep2_64(const double *__restrict__ x, const double *__restrict__ y,
                                          const double *__restrict__ z, int i, int j, double box)
{
    double dx = __dsub_rn(x[i], x[j]);
    dx = __dsub_rn(dx, __dmul_rn(box, rint(__ddiv_rn(dx, box))));
    double dy = __dsub_rn(y[i], y[j]);
    dy = __dsub_rn(dy, __dmul_rn(box, rint(__ddiv_rn(dy, box))));
    double dz = __dsub_rn(z[i], z[j]);
    dz = __dsub_rn(dz, __dmul_rn(box, rint(__ddiv_rn(dz, box))));
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ bool within64(double r2, float h)
{
    double hh = (double)h;
    return r2 < __dmul_rn(hh, hh);
}

// FP64 decision for a pair whose FP32 distance test fell inside the
// rounding band: bit 0 = (r_ij < h_a), bit 1 = (r_ij < h_b).  Rarely taken.
__device__ __forceinline__ unsigned band_decide(const double *__restrict__ x, const double *__restrict__ y,
                                             const double *__restrict__ z, int i, int j, double box, float ha,
                                             float hb)
{
    const double r2 = sep2_64(x, y, z, i, j, box);
    return (within64(r2, ha) ? 1u : 0u) | (within64(r2, hb) ? 2u : 0u);
}

}  // namespace sph
