// sph_api.cu -- the extern "C" entry points of libsph (declared in include/sph.h):
// argument checks, scratch ownership, and the host-side ordering of the passes
// (cells -> density with the h iteration -> force -> time step), which in the
// paper's design is expressed as task dependencies (Theuns et al. 2015, Sec. 3.1:
// densities must be known before pressure gradients).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "sph_internal.cuh"

namespace sph {

int red_scratch_doubles();  // sph_integrate.cu

int fail(sph_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(sph_ctx *ctx, cudaError_t e, const char *what)
{
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error in %s: %s", what, cudaGetErrorString(e));
    if (ctx) ctx->err = buf;
    return SPH_ERR_CUDA;
}

void timer_begin(sph_ctx *ctx, int kind, cudaEvent_t *out_end)
{
    *out_end = nullptr;
    if (!(ctx->p.flags & SPH_FLAG_TIMING)) return;
    Timer t;
    if (!ctx->free_timers.empty()) {
        t = ctx->free_timers.back();
        ctx->free_timers.pop_back();
    } else {
        if (cudaEventCreate(&t.a) != cudaSuccess) return;
        if (cudaEventCreate(&t.b) != cudaSuccess) {
            cudaEventDestroy(t.a);
            return;
        }
    }
    t.kind = kind;
    cudaEventRecord(t.a, ctx->stream);
    ctx->timers.push_back(t);
    *out_end = t.b;
}

void timer_end(sph_ctx *ctx, cudaEvent_t end)
{
    if (end) cudaEventRecord(end, ctx->stream);
}

static void free_particles(sph_ctx *c)
{
    void *ptrs[] = {c->pos4, c->vel4, c->thermo4, c->upred, c->h_lo, c->h_hi, c->active, c->ids, c->ids_tmp, c->ngb_hash,
                    c->keys, c->keys_alt, c->vals, c->vals_alt, c->hist, c->s64, c->s32, c->tiles,
                    c->act_tiles, c->tile_flag, c->tile_pos, c->sym_slot, c->sym_vsig};
    for (void *p : ptrs) cudaFree(p);
    c->sym_slot = nullptr;
    c->sym_vsig = nullptr;
    c->sym_cap = 0;
    c->pos4 = c->vel4 = c->thermo4 = nullptr;
    c->upred = nullptr;
    c->h_lo = c->h_hi = nullptr;
    c->active = nullptr;
    c->ids = c->ids_tmp = nullptr;
    c->ngb_hash = nullptr;
    c->keys = c->keys_alt = c->vals = c->vals_alt = c->hist = nullptr;
    c->s64 = nullptr;
    c->s32 = nullptr;
    c->tiles = nullptr;
    c->act_tiles = nullptr;
    c->tile_flag = c->tile_pos = nullptr;
    c->cap = 0;
}

static int alloc_particles(sph_ctx *c, int64_t cap)
{
    free_particles(c);
    cap = std::max<int64_t>(cap, 1);
    int64_t sort_tiles = (cap + 4095) / 4096;
    c->tile_cap = cap + cap / kMinTile + 64;
    SPH_CUDA(c, cudaMalloc(&c->pos4, sizeof(float4) * cap));
    SPH_CUDA(c, cudaMalloc(&c->vel4, sizeof(float4) * cap));
    SPH_CUDA(c, cudaMalloc(&c->thermo4, sizeof(float4) * cap));
    SPH_CUDA(c, cudaMalloc(&c->upred, sizeof(float) * cap));
    SPH_CUDA(c, cudaMalloc(&c->h_lo, sizeof(float) * cap));
    SPH_CUDA(c, cudaMalloc(&c->h_hi, sizeof(float) * cap));
    SPH_CUDA(c, cudaMalloc(&c->active, cap));
    SPH_CUDA(c, cudaMalloc(&c->ids, sizeof(int64_t) * cap));
    SPH_CUDA(c, cudaMalloc(&c->ids_tmp, sizeof(int64_t) * cap));
    SPH_CUDA(c, cudaMalloc(&c->ngb_hash, sizeof(uint64_t) * cap));
    SPH_CUDA(c, cudaMalloc(&c->keys, sizeof(uint32_t) * cap));
    SPH_CUDA(c, cudaMalloc(&c->keys_alt, sizeof(uint32_t) * cap));
    SPH_CUDA(c, cudaMalloc(&c->vals, sizeof(uint32_t) * cap));
    SPH_CUDA(c, cudaMalloc(&c->vals_alt, sizeof(uint32_t) * cap));
    SPH_CUDA(c, cudaMalloc(&c->hist, sizeof(uint32_t) * 256 * sort_tiles));
    SPH_CUDA(c, cudaMalloc(&c->s64, sizeof(double) * 6 * cap));
    SPH_CUDA(c, cudaMalloc(&c->s32, sizeof(float) * 10 * cap));
    SPH_CUDA(c, cudaMalloc(&c->tiles, sizeof(int4) * c->tile_cap));
    SPH_CUDA(c, cudaMalloc(&c->act_tiles, sizeof(int4) * c->tile_cap));
    SPH_CUDA(c, cudaMalloc(&c->tile_flag, sizeof(uint32_t) * c->tile_cap));
    SPH_CUDA(c, cudaMalloc(&c->tile_pos, sizeof(uint32_t) * c->tile_cap));
    SPH_CUDA(c, cudaMemsetAsync(c->ngb_hash, 0, sizeof(uint64_t) * cap, c->stream));
    c->cap = cap;
    return SPH_OK;
}

// individual time-steps: per-particle state of sph_step_bins, allocated on first use
static void free_bins(sph_ctx *c)
{
    void *ptrs[] = {c->bins, c->bins_tmp, c->bin_active, c->bin_active_tmp, c->bin_s32,
                    c->bin_st, c->bin_st_tmp, c->bins_cfl, c->lim_cell, c->lim_want, c->lim_list, c->lim_cmax};
    for (void *p : ptrs) cudaFree(p);
    c->bins = c->bins_tmp = nullptr;
    c->bin_active = c->bin_active_tmp = nullptr;
    c->bin_s32 = nullptr;
    c->bin_st = c->bin_st_tmp = nullptr;
    c->bins_cfl = nullptr;
    c->lim_cell = nullptr;
    c->lim_want = nullptr;
    c->lim_list = nullptr;
    c->lim_cmax = nullptr;
    c->lim_cmax_cap = 0;
    c->bin_cap = 0;
}

static int alloc_bins(sph_ctx *c)
{
    if (c->bin_cap >= c->cap && c->bins) return SPH_OK;
    free_bins(c);
    const int64_t cap = std::max<int64_t>(c->cap, 1);
    SPH_CUDA(c, cudaMalloc(&c->bins, cap));
    SPH_CUDA(c, cudaMalloc(&c->bins_tmp, cap));
    SPH_CUDA(c, cudaMalloc(&c->bin_active, cap));
    SPH_CUDA(c, cudaMalloc(&c->bin_active_tmp, cap));
    SPH_CUDA(c, cudaMalloc(&c->bin_s32, sizeof(float) * 5 * cap));
    SPH_CUDA(c, cudaMalloc(&c->bin_st, sizeof(int2) * cap));
    SPH_CUDA(c, cudaMalloc(&c->bin_st_tmp, sizeof(int2) * cap));
    SPH_CUDA(c, cudaMalloc(&c->bins_cfl, cap));
    SPH_CUDA(c, cudaMalloc(&c->lim_cell, sizeof(int32_t) * cap));
    SPH_CUDA(c, cudaMalloc(&c->lim_want, sizeof(int) * cap));
    SPH_CUDA(c, cudaMalloc(&c->lim_list, sizeof(int) * cap));
    c->bin_cap = cap;
    return SPH_OK;
}

static bool parts_ok(const sph_particles *p)
{
    const void *a[] = {p->x,   p->y, p->z, p->vx,   p->vy,    p->vz, p->m,  p->u,  p->h,  p->rho, p->P,
                       p->c,   p->f, p->divv, p->curl, p->n_ngb, p->ax, p->ay, p->az, p->dudt, p->vsig};
    for (const void *q : a)
        if (!q) return false;
    return true;
}

static int check_params(const sph_params *p, std::string &why)
{
    if (p->n < 0 || p->n >= (1ll << 31)) why = "n must be in [0, 2^31)";
    else if (!(p->box_size > 0) || !isfinite(p->box_size)) why = "box_size must be finite and > 0";
    else if (!(p->gamma > 1.f)) why = "gamma must be > 1";
    else if (!(p->n_ngb > 32.f / 3.f)) why = "n_ngb must exceed the self contribution 32/3";
    else if (!(p->h_tol > 0.f)) why = "h_tol must be > 0";
    else if (!(p->alpha_visc >= 0.f)) why = "alpha_visc must be >= 0";
    else if (!(p->cfl > 0.f)) why = "cfl must be > 0";
    else if (!(p->cell_factor >= 1.f) || !isfinite(p->cell_factor)) why = "cell_factor must be >= 1";
    else if (p->max_h_iter < 1) why = "max_h_iter must be >= 1";
    else if (p->kernel != 0) why = "kernel must be 0 (cubic spline)";
    else if (p->tile_width != 0 && p->tile_width != 16 && p->tile_width != 32) why = "tile_width must be 0, 16 or 32";
    else if (p->leaf_max < 0 || p->leaf_max > 4096) why = "leaf_max must be in [0, 4096]";
    else if (p->list_reserve < 0) why = "list_reserve must be >= 0";
    else if (p->n_boxes < 0) why = "n_boxes must be >= 0";
    else if (p->n_boxes > 1 && !p->box_offsets) why = "box_offsets required for n_boxes > 1";
    else if (p->n_boxes > 1 && (p->box_offsets[0] != 0 || p->box_offsets[p->n_boxes] != p->n)) why = "box_offsets must run from 0 to n";
    else if (p->n_boxes > 1 && !std::is_sorted(p->box_offsets, p->box_offsets + p->n_boxes + 1)) why = "box_offsets must be non-decreasing";
    else return SPH_OK;
    return SPH_ERR_INVALID_ARG;
}

static int read_counters(sph_ctx *ctx)
{
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_counters, ctx->counters, C_NCOUNTERS * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SPH_OK;
}

// Autotuner: for each candidate schedule, on the current particles, the cell build
// and one density pass (no h update) followed by one force pass are timed; the
// density + force pair runs twice and the faster repetition counts, so that one
// slow launch does not decide.  The score (build + density + force) follows the
// cost of a step, where a density-only score had preferred leaves that make the
// force pass and the later density passes slower.  Keeps the fastest schedule
// and leaves the cells built for it.  The probe passes write the force outputs;
// every caller runs the real passes after this.
static int autotune(sph_ctx *ctx, sph_particles *parts)
{
    const int tws[2] = {16, 32};
    const float cfs[3] = {1.05f, 1.25f, 1.5f};
    const int leaves[3] = {64, 128, 256};  // adaptive cells: leaf sizes instead of cell factors
    cudaEvent_t ev[4];
    for (int i = 0; i < 4; ++i) SPH_CUDA(ctx, cudaEventCreate(&ev[i]));
    // schedules whose cells are too large for the FP32 frame of the smallest h (uniform
    // grid, SPH_FRAME_RATIO) rank behind every schedule that holds it
    float best = 1e30f;
    bool best_fits = false;
    int best_tw = ctx->tile_w;
    float best_cf = ctx->p.cell_factor;
    int best_leaf = ctx->leaf_max;
    uint32_t flags = ctx->p.flags;
    ctx->p.flags &= ~SPH_FLAG_TIMING;  // probes are not part of the statistics
    int rc = SPH_OK;
    for (int a = 0; a < 2 && rc == SPH_OK; ++a)
        for (int b = 0; b < 3 && rc == SPH_OK; ++b) {
            ctx->tile_w = tws[a];
            if (ctx->adaptive) ctx->leaf_max = leaves[b];
            else ctx->p.cell_factor = cfs[b];
            SPH_CUDA(ctx, cudaEventRecord(ev[0], ctx->stream));
            rc = build_cells(ctx, parts);
            if (rc == SPH_ERR_H_EXCEEDS_CELL) {  // this cell factor cannot hold the largest h
                rc = SPH_OK;
                continue;
            }
            if (rc) break;
            SPH_CUDA(ctx, cudaEventRecord(ev[1], ctx->stream));
            SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_PREC, 0, sizeof(unsigned long long), ctx->stream));
            for (int r = 0; r < 2 && rc == SPH_OK; ++r) {
                SPH_CUDA(ctx, cudaMemsetAsync(ctx->active, 1, ctx->n, ctx->stream));
                rc = run_density_pass(ctx, parts, true, false);
                if (rc == SPH_OK) rc = ctx->adaptive ? tree_leaf_hcur(ctx, parts) : cell_reach(ctx);
                if (rc == SPH_OK) rc = run_force_pass(ctx, parts);
                if (rc == SPH_OK) SPH_CUDA(ctx, cudaEventRecord(ev[2 + r], ctx->stream));
            }
            if (rc) break;
            SPH_CUDA(ctx, cudaEventSynchronize(ev[3]));
            float t_build = 0.f, t_1 = 0.f, t_2 = 0.f;
            SPH_CUDA(ctx, cudaEventElapsedTime(&t_build, ev[0], ev[1]));
            SPH_CUDA(ctx, cudaEventElapsedTime(&t_1, ev[1], ev[2]));
            SPH_CUDA(ctx, cudaEventElapsedTime(&t_2, ev[2], ev[3]));
            const float ms = t_build + std::min(t_1, t_2);
            rc = read_counters(ctx);
            if (rc) break;
            const bool fits = ctx->h_counters[C_PREC] == 0;
            if ((fits && !best_fits) || (fits == best_fits && ms < best)) {
                best = ms;
                best_fits = fits;
                best_tw = tws[a];
                best_cf = ctx->p.cell_factor;
                best_leaf = ctx->leaf_max;
            }
        }
    ctx->p.flags = flags;
    if (rc) {
        for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
        return rc;
    }
    ctx->tile_w = best_tw;
    ctx->p.cell_factor = best_cf;
    ctx->leaf_max = best_leaf;
    ctx->tuned = true;
    if (!ctx->adaptive) {
        // staging of the pair passes: tile-box pruning alone, or after the per-axis
        // sorted sweep (SPH_FLAG_AXIS_SWEEP; Sec. 3.1, sorting) -- each a build (with
        // its 13 per-cell sorts) plus a density and a force pass, timed twice, the
        // faster repetition counting
        ctx->p.flags &= ~SPH_FLAG_TIMING;
        float ts[2] = {1e30f, 1e30f};
        for (int v = 0; v < 2 && rc == SPH_OK; ++v) {
            if (v) ctx->p.flags |= SPH_FLAG_AXIS_SWEEP;
            else ctx->p.flags &= ~SPH_FLAG_AXIS_SWEEP;
            for (int r = 0; r < 2 && rc == SPH_OK; ++r) {
                SPH_CUDA(ctx, cudaEventRecord(ev[0], ctx->stream));
                rc = build_cells(ctx, parts);
                if (rc) break;
                SPH_CUDA(ctx, cudaMemsetAsync(ctx->active, 1, ctx->n, ctx->stream));
                rc = run_density_pass(ctx, parts, true, false);
                if (rc == SPH_OK) rc = cell_reach(ctx);
                if (rc == SPH_OK) rc = run_force_pass(ctx, parts);
                if (rc) break;
                SPH_CUDA(ctx, cudaEventRecord(ev[1], ctx->stream));
                SPH_CUDA(ctx, cudaEventSynchronize(ev[1]));
                float ms = 0.f;
                SPH_CUDA(ctx, cudaEventElapsedTime(&ms, ev[0], ev[1]));
                ts[v] = std::min(ts[v], ms);
            }
        }
        const uint32_t sweep = ts[1] < ts[0] ? SPH_FLAG_AXIS_SWEEP : 0u;
        flags = (flags & ~SPH_FLAG_AXIS_SWEEP) | sweep;
        ctx->p.flags = (ctx->p.flags & ~SPH_FLAG_AXIS_SWEEP) | sweep;
    }
    if (rc == SPH_OK) rc = build_cells(ctx, parts);
    if (rc == SPH_OK && !ctx->adaptive) {
        // force pass: gather form or the symmetric variant (each unordered pair once),
        // each timed twice at these smoothing lengths, the faster repetition counting
        ctx->p.flags &= ~SPH_FLAG_TIMING;
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->active, 1, ctx->n, ctx->stream));
        rc = run_density_pass(ctx, parts, true, false);
        if (rc == SPH_OK) rc = cell_reach(ctx);
        float t[2] = {1e30f, 1e30f};
        for (int v = 0; v < 2 && rc == SPH_OK; ++v) {
            ctx->sym_force = v == 1;
            for (int r = 0; r < 2 && rc == SPH_OK; ++r) {
                SPH_CUDA(ctx, cudaEventRecord(ev[0], ctx->stream));
                rc = run_force_pass(ctx, parts);
                SPH_CUDA(ctx, cudaEventRecord(ev[1], ctx->stream));
                SPH_CUDA(ctx, cudaEventSynchronize(ev[1]));
                float ms = 0.f;
                SPH_CUDA(ctx, cudaEventElapsedTime(&ms, ev[0], ev[1]));
                t[v] = std::min(t[v], ms);
            }
        }
        ctx->sym_force = t[1] < t[0];
        ctx->p.flags = flags;
    }
    for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
    return rc;
}

// re-binnings of one density call (h outgrew the cells, or adaptive lists far too
// long); each restarts the h iteration with a fresh pass budget
constexpr int kMaxRebins = 32;

// Density targets of a call: every particle, or inside sph_step_bins the particles
// whose step ends now.
static int init_active(sph_ctx *ctx)
{
    const int64_t n = ctx->n;
    if (ctx->bin_mode)
        SPH_CUDA(ctx, cudaMemcpyAsync(ctx->active, ctx->bin_active, n, cudaMemcpyDeviceToDevice, ctx->stream));
    else
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->active, 1, n, ctx->stream));
    return SPH_OK;
}

// Tiles holding a target of ctx->active (the compaction runs only when the
// unconverged counter is nonzero: it is set to 1 here).
static int compact_bin_targets(sph_ctx *ctx)
{
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_UNCONV, 0, sizeof(unsigned long long), ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_UNCONV, 1, 1, ctx->stream));
    return ctx->adaptive ? compact_active_leaf_tiles(ctx) : compact_active_tiles(ctx);
}

static int do_density(sph_ctx *ctx, sph_particles *parts, int32_t *iters_out)
{
    if (!ctx->built) return fail(ctx, SPH_ERR_STATE, "sph_density needs sph_build_cells on the current positions");
    int n = (int)ctx->n;
    int iters = 0;
    int since = 0;     // passes since the last re-binning (each restarts the iteration)
    int rebinned = 0;  // re-binnings in this call
    unsigned long long unconv = 0;
    if (n > 0 && (ctx->p.flags & SPH_FLAG_AUTOTUNE) && !ctx->tuned) {
        // the schedules are timed at converged smoothing lengths, where the passes of
        // later steps run (an initial guess far from the root favoured schedules that
        // are slower in every later step): converge h with the current schedule first
        ctx->tuned = true;  // the inner call does not tune
        int rc = do_density(ctx, parts, nullptr);
        ctx->tuned = false;
        if (rc && rc != SPH_ERR_NOT_CONVERGED && rc != SPH_ERR_PRECISION) return rc;
        rc = autotune(ctx, parts);
        if (rc) return rc;
    }
    if (n > 0) {
        int rc = init_active(ctx);
        if (rc) return rc;
        rc = reset_h_brackets(ctx);
        if (rc) return rc;
        bool all_tiles = true;  // first pass (and after a rebuild): every tile
        if (ctx->bin_mode) {    // individual time-steps: only tiles with a target whose step ends
            rc = compact_bin_targets(ctx);
            if (rc) return rc;
            all_tiles = false;
        }
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_PREC, 0, sizeof(unsigned long long), ctx->stream));
        for (;;) {
            const bool last = since == ctx->p.max_h_iter - 1;
            SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_UNCONV, 0, 2 * sizeof(unsigned long long),
                                          ctx->stream));
            rc = run_density_pass(ctx, parts, last, !all_tiles);
            if (rc) return rc;
            ++iters;
            ++since;
            if (ctx->adaptive && !last) {
                rc = tree_shrink_count(ctx, parts);
                if (rc) return rc;
            }
            rc = read_counters(ctx);
            if (rc) return rc;
            unconv = ctx->h_counters[C_UNCONV];
            if (unconv == 0 || last) break;
            // adaptive: lists much longer than the current h need (1 leaf in 16)
            const bool shrunk = ctx->adaptive && ctx->h_counters[C_SHRINK] * 16 > (unsigned long long)ctx->tree.n_leaves;
            const bool outgrown = ctx->h_counters[C_HFLAG] != 0;
            if (outgrown && rebinned >= kMaxRebins) {
                char buf[160];
                snprintf(buf, sizeof buf, "smoothing lengths still outgrow the cells after %d re-binnings", rebinned);
                return fail(ctx, SPH_ERR_NOT_CONVERGED, buf);
            }
            if (outgrown || (shrunk && rebinned < kMaxRebins)) {
                // some h outgrew its cell: re-bin with the new h (permutes the arrays)
                cudaEvent_t end = nullptr;
                timer_begin(ctx, 2, &end);
                rc = build_cells(ctx, parts);
                timer_end(ctx, end);
                if (rc) return rc;
                ctx->st.rebuilds++;
                ++rebinned;
                since = 0;
                rc = init_active(ctx);
                if (rc) return rc;
                rc = reset_h_brackets(ctx);  // slots were permuted
                if (rc) return rc;
                SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_PREC, 0, sizeof(unsigned long long), ctx->stream));
                all_tiles = true;
                if (ctx->bin_mode) {
                    rc = compact_bin_targets(ctx);
                    if (rc) return rc;
                    all_tiles = false;
                }
            } else {
                rc = ctx->adaptive ? compact_active_leaf_tiles(ctx) : compact_active_tiles(ctx);
                if (rc) return rc;
                all_tiles = false;
            }
        }
        rc = sync_h(ctx, parts);
        if (rc) return rc;
    }
    if (iters_out) *iters_out = iters;
    ctx->density_valid = true;
    ctx->hydro_valid = false;
    if (unconv) {
        char buf[160];
        snprintf(buf, sizeof buf, "%llu smoothing lengths not converged after %d passes", unconv, iters);
        return fail(ctx, SPH_ERR_NOT_CONVERGED, buf);
    }
    if (n > 0 && ctx->h_counters[C_PREC]) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "uniform grid: some h is below cell side / %d, beyond what FP32 cell-relative positions "
                 "resolve at the density tolerance (use SPH_FLAG_ADAPTIVE)", SPH_FRAME_RATIO);
        return fail(ctx, SPH_ERR_PRECISION, buf);
    }
    return SPH_OK;
}

static int do_force(sph_ctx *ctx, sph_particles *parts)
{
    if (!ctx->density_valid) return fail(ctx, SPH_ERR_STATE, "sph_force needs sph_density on the current state");
    if (ctx->n > 0) {
        // uniform grid: reach of every cell for r < max(h_i, h_j) (adaptive cells
        // prune every source with its own h)
        int rc = ctx->adaptive ? tree_leaf_hcur(ctx, parts) : cell_reach(ctx);
        if (rc) return rc;
        if (ctx->bin_mode) {  // individual time-steps: the tiles of the targets whose step ends
            rc = init_active(ctx);
            if (rc) return rc;
            rc = compact_bin_targets(ctx);
            if (rc) return rc;
        }
        rc = run_force_pass(ctx, parts, ctx->bin_mode);
        if (rc) return rc;
    }
    ctx->hydro_valid = true;
    return SPH_OK;
}

static int do_build(sph_ctx *ctx, sph_particles *parts)
{
    cudaEvent_t end = nullptr;
    timer_begin(ctx, 2, &end);
    int rc = build_cells(ctx, parts);
    timer_end(ctx, end);
    ctx->hydro_valid = false;
    return rc;
}

// do_density inside a compound call: SPH_ERR_PRECISION leaves written results that
// only miss the density tolerance, and SPH_ERR_NOT_CONVERGED after the pass budget
// leaves every particle with results at its last iterate inside cells that hold it,
// so the call goes on (a step completes, with a consistent state) and reports the
// status at its end.  h beyond the cells after the re-binnings stops the call.
static int density_in_call(sph_ctx *ctx, sph_particles *parts)
{
    const int rc = do_density(ctx, parts, nullptr);
    const bool soft = rc == SPH_ERR_PRECISION || (rc == SPH_ERR_NOT_CONVERGED && ctx->h_counters[C_HFLAG] == 0);
    if (!soft) return rc;
    if (!ctx->soft_rc) {
        ctx->soft_rc = rc;
        ctx->soft_msg = ctx->err;
    }
    return SPH_OK;
}

// the status of a compound call: its own error, else the deferred one
static int finish_call(sph_ctx *ctx, int rc)
{
    if (rc == SPH_OK && ctx->soft_rc) rc = fail(ctx, ctx->soft_rc, ctx->soft_msg);
    ctx->soft_rc = 0;
    return rc;
}

// build -> density -> force.  in_step: the hydro pass inside a step, where the
// previous pass's outputs feed the learned h guess and the sample collection.
// Inside sph_step_host: the device-to-host copies of the results the rest of the step
// no longer writes, issued on the copy stream behind an event of the compute stream,
// so that they overlap the passes that follow.  After the density passes (and any
// re-binning they caused) the order, positions, masses, h and the density outputs are
// final; after the force pass the accelerations, du/dt and v_sig.
static int early_copies(sph_ctx *ctx, const sph_particles *d, int stage)
{
    sph_particles *hp = ctx->host_out;
    if (!hp || ctx->n <= 0) return SPH_OK;
    const size_t b8 = 8 * (size_t)ctx->n, b4 = 4 * (size_t)ctx->n;
    cudaStream_t cs = ctx->copy_stream;
    SPH_CUDA(ctx, cudaEventRecord(ctx->copy_ev, ctx->stream));
    SPH_CUDA(ctx, cudaStreamWaitEvent(cs, ctx->copy_ev, 0));
    if (stage == 0) {
        double *s64[][2] = {{hp->x, d->x}, {hp->y, d->y}, {hp->z, d->z}};
        for (auto &q : s64) SPH_CUDA(ctx, cudaMemcpyAsync(q[0], q[1], b8, cudaMemcpyDeviceToHost, cs));
        float *s32[][2] = {{hp->m, d->m}, {hp->h, d->h},     {hp->rho, d->rho}, {hp->P, d->P},
                           {hp->c, d->c}, {hp->f, d->f}, {hp->divv, d->divv}, {hp->curl, d->curl}};
        for (auto &q : s32) SPH_CUDA(ctx, cudaMemcpyAsync(q[0], q[1], b4, cudaMemcpyDeviceToHost, cs));
        SPH_CUDA(ctx, cudaMemcpyAsync(hp->n_ngb, d->n_ngb, b4, cudaMemcpyDeviceToHost, cs));
    } else {
        float *s32[][2] = {{hp->ax, d->ax}, {hp->ay, d->ay}, {hp->az, d->az}, {hp->dudt, d->dudt},
                           {hp->vsig, d->vsig}};
        for (auto &q : s32) SPH_CUDA(ctx, cudaMemcpyAsync(q[0], q[1], b4, cudaMemcpyDeviceToHost, cs));
    }
    return SPH_OK;
}

static int hydro(sph_ctx *ctx, sph_particles *parts, bool in_step = false)
{
    int rc = do_build(ctx, parts);
    if (rc) return rc;
    const bool predict = in_step && (ctx->p.flags & SPH_FLAG_HPREDICT);
    const bool collect = in_step && ctx->hp.col_feats;
    if (predict) {
        rc = hp_apply_step(ctx, parts);
        if (rc) return rc;
    } else if (collect) {
        rc = hp_features(ctx, parts);
        if (rc) return rc;
    }
    rc = density_in_call(ctx, parts);
    if (rc) return rc;
    if (collect) {
        rc = hp_collect(ctx, parts);
        if (rc) return rc;
    }
    if (in_step) {
        rc = early_copies(ctx, parts, 0);
        if (rc) return rc;
    }
    rc = do_force(ctx, parts);
    if (rc) return rc;
    return in_step ? early_copies(ctx, parts, 1) : SPH_OK;
}

static int do_step(sph_ctx *ctx, sph_particles *parts, double dt, double *dt_used, sph_conserved *out)
{
    int rc;
    ctx->predict = false;
    if (!ctx->hydro_valid) {
        rc = hydro(ctx, parts);
        if (rc) return rc;
    }
    if (dt > 0) {
        rc = set_dt(ctx, dt);
        if (rc) return rc;
    } else {
        rc = cfl_dt(ctx, parts, &dt);  // also leaves dt in *d_dt
        if (rc) return rc;
        if (!isfinite(dt)) return fail(ctx, SPH_ERR_INVALID_ARG, "no signal velocity: pass an explicit dt");
    }
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_FLOORS, 0, sizeof(unsigned long long), ctx->stream));
    rc = kick(ctx, parts);
    if (rc) return rc;
    rc = drift(ctx, parts);
    if (rc) return rc;
    // the hydro pass sees v and u predicted to the end of the step (vel4 / upred)
    ctx->predict = true;
    rc = hydro(ctx, parts, true);
    ctx->predict = false;
    if (rc) return rc;
    rc = kick(ctx, parts);
    if (rc) return rc;
    if (dt_used) *dt_used = dt;
    if (out) {
        rc = conserved_device(ctx, parts);
        if (rc) return rc;
        rc = conserved_read(ctx, out);
        if (rc) return rc;
        rc = cfl_dt(ctx, parts, &out->dt_next);
        if (rc) return rc;
    }
    return SPH_OK;
}

// ------------------------------------------------------- individual time-steps

// Advance by dt_max with each particle on its own power-of-two step (the leapfrog of
// do_step per particle).  Time runs on an integer grid of unit dt_max / 2^L.  All
// particles open a step at 0; then, from one step end to the next (the earliest
// step end over the particles): every particle drifts; the cells are built (the
// build also carries the bins, the steps and the kept density outputs along, and
// predicts every particle's v and u to the current time); the particles whose step
// ends now get density (with the h iteration) and force against all particles,
// take their closing half kick, a new bin (raised by the limiter, which may also
// wake sleeping neighbours, with SPH_FLAG_BIN_LIMITER), and (before dt_max) open
// their next step with its half kick.  The others keep h, rho, P, c, f, B, a,
// du/dt and vsig from their last update.  At dt_max every particle is synchronised
// again, with current a and du/dt.
static int do_step_bins(sph_ctx *ctx, sph_particles *parts, double dt_max, int levels, sph_conserved *out,
                        sph_bin_stats *bs)
{
    int rc;
    ctx->predict = false;
    // a synchronised start with current accelerations, and the schedule tuned before
    // (the tuner's probe passes would overwrite what inactive particles keep)
    if (!ctx->hydro_valid || ((ctx->p.flags & SPH_FLAG_AUTOTUNE) && !ctx->tuned)) {
        rc = hydro(ctx, parts);
        if (rc) return rc;
    }
    rc = alloc_bins(ctx);
    if (rc) return rc;
    const bool limiter = (ctx->p.flags & SPH_FLAG_BIN_LIMITER) != 0;
    const int64_t end = (int64_t)1 << levels;
    const double unit = ldexp(dt_max, -levels);
    ctx->bin_levels = levels;
    ctx->bin_unit = unit;
    ctx->bin_now = 0;
    const Counter zeroed[] = {C_FLOORS, C_BINOVER, C_LIMITED, C_WOKEN};
    for (Counter k : zeroed)
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + k, 0, sizeof(unsigned long long), ctx->stream));
    int64_t substeps = 0, updates = 0, sweeps = 0;
    ctx->bin_mode = true;
    auto body = [&]() -> int {
        // every particle opens a step at 0
        int r;
        if (limiter && ctx->n > 0) {
            // the limiter's neighbourhoods come from the cells: build them on the
            // positions as they are now (the kept density outputs follow the
            // permutation; every step is still empty, so nothing is predicted)
            SPH_CUDA(ctx, cudaMemsetAsync(ctx->bin_st, 0, sizeof(int2) * (size_t)ctx->n, ctx->stream));
            SPH_CUDA(ctx, cudaMemsetAsync(ctx->bin_active, 0, (size_t)ctx->n, ctx->stream));
            SPH_CUDA(ctx, cudaMemsetAsync(ctx->bins, 0, (size_t)ctx->n, ctx->stream));
            r = do_build(ctx, parts);
            if (r) return r;
        }
        r = bin_assign(ctx, parts, true, dt_max);
        if (r) return r;
        if (limiter) {
            r = bin_limit(ctx, parts, true, &sweeps);
            if (r) return r;
        }
        r = bin_open(ctx, parts, true, limiter);
        if (r) return r;
        r = bin_kick(ctx, parts, true);
        if (r) return r;
        int64_t s = 0;
        while (s < end) {
            int deepest = 0;
            unsigned long long over = 0;
            int64_t s_next = end;
            r = bin_max_read(ctx, &deepest, &over, &s_next);
            if (r) return r;
            if (ctx->n == 0) s_next = end;  // nothing steps: one step end, at dt_max
            if (s_next <= s || s_next > end) return fail(ctx, SPH_ERR_STATE, "individual time-steps: bad step end");
            r = set_dt(ctx, (double)(s_next - s) * unit);
            if (r) return r;
            r = drift(ctx, parts);
            if (r) return r;
            s = s_next;
            ctx->bin_now = s;
            unsigned long long n_act = 0;
            r = bin_active(ctx, &n_act);
            if (r) return r;
            ++substeps;
            updates += (int64_t)n_act;
            r = do_build(ctx, parts);
            if (r) return r;
            r = density_in_call(ctx, parts);
            if (r) return r;
            r = do_force(ctx, parts);
            if (r) return r;
            r = bin_kick(ctx, parts, false);  // closing half kick of the steps that end now
            if (r) return r;
            r = bin_assign(ctx, parts, false, dt_max);
            if (r) return r;
            if (s < end) {
                if (limiter) {
                    r = bin_limit(ctx, parts, false, &sweeps);
                    if (r) return r;
                }
                r = bin_open(ctx, parts, false, limiter);
                if (r) return r;
                r = bin_kick(ctx, parts, false);  // opening half kick of their next steps
                if (r) return r;
            }
        }
        return SPH_OK;
    };
    rc = body();
    ctx->bin_mode = false;
    if (rc) return rc;
    ctx->hydro_valid = true;  // all particles were active at dt_max
    if (bs) {
        memset(bs, 0, sizeof *bs);
        bs->substeps = substeps;
        bs->updates = updates;
        std::vector<int8_t> hb((size_t)std::max<int64_t>(ctx->n, 1));
        if (ctx->n > 0)
            SPH_CUDA(ctx, cudaMemcpyAsync(hb.data(), ctx->bins, (size_t)ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
        int deepest = 0;
        unsigned long long over = 0;
        rc = bin_max_read(ctx, &deepest, &over, nullptr);  // synchronises the stream
        if (rc) return rc;
        bs->cfl_over = (int64_t)over;
        SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_counters + C_LIMITED, ctx->counters + C_LIMITED,
                                      2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
        SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        bs->limited = (int64_t)ctx->h_counters[C_LIMITED];
        bs->woken = (int64_t)ctx->h_counters[C_WOKEN];
        bs->limit_sweeps = sweeps;
        for (int64_t i = 0; i < ctx->n; ++i) bs->bin_count[hb[(size_t)i]]++;
    }
    if (out) {
        rc = conserved_device(ctx, parts);
        if (rc) return rc;
        rc = conserved_read(ctx, out);
        if (rc) return rc;
        rc = cfl_dt(ctx, parts, &out->dt_next);
        if (rc) return rc;
    }
    return SPH_OK;
}

// --------------------------------------------------------- graph-captured steps

// flags of one step, ORed into C_GFLAGS: 1 = unconverged h, 2 = h beyond the cells,
// 4 = h below what the uniform grid's FP32 frame resolves, 8 = a tensor-core wait of
// the learned-h inference ran out
__global__ void k_step_flags(unsigned long long *c)
{
    unsigned long long f = 0;
    if (c[C_UNCONV]) f |= 1ull;
    if (c[C_HFLAG]) f |= 2ull;
    if (c[C_PREC]) f |= 4ull;
    if (c[C_TCERR]) f |= 8ull;
    c[C_GFLAGS] |= f;
}

// One KDK step with no host synchronisation (the plan of the cell grids is fixed).
static int graph_step(sph_ctx *ctx, sph_particles *parts, double dt, int passes)
{
    int rc = dt > 0 ? set_dt(ctx, dt) : cfl_dt_device(ctx, parts);
    if (rc) return rc;
    rc = kick(ctx, parts);
    if (rc) return rc;
    rc = drift(ctx, parts);
    if (rc) return rc;
    ctx->predict = true;
    rc = build_planned(ctx, parts);
    if (rc) return rc;
    if (ctx->p.flags & SPH_FLAG_HPREDICT) {
        rc = hp_apply_step(ctx, parts);
        if (rc) return rc;
    }
    const int n = (int)ctx->n;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->active, 1, n, ctx->stream));
    rc = reset_h_brackets(ctx);
    if (rc) return rc;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_UNCONV, 0, 2 * sizeof(unsigned long long), ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_PREC, 0, sizeof(unsigned long long), ctx->stream));
    for (int p = 0; p < passes; ++p) {
        if (p > 0) {
            rc = ctx->adaptive ? compact_active_leaf_tiles(ctx) : compact_active_tiles(ctx);
            if (rc) return rc;
            SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_UNCONV, 0, sizeof(unsigned long long), ctx->stream));
        }
        rc = run_density_pass(ctx, parts, p == passes - 1, p > 0);
        if (rc) return rc;
    }
    k_step_flags<<<1, 1, 0, ctx->stream>>>(ctx->counters);
    SPH_LAUNCH(ctx, "step flags");
    rc = sync_h(ctx, parts);
    if (rc) return rc;
    rc = ctx->adaptive ? tree_leaf_hcur(ctx, parts) : cell_reach(ctx);  // adaptive: sources' h per leaf
    if (rc) return rc;
    rc = run_force_pass(ctx, parts);
    if (rc) return rc;
    ctx->predict = false;
    rc = kick(ctx, parts);
    if (rc) return rc;
    return conserved_device(ctx, parts);
}

static int do_steps(sph_ctx *ctx, sph_particles *parts, int n_steps, double dt, double *dt_last,
                    sph_conserved *out)
{
    int rc;
    ctx->predict = false;
    if (!ctx->hydro_valid) {
        rc = hydro(ctx, parts);
        if (rc) return rc;
    }
    if (!(dt > 0)) {  // a CFL step must exist before the run starts
        double d0 = 0;
        rc = cfl_dt(ctx, parts, &d0);
        if (rc) return rc;
        if (!isfinite(d0)) return fail(ctx, SPH_ERR_INVALID_ARG, "no signal velocity: pass an explicit dt");
    }
    // the cell plan is fixed for the whole run; an existing plan (and the graph
    // captured for it) is kept while it still suits the particles
    rc = read_box_max_h(ctx, parts);
    if (rc) return rc;
    if (ctx->adaptive) {
        // adaptive cells: a particle's neighbours lie in the 27 top cells around it,
        // so the fixed top grid keeps a margin for h to grow during the run: sides
        // >= 1.15 max h (larger top cells make slower trees: measured 7 % per step on
        // the batched boxes at 1.6)
        bool good = ctx->planned;
        for (int b = 0; b < ctx->n_boxes && good; ++b)
            if (ctx->box_off[b + 1] > ctx->box_off[b] && 1.15 * (double)ctx->h_box_hmax[b] > ctx->h_boxes[b].L64)
                good = false;
        if (!good) {
            const float cf = ctx->p.cell_factor;
            ctx->p.cell_factor = std::max(cf, 1.15f);
            rc = plan_from_hmax(ctx);
            ctx->p.cell_factor = cf;
            if (rc) return rc;
        }
    } else if (!plan_still_good(ctx)) {
        rc = plan_from_hmax(ctx);
        if (rc) return rc;
    }
    const int passes = std::max(1, std::min(ctx->p.max_h_iter, 6));
    if (ctx->p.flags & SPH_FLAG_HPREDICT) {  // allocate before any capture
        rc = hp_ensure(ctx, std::max<int64_t>(ctx->n, 1));
        if (rc) return rc;
    }
    // adaptive cells: the captured build keeps its sizes on the device, in arrays of
    // fixed capacity allocated here
    uint64_t tree_sig = 0;
    if (ctx->adaptive && ctx->n > 0) {
        rc = tree_prepare_device(ctx, &tree_sig);
        if (rc) return rc;
    }
    // capture one step on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is then launched on the caller's
    // stream.  The timing flag is suspended while capturing.  A graph captured for
    // the same arrays, dt mode and launch shapes is reused.
    if (ctx->sym_force && !ctx->adaptive) {  // the symmetric force pass's slots, before any capture
        rc = ensure_sym(ctx);
        if (rc) return rc;
    }
    sph_ctx::GraphKey key{*parts, dt > 0 ? dt : 0.0, ctx->n, ctx->grid.n_cells, ctx->grid.key_bits, passes, ctx->tile_w,
                          tree_sig, ctx->sym_force};
    if (!ctx->step_exec || !(key == ctx->graph_key)) {
        if (!ctx->cap_stream) SPH_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        const uint32_t flags = ctx->p.flags;
        ctx->p.flags &= ~SPH_FLAG_TIMING;
        SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cudaStream_t user = ctx->stream;
        ctx->stream = ctx->cap_stream;
        cudaError_t ce = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) {
            ctx->stream = user;
            ctx->p.flags = flags;
            return cuda_fail(ctx, ce, "begin capture");
        }
        const int64_t launches0 = ctx->st.kernel_launches;
        const int64_t passes0 = ctx->st.density_passes, fpasses0 = ctx->st.force_passes;
        ctx->tree.device_sized = ctx->adaptive;
        rc = graph_step(ctx, parts, dt, passes);
        ctx->tree.device_sized = false;
        ctx->graph_launches = ctx->st.kernel_launches - launches0;
        ctx->st.kernel_launches = launches0;  // capture launched nothing
        ctx->st.density_passes = passes0;
        ctx->st.force_passes = fpasses0;
        cudaGraph_t graph = nullptr;
        ce = cudaStreamEndCapture(ctx->stream, &graph);
        ctx->stream = user;
        ctx->p.flags = flags;
        ctx->predict = false;
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "graph capture");
        if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
        ctx->step_exec = nullptr;
        ce = cudaGraphInstantiate(&ctx->step_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "graph instantiate");
        ctx->graph_key = key;
        ctx->g_keys = ctx->keys;
        ctx->g_keys_alt = ctx->keys_alt;
        ctx->g_vals = ctx->vals;
        ctx->g_vals_alt = ctx->vals_alt;
        ctx->g_keys64 = ctx->keys64;
        ctx->g_keys64_alt = ctx->keys64_alt;
    }
    if (n_steps == 0) return SPH_OK;  // prepared: hydro, plan and graph are ready
    const int64_t per_step = ctx->graph_launches;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_FLOORS, 0, sizeof(unsigned long long), ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_GFLAGS, 0, sizeof(unsigned long long), ctx->stream));
    for (int k = 0; k < n_steps; ++k) SPH_CUDA(ctx, cudaGraphLaunch(ctx->step_exec, ctx->stream));
    // host builds since the capture may have swapped the sort buffers back
    ctx->keys = ctx->g_keys;
    ctx->keys_alt = ctx->g_keys_alt;
    ctx->vals = ctx->g_vals;
    ctx->vals_alt = ctx->g_vals_alt;
    ctx->keys64 = ctx->g_keys64;
    ctx->keys64_alt = ctx->g_keys64_alt;
    ctx->st.kernel_launches += per_step * n_steps;
    ctx->st.density_passes += (int64_t)passes * n_steps;
    ctx->st.force_passes += n_steps;
    ctx->st.graph_steps += n_steps;
    ctx->hydro_valid = true;
    ctx->density_valid = true;
    ctx->built = true;
    sph_conserved tmp;
    rc = conserved_read(ctx, out ? out : &tmp);
    if (rc) return rc;
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_dt, ctx->d_dt, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (dt_last) *dt_last = *ctx->h_dt;
    if (out) {
        double nd = 0;
        rc = cfl_dt(ctx, parts, &nd);
        if (rc) return rc;
        out->dt_next = nd;
    }
    if (ctx->adaptive) {
        rc = tree_read_device(ctx);
        if (rc) return rc;
    }
    const unsigned long long gf = ctx->h_counters[C_GFLAGS];
    if (gf & 8ull) return fail(ctx, SPH_ERR_TIMEOUT, "predictor: a tensor-core wait ran out in a captured step");
    if (gf & 2ull) return fail(ctx, SPH_ERR_H_EXCEEDS_CELL, "some h grew beyond twice the planned cell side");
    if (gf & 1ull) return fail(ctx, SPH_ERR_NOT_CONVERGED, "smoothing lengths not converged in a captured step");
    if (gf & 4ull) return fail(ctx, SPH_ERR_PRECISION, "uniform grid: some h fell below cell side / SPH_FRAME_RATIO");
    return SPH_OK;
}

}  // namespace sph

using namespace sph;

extern "C" {

int sph_default_params(sph_params *p)
{
    if (!p) return SPH_ERR_INVALID_ARG;
    memset(p, 0, sizeof *p);
    p->n = 0;
    p->box_size = 1.0;
    p->gamma = 5.f / 3.f;
    p->n_ngb = 48.f;
    p->h_tol = 1e-4f;
    p->alpha_visc = 0.8f;
    p->cfl = 0.1f;
    p->cell_factor = 1.1f;
    p->max_h_iter = 30;
    p->use_balsara = 1;
    p->kernel = 0;
    p->flags = 0;
    return SPH_OK;
}

int sph_init(sph_ctx **out, const sph_params *p, int device, void *cuda_stream)
{
    if (!out) return SPH_ERR_INVALID_ARG;
    *out = nullptr;
    if (!p) return SPH_ERR_INVALID_ARG;
    std::string why;
    if (check_params(p, why)) return SPH_ERR_INVALID_ARG;
    sph_ctx *c = new sph_ctx();
    c->p = *p;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->n = p->n;
    c->tile_w = p->tile_width == 32 ? 32 : 16;
    c->adaptive = (p->flags & SPH_FLAG_ADAPTIVE) != 0;
    c->sym_force = (p->flags & SPH_FLAG_SYMMETRIC) != 0 && !c->adaptive;
    c->leaf_max = p->leaf_max > 0 ? p->leaf_max : 64;
    c->h_guess_pending = c->adaptive && (p->flags & SPH_FLAG_TREE_H_GUESS);
    c->n_boxes = p->n_boxes > 1 ? p->n_boxes : 1;
    if (p->n_boxes > 1) c->box_off.assign(p->box_offsets, p->box_offsets + p->n_boxes + 1);
    else c->box_off = {0, p->n};
    c->p.box_offsets = nullptr;  // the caller's array need not outlive sph_init
    int rc = SPH_OK;
    auto bail = [&](int code) {
        sph_destroy(c);
        return code;
    };
    if (cudaSetDevice(device) != cudaSuccess) return bail(SPH_ERR_CUDA);
    if (cudaMalloc(&c->counters, C_NCOUNTERS * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&c->h_counters, C_NCOUNTERS * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_scalars, 8 * sizeof(float)) != cudaSuccess ||
        cudaMallocHost(&c->h_scalars, 8 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&c->d_red, red_scratch_doubles() * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->h_red, 8 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->scan_aux, kScanAuxCap * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&c->n_tiles, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->n_act_tiles, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_dt, sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->h_dt, sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_boxes, sizeof(BoxDev) * c->n_boxes) != cudaSuccess ||
        cudaMallocHost(&c->h_boxes, sizeof(BoxDev) * c->n_boxes) != cudaSuccess ||
        cudaMalloc(&c->d_box_hmax, sizeof(float) * c->n_boxes) != cudaSuccess ||
        cudaMallocHost(&c->h_box_hmax, sizeof(float) * c->n_boxes) != cudaSuccess ||
        cudaMalloc(&c->d_box_off, sizeof(int64_t) * (c->n_boxes + 1)) != cudaSuccess)
        return bail(SPH_ERR_CUDA);
    if (cudaMemcpy(c->d_box_off, c->box_off.data(), sizeof(int64_t) * (c->n_boxes + 1), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return bail(SPH_ERR_CUDA);
    if (cudaMemsetAsync(c->counters, 0, C_NCOUNTERS * sizeof(unsigned long long), c->stream) != cudaSuccess)
        return bail(SPH_ERR_CUDA);
    rc = alloc_particles(c, c->n);
    if (rc) return bail(rc);
    *out = c;
    return SPH_OK;
}

int sph_set_n(sph_ctx *ctx, int64_t n)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (n < 0 || n >= (1ll << 31)) return fail(ctx, SPH_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    if (ctx->n_boxes > 1) return fail(ctx, SPH_ERR_STATE, "sph_set_n applies to single-box contexts");
    ctx->box_off = {0, n};
    SPH_CUDA(ctx, cudaMemcpy(ctx->d_box_off, ctx->box_off.data(), sizeof(int64_t) * 2, cudaMemcpyHostToDevice));
    if (n > ctx->cap) {
        int rc = alloc_particles(ctx, n);
        if (rc) return rc;
    }
    ctx->n = n;
    ctx->p.n = n;
    ctx->built = ctx->density_valid = ctx->hydro_valid = false;
    ctx->ids_valid = false;
    return SPH_OK;
}

int sph_build_cells(sph_ctx *ctx, sph_particles *parts)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!parts || (ctx->n > 0 && !parts_ok(parts))) return fail(ctx, SPH_ERR_INVALID_ARG, "null particle array");
    ctx->predict = false;
    return do_build(ctx, parts);
}

int sph_density(sph_ctx *ctx, sph_particles *parts, int32_t *iters_out)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!parts || (ctx->n > 0 && !parts_ok(parts))) return fail(ctx, SPH_ERR_INVALID_ARG, "null particle array");
    return do_density(ctx, parts, iters_out);
}

int sph_force(sph_ctx *ctx, sph_particles *parts)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!parts || (ctx->n > 0 && !parts_ok(parts))) return fail(ctx, SPH_ERR_INVALID_ARG, "null particle array");
    return do_force(ctx, parts);
}

int sph_step(sph_ctx *ctx, sph_particles *parts, double dt, double *dt_used, sph_conserved *out)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!parts || (ctx->n > 0 && !parts_ok(parts))) return fail(ctx, SPH_ERR_INVALID_ARG, "null particle array");
    if (!isfinite(dt)) return fail(ctx, SPH_ERR_INVALID_ARG, "dt must be finite");
    if ((ctx->p.flags & SPH_FLAG_HPREDICT) && !ctx->hp.ready)
        return fail(ctx, SPH_ERR_STATE, "SPH_FLAG_HPREDICT without predictor weights");
    ctx->soft_rc = 0;
    return finish_call(ctx, do_step(ctx, parts, dt, dt_used, out));
}

int sph_step_bins(sph_ctx *ctx, sph_particles *parts, double dt_max, int32_t n_bins, sph_conserved *out,
                  sph_bin_stats *stats)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!parts || (ctx->n > 0 && !parts_ok(parts))) return fail(ctx, SPH_ERR_INVALID_ARG, "null particle array");
    if (!(dt_max > 0) || !isfinite(dt_max)) return fail(ctx, SPH_ERR_INVALID_ARG, "dt_max must be finite and > 0");
    if (n_bins < 0 || n_bins > SPH_MAX_BINS) return fail(ctx, SPH_ERR_INVALID_ARG, "n_bins must be in [0, SPH_MAX_BINS]");
    ctx->soft_rc = 0;
    return finish_call(ctx, do_step_bins(ctx, parts, dt_max, n_bins, out, stats));
}

int sph_get_bins(sph_ctx *ctx, int8_t *dev_bins)
{
    if (!ctx || !dev_bins) return SPH_ERR_INVALID_ARG;
    if (!ctx->bins) return fail(ctx, SPH_ERR_STATE, "no sph_step_bins call yet");
    if (ctx->n > 0)
        SPH_CUDA(ctx, cudaMemcpyAsync(dev_bins, ctx->bins, (size_t)ctx->n, cudaMemcpyDeviceToDevice, ctx->stream));
    return SPH_OK;
}

int sph_steps(sph_ctx *ctx, sph_particles *parts, int32_t n_steps, double dt, double *dt_last, sph_conserved *out)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!parts || (ctx->n > 0 && !parts_ok(parts))) return fail(ctx, SPH_ERR_INVALID_ARG, "null particle array");
    if (!isfinite(dt)) return fail(ctx, SPH_ERR_INVALID_ARG, "dt must be finite");
    if (n_steps < 0) return fail(ctx, SPH_ERR_INVALID_ARG, "n_steps must be >= 0");
    if ((ctx->p.flags & SPH_FLAG_HPREDICT) && !ctx->hp.ready)
        return fail(ctx, SPH_ERR_STATE, "SPH_FLAG_HPREDICT without predictor weights");
    ctx->soft_rc = 0;
    return finish_call(ctx, do_steps(ctx, parts, n_steps, dt, dt_last, out));
}

int sph_step_host(sph_ctx *ctx, sph_particles *hp, double dt, double *dt_used, sph_conserved *out)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!hp || (ctx->n > 0 && !parts_ok(hp))) return fail(ctx, SPH_ERR_INVALID_ARG, "null particle array");
    if (!isfinite(dt)) return fail(ctx, SPH_ERR_INVALID_ARG, "dt must be finite");
    const int64_t n = ctx->n;
    if (ctx->mirror_cap < n || !ctx->mirror_block) {
        cudaFree(ctx->mirror_block);
        ctx->mirror_block = nullptr;
        int64_t cap = std::max<int64_t>(n, 1);
        size_t bytes = (size_t)cap * (6 * 8 + 15 * 4) + 32 * 256;
        SPH_CUDA(ctx, cudaMalloc(&ctx->mirror_block, bytes));
        char *b = (char *)ctx->mirror_block;
        auto take = [&](size_t sz) {
            char *r = b;
            b += (sz + 255) & ~(size_t)255;
            return r;
        };
        sph_particles &m = ctx->dev_mirror;
        m.x = (double *)take(8 * cap);
        m.y = (double *)take(8 * cap);
        m.z = (double *)take(8 * cap);
        m.vx = (double *)take(8 * cap);
        m.vy = (double *)take(8 * cap);
        m.vz = (double *)take(8 * cap);
        float **f32[] = {&m.m, &m.u, &m.h, &m.rho, &m.P, &m.c, &m.f, &m.divv, &m.curl,
                         &m.ax, &m.ay, &m.az, &m.dudt, &m.vsig};
        for (float **q : f32) *q = (float *)take(4 * cap);
        m.n_ngb = (int32_t *)take(4 * cap);
        ctx->mirror_cap = cap;
    }
    if (!ctx->copy_stream) {
        SPH_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        SPH_CUDA(ctx, cudaEventCreateWithFlags(&ctx->copy_ev, cudaEventDisableTiming));
    }
    sph_particles &d = ctx->dev_mirror;
    cudaStream_t s = ctx->stream;
    const size_t b8 = 8 * (size_t)n, b4 = 4 * (size_t)n;
    // inputs of a step: the state and the rates from the previous hydro pass
    double *in64[][2] = {{d.x, hp->x}, {d.y, hp->y}, {d.z, hp->z}, {d.vx, hp->vx}, {d.vy, hp->vy}, {d.vz, hp->vz}};
    float *in32[][2] = {{d.m, hp->m},   {d.u, hp->u},   {d.h, hp->h},       {d.ax, hp->ax},
                        {d.ay, hp->ay}, {d.az, hp->az}, {d.dudt, hp->dudt}, {d.vsig, hp->vsig}};
    for (auto &q : in64) SPH_CUDA(ctx, cudaMemcpyAsync(q[0], q[1], b8, cudaMemcpyHostToDevice, s));
    for (auto &q : in32) SPH_CUDA(ctx, cudaMemcpyAsync(q[0], q[1], b4, cudaMemcpyHostToDevice, s));
    // the device copies replace whatever the context held: cells must be rebuilt
    ctx->built = ctx->density_valid = false;
    ctx->soft_rc = 0;
    // results go back as soon as the step is done with them (the copy stream), the
    // velocities and u (closing kick) at the end
    ctx->host_out = hp;
    int rc = do_step(ctx, &d, dt, dt_used, out);
    ctx->host_out = nullptr;
    if (rc) {
        cudaStreamSynchronize(ctx->copy_stream);  // (nothing in flight is left reading the mirror)
        ctx->soft_rc = 0;
        return rc;
    }
    double *end64[][2] = {{d.vx, hp->vx}, {d.vy, hp->vy}, {d.vz, hp->vz}};
    for (auto &q : end64) SPH_CUDA(ctx, cudaMemcpyAsync(q[1], q[0], b8, cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaMemcpyAsync(hp->u, d.u, b4, cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->copy_stream));
    return finish_call(ctx, SPH_OK);
}

int sph_gravity_p2p(sph_ctx *ctx, double G, double eps, float *ax, float *ay, float *az, float *phi)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!isfinite(G) || !isfinite(eps) || eps < 0.0)
        return fail(ctx, SPH_ERR_INVALID_ARG, "G and eps must be finite, eps >= 0");
    if (ctx->n > 0 && (!ax || !ay || !az)) return fail(ctx, SPH_ERR_INVALID_ARG, "null acceleration array");
    if (ctx->adaptive)
        return fail(ctx, SPH_ERR_STATE, "the gravity near field runs on the uniform grid (not SPH_FLAG_ADAPTIVE)");
    if (!ctx->built) return fail(ctx, SPH_ERR_STATE, "sph_gravity_p2p needs sph_build_cells on the current positions");
    if (ctx->n == 0) return SPH_OK;
    return run_gravity_pass(ctx, G, eps, ax, ay, az, phi);
}

int sph_get_permutation(sph_ctx *ctx, int64_t *dev_perm)
{
    if (!ctx || !dev_perm) return SPH_ERR_INVALID_ARG;
    if (!ctx->ids_valid) return fail(ctx, SPH_ERR_STATE, "no cell build yet");
    SPH_CUDA(ctx, cudaMemcpyAsync(dev_perm, ctx->ids, sizeof(int64_t) * ctx->n, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    return SPH_OK;
}

int sph_reset_ids(sph_ctx *ctx)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    ctx->ids_valid = false;
    return SPH_OK;
}

int sph_get_cell_keys(sph_ctx *ctx, int32_t *dev_keys)
{
    if (!ctx || !dev_keys) return SPH_ERR_INVALID_ARG;
    if (!ctx->built) return fail(ctx, SPH_ERR_STATE, "no cell build on the current positions");
    return ctx->adaptive ? tree_cell_keys_out(ctx, dev_keys) : cell_keys_out(ctx, dev_keys);
}

int sph_get_ngb_hash(sph_ctx *ctx, uint64_t *dev_hash)
{
    if (!ctx || !dev_hash) return SPH_ERR_INVALID_ARG;
    if (!(ctx->p.flags & SPH_FLAG_NGB_HASH)) return fail(ctx, SPH_ERR_STATE, "SPH_FLAG_NGB_HASH not set");
    SPH_CUDA(ctx, cudaMemcpyAsync(dev_hash, ctx->ngb_hash, sizeof(uint64_t) * ctx->n, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    return SPH_OK;
}

int sph_get_stats(sph_ctx *ctx, sph_stats *s)
{
    if (!ctx || !s) return SPH_ERR_INVALID_ARG;
    int rc = read_counters(ctx);
    if (rc) return rc;
    double t[4] = {0, 0, 0, 0};
    for (Timer &tm : ctx->timers) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, tm.a, tm.b) == cudaSuccess) t[tm.kind] += ms;
    }
    sph_stats &st = ctx->st;
    st.density_pairs = (int64_t)ctx->h_counters[C_DPAIRS];
    st.force_pairs = (int64_t)ctx->h_counters[C_FPAIRS];
    st.density_candidates = (int64_t)ctx->h_counters[C_DCAND];
    st.force_candidates = (int64_t)ctx->h_counters[C_FCAND];
    st.density_targets = (int64_t)ctx->h_counters[C_DTARGETS];
    st.t_density_ms = t[0];
    st.t_force_ms = t[1];
    st.t_build_ms = t[2];
    st.t_grav_ms = t[3];
    st.grav_pairs = (int64_t)ctx->h_counters[C_GPAIRS];
    st.force_symmetric = ctx->sym_force ? 1 : 0;
    st.axis_sweep = (ctx->p.flags & SPH_FLAG_AXIS_SWEEP) && !ctx->adaptive ? 1 : 0;
    st.density_streamed = (int64_t)ctx->h_counters[C_DSTREAM];
    st.density_staged = (int64_t)ctx->h_counters[C_DSTAGED];
    st.force_streamed = (int64_t)ctx->h_counters[C_FSTREAM];
    st.force_staged = (int64_t)ctx->h_counters[C_FSTAGED];
    st.tile_width = ctx->tile_w;
    st.cell_factor = ctx->p.cell_factor;
    st.leaf_max = ctx->adaptive ? ctx->leaf_max : 0;
    st.hp_samples = ctx->hp.col_n;
    *s = st;
    return SPH_OK;
}

int sph_reset_stats(sph_ctx *ctx)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (Timer &t : ctx->timers) ctx->free_timers.push_back(t);
    ctx->timers.clear();
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_DPAIRS, 0, 6 * sizeof(unsigned long long), ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_GPAIRS, 0, sizeof(unsigned long long), ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_DSTREAM, 0, 4 * sizeof(unsigned long long), ctx->stream));
    int nc = ctx->st.nc;
    int64_t ncell = ctx->st.n_cells;
    double cs = ctx->st.cell_size;
    memset(&ctx->st, 0, sizeof ctx->st);
    ctx->st.nc = nc;
    ctx->st.n_cells = ncell;
    ctx->st.cell_size = cs;
    return SPH_OK;
}

int sph_hpredict_init(sph_ctx *ctx, uint64_t seed)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    return hp_init(ctx, seed);
}

int sph_hpredict_load(sph_ctx *ctx, const uint16_t *w_bf16, const float *f32)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!w_bf16 || !f32) return fail(ctx, SPH_ERR_INVALID_ARG, "null weight array");
    return hp_load(ctx, w_bf16, f32);
}

int sph_hpredict_save(sph_ctx *ctx, uint16_t *w_bf16, float *f32)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!w_bf16 || !f32) return fail(ctx, SPH_ERR_INVALID_ARG, "null weight array");
    return hp_save(ctx, w_bf16, f32);
}

int sph_hpredict_params(sph_ctx *ctx, float *params)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!params) return fail(ctx, SPH_ERR_INVALID_ARG, "null array");
    return hp_params(ctx, params);
}

int sph_hpredict_features(sph_ctx *ctx, sph_particles *parts, double dt, float *dev_feats)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!parts || (ctx->n > 0 && !parts_ok(parts))) return fail(ctx, SPH_ERR_INVALID_ARG, "null particle array");
    if (!isfinite(dt) || dt < 0) return fail(ctx, SPH_ERR_INVALID_ARG, "dt must be finite and >= 0");
    int rc = set_dt(ctx, dt);
    if (rc) return rc;
    rc = hp_features(ctx, parts);
    if (rc) return rc;
    if (dev_feats && ctx->n > 0)
        SPH_CUDA(ctx, cudaMemcpyAsync(dev_feats, ctx->hp.feats, sizeof(float) * 6 * ctx->n,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    return SPH_OK;
}

int sph_hpredict_targets(sph_ctx *ctx, sph_particles *parts, float *dev_target)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!parts || !dev_target) return fail(ctx, SPH_ERR_INVALID_ARG, "null array");
    return hp_targets(ctx, parts, dev_target);
}

int sph_hpredict_eval(sph_ctx *ctx, const float *dev_feats, int64_t n, float *dev_out)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (n < 0 || n >= (1ll << 31)) return fail(ctx, SPH_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    if (n > 0 && (!dev_feats || !dev_out)) return fail(ctx, SPH_ERR_INVALID_ARG, "null array");
    return hp_run(ctx, dev_feats, nullptr, dev_out, n, logf(0.5f), logf(1.2f));
}

int sph_hpredict_train(sph_ctx *ctx, const float *dev_feats, const float *dev_target, int64_t n, int32_t epochs,
                       float lr, uint64_t seed, float *loss_out)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (n <= 0 || !dev_feats || !dev_target) return fail(ctx, SPH_ERR_INVALID_ARG, "need n > 0 training pairs");
    if (epochs < 0 || !(lr > 0.f) || !isfinite(lr)) return fail(ctx, SPH_ERR_INVALID_ARG, "bad epochs or lr");
    return hp_train(ctx, dev_feats, dev_target, n, epochs, lr, seed, loss_out);
}

int sph_hpredict_collect(sph_ctx *ctx, float *dev_feats, float *dev_target, int64_t capacity)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (capacity < 0) return fail(ctx, SPH_ERR_INVALID_ARG, "capacity must be >= 0");
    if (capacity > 0 && (!dev_feats || !dev_target)) return fail(ctx, SPH_ERR_INVALID_ARG, "null buffer");
    HPredictor &H = ctx->hp;
    H.col_feats = capacity > 0 ? dev_feats : nullptr;
    H.col_target = capacity > 0 ? dev_target : nullptr;
    H.col_cap = capacity;
    H.col_n = 0;
    return SPH_OK;
}

const char *sph_last_error(const sph_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

void sph_destroy(sph_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    free_particles(ctx);
    free_bins(ctx);
    free_tree(ctx);
    cudaFree(ctx->axis);
    hp_free(ctx);
    cudaFree(ctx->cell_start);
    cudaFree(ctx->cell_tiles);
    cudaFree(ctx->counters);
    cudaFreeHost(ctx->h_counters);
    cudaFree(ctx->d_scalars);
    cudaFreeHost(ctx->h_scalars);
    cudaFree(ctx->d_red);
    cudaFreeHost(ctx->h_red);
    cudaFree(ctx->scan_aux);
    cudaFree(ctx->n_tiles);
    cudaFree(ctx->n_act_tiles);
    cudaFree(ctx->d_dt);
    cudaFreeHost(ctx->h_dt);
    cudaFree(ctx->d_boxes);
    cudaFreeHost(ctx->h_boxes);
    cudaFree(ctx->d_box_hmax);
    cudaFreeHost(ctx->h_box_hmax);
    cudaFree(ctx->d_box_off);
    if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->copy_ev) cudaEventDestroy(ctx->copy_ev);
    cudaFree(ctx->mirror_block);
    for (Timer &t : ctx->timers) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (Timer &t : ctx->free_timers) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    delete ctx;
}

}  // extern "C"
