// sph_integrate.cu -- marching particles forward in time (Theuns et al. 2015,
// Sec. 2: "positions by velocities, velocities by accelerations") and the O(N)
// reductions around the pair passes: CFL time step and the conserved quantities.
// Positions, velocities, kicks, drifts and the global sums are FP64; the sums use a
// fixed grid and tree order, so they are deterministic.  The step's dt lives on the
// device (ctx->d_dt), so a whole step can be replayed from a CUDA graph.
#include <math.h>

#include <utility>

#include "sph_internal.cuh"

namespace sph {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 304;  // fixed grid (2 x 152 SMs) for deterministic sums

__global__ void k_set_dt(double *d_dt, double dt) { *d_dt = dt; }

int set_dt(sph_ctx *ctx, double dt)
{
    k_set_dt<<<1, 1, 0, ctx->stream>>>(ctx->d_dt, dt);
    SPH_LAUNCH(ctx, "set dt");
    return SPH_OK;
}

// v += a * dt/2 (FP64); u <- max(u + dudt * dt/2, 0), counting floors
__global__ void k_kick(sph_particles P, int n, const double *__restrict__ d_dt, unsigned long long *floors)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double half_dt = 0.5 * *d_dt;
    bool fl = false;
    if (i < n) {
        P.vx[i] += (double)P.ax[i] * half_dt;
        P.vy[i] += (double)P.ay[i] * half_dt;
        P.vz[i] += (double)P.az[i] * half_dt;
        double u = (double)P.u[i] + (double)P.dudt[i] * half_dt;
        fl = u < 0.0;
        P.u[i] = (float)(fl ? 0.0 : u);
    }
    unsigned b = __ballot_sync(kFull, fl);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(floors, (unsigned long long)__popc(b));
}

int kick(sph_ctx *ctx, sph_particles *parts)
{
    int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    k_kick<<<(n + 255) / 256, 256, 0, ctx->stream>>>(*parts, n, ctx->d_dt, ctx->counters + C_FLOORS);
    SPH_LAUNCH(ctx, "kick");
    return SPH_OK;
}

// x += v dt (FP64); the periodic wrap follows in the cell build
__global__ void k_drift(sph_particles P, int n, const double *__restrict__ d_dt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dt = *d_dt;
    P.x[i] += P.vx[i] * dt;
    P.y[i] += P.vy[i] * dt;
    P.z[i] += P.vz[i] * dt;
}

int drift(sph_ctx *ctx, sph_particles *parts)
{
    int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    k_drift<<<(n + 255) / 256, 256, 0, ctx->stream>>>(*parts, n, ctx->d_dt);
    SPH_LAUNCH(ctx, "drift");
    return SPH_OK;
}

// min_i h_i / vsig_i over vsig_i > 0 (positive floats order like their bit patterns)
__global__ void k_cfl(const float *__restrict__ h, const float *__restrict__ vsig, int n,
                      unsigned *__restrict__ out)
{
    unsigned m = 0x7f800000u;  // +inf
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float v = vsig[i];
        if (v > 0.f) m = min(m, __float_as_uint(h[i] / v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) atomicMin(out, m);
}

__global__ void k_cfl_init(unsigned *out) { *out = 0x7f800000u; }

// dt = cfl * min h/vsig (+inf without signal velocities)
__global__ void k_cfl_final(const unsigned *__restrict__ m, double cfl, double *__restrict__ d_dt)
{
    const float r = __uint_as_float(*m);
    *d_dt = isfinite(r) ? cfl * (double)r : INFINITY;
}

int cfl_dt_device(sph_ctx *ctx, sph_particles *parts)
{
    unsigned *slot = (unsigned *)(ctx->d_scalars + 1);
    k_cfl_init<<<1, 1, 0, ctx->stream>>>(slot);
    SPH_LAUNCH(ctx, "cfl init");
    if (ctx->n > 0) {
        k_cfl<<<kRedBlocks * 4, kRedThreads, 0, ctx->stream>>>(parts->h, parts->vsig, (int)ctx->n, slot);
        SPH_LAUNCH(ctx, "cfl");
    }
    k_cfl_final<<<1, 1, 0, ctx->stream>>>(slot, (double)ctx->p.cfl, ctx->d_dt);
    SPH_LAUNCH(ctx, "cfl final");
    return SPH_OK;
}

int cfl_dt(sph_ctx *ctx, sph_particles *parts, double *dt_out)
{
    int rc = cfl_dt_device(ctx, parts);
    if (rc) return rc;
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_dt, ctx->d_dt, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *dt_out = *ctx->h_dt;
    return SPH_OK;
}

// FP64 sums {m vx, m vy, m vz, m v^2/2, m u}: per-block partials, fixed order
__global__ void __launch_bounds__(kRedThreads) k_conserved_part(sph_particles P, int n, double *part)
{
    double s[5] = {0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double m = (double)P.m[i], vx = P.vx[i], vy = P.vy[i], vz = P.vz[i];
        s[0] += m * vx;
        s[1] += m * vy;
        s[2] += m * vz;
        s[3] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        s[4] += m * (double)P.u[i];
    }
    __shared__ double sh[5][kRedThreads];
#pragma unroll
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < 5) part[threadIdx.x * kRedBlocks + blockIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_conserved_final(const double *part, double *out)
{
    // 5 warps, one quantity each; lanes stride the partials in a fixed order
    int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s = 0;
    for (int b = lane; b < kRedBlocks; b += 32) s += part[k * kRedBlocks + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) out[k] = s;
}

int conserved_device(sph_ctx *ctx, sph_particles *parts)
{
    int n = (int)ctx->n;
    k_conserved_part<<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(*parts, n, ctx->d_red);
    SPH_LAUNCH(ctx, "conserved partials");
    k_conserved_final<<<1, 160, 0, ctx->stream>>>(ctx->d_red, ctx->d_red + 5 * kRedBlocks);
    SPH_LAUNCH(ctx, "conserved final");
    return SPH_OK;
}

int conserved_read(sph_ctx *ctx, sph_conserved *out)
{
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_red, ctx->d_red + 5 * kRedBlocks, 5 * sizeof(double),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_counters, ctx->counters, C_NCOUNTERS * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    out->momentum[0] = ctx->h_red[0];
    out->momentum[1] = ctx->h_red[1];
    out->momentum[2] = ctx->h_red[2];
    out->e_kin = ctx->h_red[3];
    out->e_th = ctx->h_red[4];
    out->u_floors = (int64_t)ctx->h_counters[C_FLOORS];
    return SPH_OK;
}

int red_scratch_doubles() { return 5 * kRedBlocks + 8; }

// ------------------------------------------------------- individual time-steps
// Power-of-two steps on an integer time grid of unit dt_max / 2^L (L = n_bins): a
// particle in bin b steps by 2^(L-b) units, and each of its steps starts on a
// multiple of that length, so that all steps end together at dt_max.  The paper is
// silent on time-stepping; this is the scheme of the Gadget-2 lineage its force law
// comes from.  Every particle keeps the start and end of its current step, {s0, T}
// (int2: the grid has at most 2^SPH_MAX_BINS units), since a wake-up of the
// time-step limiter cuts a step short of its bin's length.

__device__ __forceinline__ int64_t bin_len(int L, int b) { return (int64_t)1 << (L - b); }

// act[i] = the particle's step ends at integer time s; counts them
__global__ void k_bin_active(const int2 *__restrict__ st, int n, int64_t s, uint8_t *__restrict__ act,
                             unsigned long long *count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool a = false;
    if (i < n) {
        a = (int64_t)st[i].y == s;
        act[i] = a ? 1 : 0;
    }
    unsigned m = __ballot_sync(kFull, a);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(count, (unsigned long long)__popc(m));
}

// half kick of the active particles (all of them if act is null) over their own
// step {s0, T}: v += a dt/2 (FP64); u <- max(u + dudt dt/2, 0), counting floors.  The
// arithmetic is k_kick's with dt = (T - s0) unit.
__global__ void k_bin_kick(sph_particles P, int n, const int2 *__restrict__ st, const uint8_t *__restrict__ act,
                           double unit, unsigned long long *floors)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool fl = false;
    if (i < n && (act == nullptr || act[i])) {
        const int2 q = st[i];
        const double half_dt = 0.5 * ((double)(q.y - q.x) * unit);
        P.vx[i] += (double)P.ax[i] * half_dt;
        P.vy[i] += (double)P.ay[i] * half_dt;
        P.vz[i] += (double)P.az[i] * half_dt;
        double u = (double)P.u[i] + (double)P.dudt[i] * half_dt;
        fl = u < 0.0;
        P.u[i] = (float)(fl ? 0.0 : u);
    }
    unsigned b = __ballot_sync(kFull, fl);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(floors, (unsigned long long)__popc(b));
}

// Bins of the active particles (all if act is null) starting a step at time s: the
// largest step dt_max / 2^b not above cfl h / vsig (bin L, counted, if even the
// smallest is above it), then smaller until s is a multiple of its length.
__global__ void k_bin_assign(const float *__restrict__ h, const float *__restrict__ vsig,
                             const uint8_t *__restrict__ act, int8_t *__restrict__ bins, int n, int64_t s, int L,
                             double dt_max, double cfl, unsigned long long *over)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool ov = false;
    if (i < n && (act == nullptr || act[i])) {
        const float v = vsig[i];
        const double dtc = v > 0.f ? cfl * (double)h[i] / (double)v : (double)INFINITY;
        int b = L;
        for (int k = L; k >= 0; --k)
            if (ldexp(dt_max, -k) <= dtc) b = k;
        ov = ldexp(dt_max, -L) > dtc;
        while (b < L && (s & (bin_len(L, b) - 1)) != 0) ++b;
        bins[i] = (int8_t)b;
    }
    unsigned m = __ballot_sync(kFull, ov);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(over, (unsigned long long)__popc(m));
}

// The active particles (all if act is null) open a step at s: {s, s + 2^(L-b)}.
// With the limiter, the sleeping ones whose raised bin's step, counted from the
// grid, ends at T' = (s / D' + 1) D' before their own end T are woken: T <- T', and
// their opening half kick is corrected by (T' - T) / 2 (k_kick's arithmetic; floors
// counted).  cfl_bins (limiter only) are the bins before the limiter: starting
// steps whose bin it raised are counted.
__global__ void k_bin_open(sph_particles P, int n, const int8_t *__restrict__ bins,
                           const int8_t *__restrict__ cfl_bins, const uint8_t *__restrict__ act,
                           int2 *__restrict__ st, int64_t s, int L, double unit, unsigned long long *floors,
                           unsigned long long *limited, unsigned long long *woken)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool fl = false, lim = false, wk = false;
    if (i < n) {
        const int b = bins[i];
        const int64_t D = bin_len(L, b);
        if (act == nullptr || act[i]) {
            st[i] = make_int2((int)s, (int)(s + D));
            lim = cfl_bins != nullptr && cfl_bins[i] != b;
        } else if (cfl_bins != nullptr) {
            const int2 q = st[i];
            const int64_t Tn = (s / D + 1) * D;
            if (Tn < (int64_t)q.y) {
                wk = true;
                const double half_dt = 0.5 * ((double)(Tn - (int64_t)q.y) * unit);
                P.vx[i] += (double)P.ax[i] * half_dt;
                P.vy[i] += (double)P.ay[i] * half_dt;
                P.vz[i] += (double)P.az[i] * half_dt;
                double u = (double)P.u[i] + (double)P.dudt[i] * half_dt;
                fl = u < 0.0;
                P.u[i] = (float)(fl ? 0.0 : u);
                st[i] = make_int2(q.x, (int)Tn);
            }
        }
    }
    const unsigned bf = __ballot_sync(kFull, fl), bl = __ballot_sync(kFull, lim), bw = __ballot_sync(kFull, wk);
    if ((threadIdx.x & 31) == 0) {
        if (bf) atomicAdd(floors, (unsigned long long)__popc(bf));
        if (bl) atomicAdd(limited, (unsigned long long)__popc(bl));
        if (bw) atomicAdd(woken, (unsigned long long)__popc(bw));
    }
}

// ---- time-step limiter (Saitoh & Makino 2009)
// One pass of the limiter's monotone map: a particle whose step ends now takes
// max(b_i, max over neighbours j of b_j - K), a sleeping one max(b_j, max over
// neighbours i whose step ends now of b_i - K), neighbours the pairs
// r_ij < max(h_i, h_j) of the force sum.  The pair set is symmetric, so both halves
// are done from the active particles alone: each gathers the largest b_j - K of
// its neighbours and scatters b_i - K to its sleeping ones, both as atomic maxima
// into `want` (which does not depend on their order); a last kernel folds `want`
// into the bins.  Passes repeat until none changes anything: the least fixed point
// above the starting bins.  The cells around a particle hold all its neighbours:
// on the uniform grid the 27 around its cell, or the 125 where a cutoff can exceed
// the cell side (every h stays within two sides); with adaptive cells the 27 top
// cells around it (every h within its top cell's side).
// Work items are (active particle, stencil cell) pairs, one per thread, so that a
// pass over a few thousand active particles still spreads over the whole GPU.  What
// keeps a pass cheap:
//  - per cell, the largest bin (over all particles) and the smallest bin of a
//    sleeping particle: a cell that can neither raise the particle nor be raised by
//    it is skipped unread, and within a cell only such pairs are tested;
//  - after the first pass a particle gathers only from the cells that changed in
//    the pass before (what the others give is already in its bin), and scatters
//    only if its own cell changed;
//  - the distance test runs in FP32 (uniform grid: the cell-relative positions
//    shifted by the cell offset; adaptive cells: differences of the FP64 positions,
//    rounded), and only pairs within the rounding band of r_ij^2 = max(h)^2 are
//    re-decided in FP64 from the absolute positions, with the operation order of
//    the plain definition -- the decision is the FP64 one, at FP32 cost (FP64 runs
//    at a small fraction of the FP32 rate on this part).
struct LimArgs {
    const double *__restrict__ x, *__restrict__ y, *__restrict__ z;
    const float4 *__restrict__ pos4;  // uniform grid: {x, y, z} relative to the cell centre
    const float *__restrict__ h;
    const int8_t *__restrict__ bins;
    const uint8_t *__restrict__ act;
    const int32_t *__restrict__ cell;  // global (top-level) cell of each slot
    const int *__restrict__ cell_start;
    const int *__restrict__ cmax_all, *__restrict__ cmin_sleep;
    const float *__restrict__ reach;    // uniform grid: per cell, the largest h that can reach it
    const uint8_t *__restrict__ dirty;  // cells changed by the previous pass (null: first pass)
    const int *__restrict__ list;       // the active slots
    const unsigned long long *n_list;
    const BoxDev *__restrict__ boxes;
    int nb, n, K, adaptive;
    double box;
    int *__restrict__ want;  // largest bin gathered by / scattered to each particle (-1: none)
};

constexpr int kNoSleeper = 0x7f7f7f7f;  // cmin_sleep of a cell without sleeping particles
constexpr int kStencil = 125;           // work items per active particle: the radius-2 stencil

// per cell: largest bin over all particles, smallest bin over sleeping ones (the
// lanes of one cell combined before the atomics: consecutive slots share a cell)
__global__ void k_lim_cellstat(const int32_t *__restrict__ cell, const int8_t *__restrict__ bins,
                               const uint8_t *__restrict__ act, int n, int *__restrict__ cmax_all,
                               int *__restrict__ cmin_sleep)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = i < n;
    const int c = in ? cell[i] : -1, b = in ? (int)bins[i] : -1;
    const int bs = in && !act[i] ? b : kNoSleeper;
    const unsigned grp = __match_any_sync(kFull, c);
    const int mall = __reduce_max_sync(grp, b), msl = __reduce_min_sync(grp, bs);
    if (in && (int)(threadIdx.x & 31) == __ffs(grp) - 1) {
        atomicMax(cmax_all + c, mall);
        if (msl != kNoSleeper) atomicMin(cmin_sleep + c, msl);
    }
}

// the active slots, in any order (the passes take maxima only)
__global__ void k_lim_list(const uint8_t *__restrict__ act, int n, int *__restrict__ list,
                           unsigned long long *count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool a = i < n && act[i];
    const unsigned m = __ballot_sync(kFull, a);
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0 && m) base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, 0);
    if (a) list[base + __popc(m & ((1u << lane) - 1u))] = i;
}

__device__ __forceinline__ int lim_wrap(int j, int nc) { return j < 0 ? j + nc : (j >= nc ? j - nc : j); }

__device__ __forceinline__ float lim_image(float d, float box)
{
    return d > 0.5f * box ? d - box : (d < -0.5f * box ? d + box : d);
}

__global__ void k_lim_pairs(LimArgs a)
{
    const long long total = (long long)*a.n_list * kStencil;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int pi = a.list[t / kStencil], o = (int)(t % kStencil);
        const int b = a.bins[pi], cp = a.cell[pi];
        int lo = 0, hi = a.nb - 1;  // the box holding slot pi (boxes are in slot order)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.boxes[mid].p_begin <= pi) lo = mid;
            else hi = mid - 1;
        }
        const BoxDev bx = a.boxes[lo];
        const float hp = a.h[pi];
        const float L = bx.L32;
        // stencil radius: 2 where some pair's cutoff max(h_i, h_j) can exceed a cell side
        const int R = a.adaptive ? 1 : (fmaxf(hp, a.reach[cp]) * (1.f + kPruneMargin) > L ? 2 : 1);
        const int W = 2 * R + 1;
        if (o >= W * W * W) continue;
        const int nc = bx.nc;
        const int ca = cp - bx.cell_off;
        const int ix = ca % nc, iy = (ca / nc) % nc, iz = ca / (nc * nc);
        const int ox_ = o % W - R, oy_ = (o / W) % W - R, oz_ = o / (W * W) - R;
        const int cb = bx.cell_off + (lim_wrap(iz + oz_, nc) * nc + lim_wrap(iy + oy_, nc)) * nc + lim_wrap(ix + ox_, nc);
        const int give = b - a.K;  // what the particle scatters
        const bool cg = a.cmax_all[cb] - a.K > b && (a.dirty == nullptr || a.dirty[cb]);
        const bool cs = give > a.cmin_sleep[cb] && (a.dirty == nullptr || a.dirty[cp]);
        if (!cg && !cs) continue;
        const float boxf = (float)a.box;
        const float ext = a.adaptive ? boxf : L;  // scale of the FP32 position errors
        const float4 pp = a.adaptive ? make_float4(0.f, 0.f, 0.f, 0.f) : a.pos4[pi];
        const double xp = a.x[pi], yp = a.y[pi], zp = a.z[pi];
        const float ox = (float)ox_ * L, oy = (float)oy_ * L, oz = (float)oz_ * L;
        int m = b;
        const int q1 = a.cell_start[cb + 1];
        for (int q = a.cell_start[cb]; q < q1; ++q) {
            const int bq = a.bins[q];
            const bool ng = cg && bq - a.K > m;
            const bool ns = cs && give > bq && !a.act[q];
            if (q == pi || !(ng || ns)) continue;
            float dx, dy, dz;
            if (a.adaptive) {
                dx = lim_image((float)(a.x[q] - xp), boxf);
                dy = lim_image((float)(a.y[q] - yp), boxf);
                dz = lim_image((float)(a.z[q] - zp), boxf);
            } else {
                const float4 pq = a.pos4[q];
                dx = (pq.x + ox) - pp.x;
                dy = (pq.y + oy) - pp.y;
                dz = (pq.z + oz) - pp.z;
            }
            const float H = fmaxf(hp, a.h[q]);
            const float r2 = dx * dx + dy * dy + dz * dz, H2 = H * H;
            const float band = kBandK * H * (H + ext);
            bool hit = r2 < H2 - band;
            if (!hit && r2 <= H2 + band) hit = within64(sep2_64(a.x, a.y, a.z, pi, q, a.box), H);
            if (!hit) continue;
            if (ng) m = bq - a.K;
            if (ns) atomicMax(a.want + q, give);
        }
        if (m > b) atomicMax(a.want + pi, m);
    }
}

// Fold the gathered and scattered maxima into the bins (and reset `want`), mark the
// cells of the particles that changed, count them.
__global__ void k_lim_finish(const int8_t *__restrict__ bins, const int32_t *__restrict__ cell, int n,
                             int *__restrict__ want, int8_t *__restrict__ out, uint8_t *__restrict__ dirty_next,
                             unsigned long long *changed)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    bool chg = false;
    if (p < n) {
        const int b = bins[p], w = want[p];
        if (w >= 0) want[p] = -1;
        const int nb = max(b, w);
        out[p] = (int8_t)nb;
        chg = nb != b;
        if (chg) dirty_next[cell[p]] = 1;
    }
    const unsigned c = __ballot_sync(kFull, chg);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(changed, (unsigned long long)__popc(c));
}

// deepest bin and earliest step end over all particles
__global__ void k_bin_max(const int8_t *__restrict__ bins, const int2 *__restrict__ st, int n,
                          unsigned long long *out, unsigned long long *tmin)
{
    unsigned m = 0, t = 0xffffffffu;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        m = max(m, (unsigned)bins[i]);
        t = min(t, (unsigned)st[i].y);
    }
    m = __reduce_max_sync(kFull, m);
    t = __reduce_min_sync(kFull, t);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)m);
        atomicMin(tmin, (unsigned long long)t);
    }
}

// The cell build permutes the particle arrays it knows; the density outputs that
// inactive particles keep (rho, P, c, f, |curl v|), their bins, steps and active
// flags follow the same permutation here (slot p takes what slot perm[p] held).
__global__ void k_bin_gather(const uint32_t *__restrict__ perm, int n, sph_particles P,
                             const int8_t *__restrict__ bins, const uint8_t *__restrict__ act,
                             const int2 *__restrict__ st, float *__restrict__ s32, int64_t cap,
                             int8_t *__restrict__ bins_out, uint8_t *__restrict__ act_out, int2 *__restrict__ st_out)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int src = (int)perm[p];
    s32[p] = P.rho[src];
    s32[cap + p] = P.P[src];
    s32[2 * cap + p] = P.c[src];
    s32[3 * cap + p] = P.f[src];
    s32[4 * cap + p] = P.curl[src];
    bins_out[p] = bins[src];
    act_out[p] = act[src];
    st_out[p] = st[src];
}

// Copy the gathered outputs back; then, per particle, the velocity and internal
// energy predicted to the current time s (v_half + a (t - t_mid), t_mid = (s0 + T) / 2
// the middle of the particle's own step: +dt/2 at its end, as in the global step) and
// the packed force inputs of the density pass (rho, f P / rho^2, c, Balsara B), for
// the particles that keep their last density.
__global__ void k_bin_predict(sph_particles P, int n, const float *__restrict__ s32, int64_t cap,
                              const int2 *__restrict__ st, int64_t s, double unit, int use_balsara,
                              float4 *__restrict__ vel4, float *__restrict__ upred, float4 *__restrict__ thermo4)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float rho = s32[p], Pp = s32[cap + p], cs = s32[2 * cap + p], fgh = s32[3 * cap + p],
                curl = s32[4 * cap + p];
    P.rho[p] = rho;
    P.P[p] = Pp;
    P.c[p] = cs;
    P.f[p] = fgh;
    P.curl[p] = curl;
    const int2 q = st[p];
    const double tau = 0.5 * ((double)(2 * s - (int64_t)q.x - (int64_t)q.y) * unit);
    vel4[p] = make_float4((float)(P.vx[p] + (double)P.ax[p] * tau), (float)(P.vy[p] + (double)P.ay[p] * tau),
                          (float)(P.vz[p] + (double)P.az[p] * tau), P.m[p]);
    const double up = (double)P.u[p] + (double)P.dudt[p] * tau;
    upred[p] = (float)(up > 0.0 ? up : 0.0);
    float Bq = 1.f;
    if (use_balsara) {
        const float ad = fabsf(P.divv[p]);
        const float hinv = 1.f / P.h[p];
        const float den = ad + curl + 1e-4f * cs * hinv;
        Bq = den > 0.f ? ad / den : 0.f;
    }
    thermo4[p] = make_float4(rho, fgh * Pp / (rho * rho), cs, Bq);
}

int bin_permute(sph_ctx *ctx, sph_particles *parts)
{
    const int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    k_bin_gather<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->vals, n, *parts, ctx->bins, ctx->bin_active,
                                                           ctx->bin_st, ctx->bin_s32, ctx->bin_cap, ctx->bins_tmp,
                                                           ctx->bin_active_tmp, ctx->bin_st_tmp);
    SPH_LAUNCH(ctx, "bin gather");
    std::swap(ctx->bins, ctx->bins_tmp);
    std::swap(ctx->bin_active, ctx->bin_active_tmp);
    std::swap(ctx->bin_st, ctx->bin_st_tmp);
    k_bin_predict<<<(n + 255) / 256, 256, 0, ctx->stream>>>(*parts, n, ctx->bin_s32, ctx->bin_cap, ctx->bin_st,
                                                            ctx->bin_now, ctx->bin_unit, ctx->p.use_balsara,
                                                            ctx->vel4, ctx->upred, ctx->thermo4);
    SPH_LAUNCH(ctx, "bin predict");
    return SPH_OK;
}

int bin_active(sph_ctx *ctx, unsigned long long *n_active)
{
    const int n = (int)ctx->n;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_BINACT, 0, sizeof(unsigned long long), ctx->stream));
    if (n > 0) {
        k_bin_active<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->bin_st, n, ctx->bin_now, ctx->bin_active,
                                                               ctx->counters + C_BINACT);
        SPH_LAUNCH(ctx, "bin active");
    }
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_counters + C_BINACT, ctx->counters + C_BINACT, sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *n_active = ctx->h_counters[C_BINACT];
    return SPH_OK;
}

int bin_kick(sph_ctx *ctx, sph_particles *parts, bool all)
{
    const int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    k_bin_kick<<<(n + 255) / 256, 256, 0, ctx->stream>>>(*parts, n, ctx->bin_st, all ? nullptr : ctx->bin_active,
                                                         ctx->bin_unit, ctx->counters + C_FLOORS);
    SPH_LAUNCH(ctx, "bin kick");
    return SPH_OK;
}

int bin_assign(sph_ctx *ctx, sph_particles *parts, bool all, double dt_max)
{
    const int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    k_bin_assign<<<(n + 255) / 256, 256, 0, ctx->stream>>>(parts->h, parts->vsig, all ? nullptr : ctx->bin_active,
                                                           ctx->bins, n, ctx->bin_now, ctx->bin_levels, dt_max,
                                                           (double)ctx->p.cfl, ctx->counters + C_BINOVER);
    SPH_LAUNCH(ctx, "bin assign");
    return SPH_OK;
}

// The limiter's passes until none changes a bin (host read after each), then the
// opening of the active particles' steps and the wake-ups (bin_open).  The cells of
// the current build give each particle's 27-cell neighbourhood.
int bin_limit(sph_ctx *ctx, sph_particles *parts, bool all, int64_t *sweeps)
{
    const int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    if (all) SPH_CUDA(ctx, cudaMemsetAsync(ctx->bin_active, 1, (size_t)n, ctx->stream));
    const int64_t nc = ctx->grid.n_cells;
    if (ctx->lim_cmax_cap < nc) {  // 2 x nc ints of cell bins, then 2 x nc dirty bytes
        if (ctx->lim_cmax) cudaFree(ctx->lim_cmax);
        ctx->lim_cmax = nullptr;
        ctx->lim_cmax_cap = 0;
        SPH_CUDA(ctx, cudaMalloc(&ctx->lim_cmax, (sizeof(int) * 2 + 2) * (size_t)nc));
        ctx->lim_cmax_cap = nc;
    }
    uint8_t *dirty[2] = {reinterpret_cast<uint8_t *>(ctx->lim_cmax + 2 * nc),
                         reinterpret_cast<uint8_t *>(ctx->lim_cmax + 2 * nc) + nc};
    int rc = ctx->adaptive ? tree_cell_keys_out(ctx, ctx->lim_cell) : cell_keys_out(ctx, ctx->lim_cell);
    if (rc) return rc;
    if (!ctx->adaptive) {  // per cell the largest h that can reach it (into cell_tmp)
        rc = cell_reach(ctx);
        if (rc) return rc;
    }
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->bins_cfl, ctx->bins, (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->lim_want, 0xff, sizeof(int) * (size_t)n, ctx->stream));
    LimArgs a{};
    a.x = parts->x;
    a.y = parts->y;
    a.z = parts->z;
    a.pos4 = ctx->pos4;
    a.h = parts->h;
    a.act = ctx->bin_active;
    a.cell = ctx->lim_cell;
    a.cell_start = ctx->cell_start;
    a.cmax_all = ctx->lim_cmax;
    a.cmin_sleep = ctx->lim_cmax + nc;
    a.reach = ctx->cell_tmp;
    a.boxes = ctx->d_boxes;
    a.nb = (int)ctx->n_boxes;
    a.n = n;
    a.K = SPH_BIN_LIMIT_LEVELS;
    a.adaptive = ctx->adaptive ? 1 : 0;
    a.box = ctx->p.box_size;
    a.want = ctx->lim_want;
    a.list = ctx->lim_list;
    a.n_list = ctx->counters + C_LIMACT;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_LIMACT, 0, sizeof(unsigned long long), ctx->stream));
    k_lim_list<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->bin_active, n, ctx->lim_list, ctx->counters + C_LIMACT);
    SPH_LAUNCH(ctx, "limiter active list");
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || sms <= 0)
        sms = 148;
    const unsigned pair_blocks = (unsigned)(8 * sms);
    // each pass raises a bin to some neighbour's bin minus K >= 1, so a chain of
    // raises is at most SPH_MAX_BINS / K + 1 long; passes beyond that find nothing
    const int max_sweeps = SPH_MAX_BINS + 2;
    for (int k = 0;; ++k) {
        if (k >= max_sweeps) return fail(ctx, SPH_ERR_TIMEOUT, "time-step limiter did not settle");
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->lim_cmax, 0xff, sizeof(int) * (size_t)nc, ctx->stream));
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->lim_cmax + nc, 0x7f, sizeof(int) * (size_t)nc, ctx->stream));
        k_lim_cellstat<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->lim_cell, ctx->bins, ctx->bin_active, n,
                                                                 ctx->lim_cmax, ctx->lim_cmax + nc);
        SPH_LAUNCH(ctx, "limiter cell bins");
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_LIMCHG, 0, sizeof(unsigned long long), ctx->stream));
        SPH_CUDA(ctx, cudaMemsetAsync(dirty[(k + 1) & 1], 0, (size_t)nc, ctx->stream));
        a.bins = ctx->bins;
        a.dirty = k == 0 ? nullptr : dirty[k & 1];
        k_lim_pairs<<<pair_blocks, 256, 0, ctx->stream>>>(a);
        SPH_LAUNCH(ctx, "limiter pass");
        k_lim_finish<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->bins, ctx->lim_cell, n, ctx->lim_want,
                                                               ctx->bins_tmp, dirty[(k + 1) & 1],
                                                               ctx->counters + C_LIMCHG);
        SPH_LAUNCH(ctx, "limiter fold");
        std::swap(ctx->bins, ctx->bins_tmp);
        SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_counters + C_LIMCHG, ctx->counters + C_LIMCHG,
                                      sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
        SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        ++*sweeps;
        if (ctx->h_counters[C_LIMCHG] == 0) break;
    }
    return SPH_OK;
}

int bin_open(sph_ctx *ctx, sph_particles *parts, bool all, bool limiter)
{
    const int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    k_bin_open<<<(n + 255) / 256, 256, 0, ctx->stream>>>(
        *parts, n, ctx->bins, limiter ? ctx->bins_cfl : nullptr, all ? nullptr : ctx->bin_active, ctx->bin_st,
        ctx->bin_now, ctx->bin_levels, ctx->bin_unit, ctx->counters + C_FLOORS, ctx->counters + C_LIMITED,
        ctx->counters + C_WOKEN);
    SPH_LAUNCH(ctx, "bin open");
    return SPH_OK;
}

int bin_max_read(sph_ctx *ctx, int *max_bin, unsigned long long *over, int64_t *t_min)
{
    const int n = (int)ctx->n;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_BINMAX, 0, sizeof(unsigned long long), ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_TMIN, 0xff, sizeof(unsigned long long), ctx->stream));
    if (n > 0) {
        k_bin_max<<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(ctx->bins, ctx->bin_st, n, ctx->counters + C_BINMAX,
                                                              ctx->counters + C_TMIN);
        SPH_LAUNCH(ctx, "bin max");
    }
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_counters + C_BINMAX, ctx->counters + C_BINMAX,
                                  2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_counters + C_TMIN, ctx->counters + C_TMIN, sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *max_bin = (int)ctx->h_counters[C_BINMAX];
    *over = ctx->h_counters[C_BINOVER];
    if (t_min) *t_min = (int64_t)ctx->h_counters[C_TMIN];
    return SPH_OK;
}

}  // namespace sph
