// sph_gravity.cu -- the near field of the gravity of Theuns et al. 2015, Sec. 3.2
// (Eq. 3): the tree walk of that section ends in tasks in which a node meets the
// multipole of a distant node, and tasks in which all particles of one node
// interact with all particles of a nearby node, "implemented ... using the same
// task-based approach as used for SPH".  This file is the second kind on the SPH
// cell grid: every particle sums the Plummer-softened Eq. 3 over every other
// particle of its own cell and of the 26 adjacent cells (periodic, minimal image).
//
// Work decomposition: the SPH path's tiles (up to TW targets of one cell, one lane
// per target) handed out by the same ticket counter.  For each of the 27 cells a
// tile's lanes load TW sources at a time (one coalesced float4 each), shifted into
// the tile's cell frame, into shared memory; every lane then runs over all staged
// sources (broadcast reads).  No distance test, no pruning: each staged source is an
// interaction, so the inner loop is straight-line FP32 arithmetic -- 3 FADD, 6 FFMA,
// 3 FMUL, 1 FADD and one MUFU reciprocal square root per pair.  The terms of one
// cell are summed plainly and the 27 cell sums added with Kahan compensation; the
// summation order of a target never depends on which warp runs its tile.
#include <algorithm>

#include "sph_internal.cuh"

namespace sph {

constexpr int kGravThreads = 256;
// staging pads: far away (r^2 overflows to +inf, so rsqrt gives 0) and massless
constexpr float kGravFar = 1e30f;

struct GravArgs {
    const float4 *__restrict__ pos4;  // {x, y, z} relative to the cell centre, h
    const float4 *__restrict__ vel4;  // {vx, vy, vz, m}
    const int *__restrict__ cell_start;
    const int4 *__restrict__ tiles;
    const int *__restrict__ n_tiles;
    const BoxDev *__restrict__ boxes;
    float *ax, *ay, *az, *phi;  // caller's outputs (phi may be null)
    unsigned long long *counters;
    float G, eps2;
};

__device__ __forceinline__ int wrapg(int j, int nc) { return j < 0 ? j + nc : (j >= nc ? j - nc : j); }

// SOFT: eps > 0 (the target's own term is masked by its staged index); otherwise
// pairs at zero separation (the target itself, coincident particles) are dropped by
// their r^2
template <int TW, bool SOFT>
__global__ void __launch_bounds__(kGravThreads) k_gravity(GravArgs a)
{
    constexpr int TPW = 32 / TW;
    __shared__ float4 stage[kGravThreads / 32][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int sub = lane / TW, tl = lane % TW;
    float4 *sA = stage[wib] + sub * TW;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int ntiles = *a.n_tiles;
    const int ngroups = (ntiles + TPW - 1) / TPW;
    unsigned long long acc_pairs = 0ull;
    unsigned *ticket = reinterpret_cast<unsigned *>(a.counters + C_TICKET);
    unsigned tk = 0u;
    if (lane == 0) tk = atomicAdd(ticket, 1u);
    for (int grp = gw, g_after = 0; grp < ngroups; grp = g_after) {
        g_after = nw + (int)__shfl_sync(kFull, tk, 0);
        if (lane == 0 && g_after < ngroups) tk = atomicAdd(ticket, 1u);
        const int t = grp * TPW + sub;
        const int4 tile = t < ntiles ? a.tiles[t] : make_int4(0, 0, 0, 0);
        const bool valid = tl < tile.z;
        const int i = tile.y + tl;
        const float4 pi = valid ? a.pos4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const BoxDev bx = a.boxes[tile.w];
        const int nc = bx.nc;
        const float L = bx.L32;
        const int ca = tile.x - bx.cell_off;
        const int ix = ca % nc, iy = (ca / nc) % nc, iz = ca / (nc * nc);
        // the 27 cell ranges, fetched at once: lane tl holds cells tl and tl + TW;
        // cell o is at offset (o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1), o = 13 its own
        int cs0 = 0, ce0 = 0, cs1 = 0, ce1 = 0;
        if (tile.z > 0) {
            if (tl < 27) {
                const int cb = bx.cell_off + (wrapg(iz + tl / 9 - 1, nc) * nc + wrapg(iy + (tl / 3) % 3 - 1, nc)) * nc +
                               wrapg(ix + tl % 3 - 1, nc);
                cs0 = a.cell_start[cb];
                ce0 = a.cell_start[cb + 1];
            }
            if (tl + TW < 27) {
                const int o2 = tl + TW;
                const int cb = bx.cell_off + (wrapg(iz + o2 / 9 - 1, nc) * nc + wrapg(iy + (o2 / 3) % 3 - 1, nc)) * nc +
                               wrapg(ix + o2 % 3 - 1, nc);
                cs1 = a.cell_start[cb];
                ce1 = a.cell_start[cb + 1];
            }
        }
        float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f, sz = 0.f, cz = 0.f, sp = 0.f, cp = 0.f;
        int nsrc = 0;
        for (int o = 0; o < 27; ++o) {
            const int src = o < TW ? o : o - TW;
            const int bs = __shfl_sync(kFull, o < TW ? cs0 : cs1, src, TW);
            const int be = __shfl_sync(kFull, o < TW ? ce0 : ce1, src, TW);
            nsrc += be - bs;
            const float shx = (float)(o % 3 - 1) * L, shy = (float)((o / 3) % 3 - 1) * L,
                        shz = (float)(o / 9 - 1) * L;
            const int nch = (int)__reduce_max_sync(kFull, (unsigned)((be - bs + TW - 1) / TW));
            float bxs = 0.f, bys = 0.f, bzs = 0.f, bps = 0.f;  // this cell's terms
            // the sum over the staged sources: straight-line, or with the target's own
            // slot masked (own cell, softened: its term would be m_i / eps)
            auto sum = [&](int self) {
#pragma unroll 8
                for (int k = 0; k < TW; ++k) {
                    const float4 q = sA[k];
                    const float dx = q.x - pi.x, dy = q.y - pi.y, dz = q.z - pi.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, a.eps2)));
                    float inv = rsqrtf(r2);
                    if (!SOFT) inv = r2 > 0.f ? inv : 0.f;
                    const float mj = (SOFT && k == self) ? 0.f : q.w;
                    const float mi = mj * inv;
                    bps += mi;
                    const float mi3 = mi * inv * inv;
                    bxs = fmaf(mi3, dx, bxs);
                    bys = fmaf(mi3, dy, bys);
                    bzs = fmaf(mi3, dz, bzs);
                }
            };
            for (int ch = 0; ch < nch; ++ch) {
                const int j = bs + ch * TW + tl;
                float4 s = make_float4(kGravFar, kGravFar, kGravFar, 0.f);
                if (j < be) {
                    const float4 p = __ldg(a.pos4 + j);
                    s = make_float4(p.x + shx, p.y + shy, p.z + shz, __ldg(&a.vel4[j].w));
                }
                __syncwarp();
                sA[tl] = s;
                __syncwarp();
                if (SOFT && o == 13) sum(i - (bs + ch * TW));
                else sum(-1);
            }
            kahan_add(sx, cx, bxs);
            kahan_add(sy, cy, bys);
            kahan_add(sz, cz, bzs);
            kahan_add(sp, cp, bps);
        }
        if (!valid) continue;
        acc_pairs += (unsigned long long)(nsrc - 1);
        // a_i = -G sum m_j (r_i - r_j) / (r^2 + eps^2)^(3/2): the sums above run over
        // r_j - r_i, hence +G
        a.ax[i] = a.G * (sx - cx);
        a.ay[i] = a.G * (sy - cy);
        a.az[i] = a.G * (sz - cz);
        if (a.phi) a.phi[i] = -a.G * (sp - cp);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc_pairs += __shfl_xor_sync(kFull, acc_pairs, o);
    if (lane == 0 && acc_pairs) atomicAdd(a.counters + C_GPAIRS, acc_pairs);
}

template <int TW, bool SOFT>
static int launch_gravity(sph_ctx *ctx, const GravArgs &a)
{
    static int blocks_per_sm = 0;  // occupancy of this instantiation (per process)
    if (blocks_per_sm == 0) {
        SPH_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_gravity<TW, SOFT>, kGravThreads,
                                                                    0));
        blocks_per_sm = std::max(blocks_per_sm, 1);
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (sms <= 0) sms = 148;
    // persistent grid: every resident warp, no more than the tile groups need
    const int64_t want = ((int64_t)ctx->n / ctx->tile_w + ctx->grid.n_cells) / (kGravThreads / 32) + 1;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * blocks_per_sm, want));
    k_gravity<TW, SOFT><<<g, kGravThreads, 0, ctx->stream>>>(a);
    return SPH_OK;
}

int run_gravity_pass(sph_ctx *ctx, double G, double eps, float *ax, float *ay, float *az, float *phi)
{
    GravArgs a{};
    a.pos4 = ctx->pos4;
    a.vel4 = ctx->vel4;
    a.cell_start = ctx->cell_start;
    a.tiles = ctx->tiles;
    a.n_tiles = ctx->n_tiles;
    a.boxes = ctx->d_boxes;
    a.ax = ax;
    a.ay = ay;
    a.az = az;
    a.phi = phi;
    a.counters = ctx->counters;
    a.G = (float)G;
    a.eps2 = (float)(eps * eps);
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_TICKET, 0, sizeof(unsigned long long), ctx->stream));
    cudaEvent_t end = nullptr;
    timer_begin(ctx, 3, &end);
    const bool soft = eps > 0.0;
    int rc;
    if (ctx->tile_w == 32) rc = soft ? launch_gravity<32, true>(ctx, a) : launch_gravity<32, false>(ctx, a);
    else rc = soft ? launch_gravity<16, true>(ctx, a) : launch_gravity<16, false>(ctx, a);
    if (rc) return rc;
    timer_end(ctx, end);
    SPH_LAUNCH(ctx, "gravity kernel");
    ctx->st.grav_passes++;
    return SPH_OK;
}

}  // namespace sph
