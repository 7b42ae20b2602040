// sph_gravity.cu -- the near field of the gravity of Theuns et al. 2015, Sec. 3.2
// (Eq. 3): the tree walk of that section ends in tasks in which a node meets the
// multipole of a distant node, and tasks in which all particles of one node
// interact with all particles of a nearby node, "implemented ... using the same
// task-based approach as used for SPH".  This file is the second kind on the SPH
// cell grid: every particle sums the Plummer-softened Eq. 3 over every other
// particle of its own cell and of the 26 adjacent cells (periodic, minimal image).
//
// Work decomposition: the SPH path's tiles (up to TW targets of one cell, one lane
// per target) handed out by the same ticket counter.  The 27 cells' particles form
// one source stream per tile; its lanes load TW stream positions at a time (one
// coalesced float4 each, across cell boundaries, so that only the stream's last
// chunk has pads), shifted into the tile's cell frame, into shared memory; every
// lane then runs over all staged sources (broadcast reads).  No distance test, no
// pruning: each staged source is an interaction, so the inner loop is straight-line
// FP32 arithmetic -- 3 FADD, 3 FFMA for r^2, one MUFU reciprocal square root, 3 FMUL,
// 1 FADD and 3 FFMA per pair.  The terms of 128 staged sources are summed plainly and
// the batch sums added with Kahan compensation; the summation order of a target
// never depends on which warp runs its tile.
#include <algorithm>

#include "sph_internal.cuh"

namespace sph {

constexpr int kGravThreads = 256;
// staging pads: far away (r^2 overflows to +inf, so rsqrt gives 0) and massless
constexpr float kGravFar = 1e30f;
// smallest squared separation (box units) an unsoftened pair contributes at, and the
// smallest eps^2 the softened kernel runs with: FP32 positions relative to a cell
// centre cannot resolve separations near 1e-15 anyway
constexpr float kGravMinR2 = 1e-30f;

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

// 1/sqrt(x) as the one MUFU instruction, with denormal inputs and results flushed
// to zero: the squared separations here are at least eps^2 >= kGravMinR2 (softened)
// or, unsoftened, taken only above kGravMinR2 -- never denormal -- so nothing else is
// needed around it; rsqrt(+inf) = 0 keeps the staging pads inert.
__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// SOFT: eps^2 >= kGravMinR2 -- every staged source enters the sums, and the target's
// own term (exactly m_i / eps: its separation is exactly 0) is taken out once at the
// end; otherwise pairs closer than sqrt(kGravMinR2) (the target itself, coincident
// particles) are dropped by their r^2.
template <int TW, bool SOFT>
__global__ void __launch_bounds__(kGravThreads) k_gravity(GravArgs a)
{
    constexpr int TPW = 32 / TW;
    constexpr int kFlush = 128 / TW;  // chunks per compensated batch (128 sources)
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
        // The sources of a tile as one stream: the 27 cells in order o = 0..26 (cell o
        // at offset (o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1), o = 13 the tile's own),
        // each cell's particles in slot order.  Lane tl describes cell tl (and, for
        // TW = 16, cell tl + 16): where the cell ends in the stream, and slot - stream
        // position for its particles.
        int endA = 0, offA = 0, endB = 0, offB = 0;
        {
            int bsA = 0, cA = 0, bsB = 0, cB = 0;
            if (tile.z > 0) {
                if (tl < 27) {
                    const int cb = bx.cell_off +
                                   (wrapg(iz + tl / 9 - 1, nc) * nc + wrapg(iy + (tl / 3) % 3 - 1, nc)) * nc +
                                   wrapg(ix + tl % 3 - 1, nc);
                    bsA = a.cell_start[cb];
                    cA = a.cell_start[cb + 1] - bsA;
                }
                if (tl + TW < 27) {
                    const int o2 = tl + TW;
                    const int cb = bx.cell_off +
                                   (wrapg(iz + o2 / 9 - 1, nc) * nc + wrapg(iy + (o2 / 3) % 3 - 1, nc)) * nc +
                                   wrapg(ix + o2 % 3 - 1, nc);
                    bsB = a.cell_start[cb];
                    cB = a.cell_start[cb + 1] - bsB;
                }
            }
            endA = cA;
            endB = cB;
#pragma unroll
            for (int d = 1; d < TW; d <<= 1) {
                const int vA = __shfl_up_sync(kFull, endA, d, TW), vB = __shfl_up_sync(kFull, endB, d, TW);
                if (tl >= d) {
                    endA += vA;
                    endB += vB;
                }
            }
            endB += __shfl_sync(kFull, endA, TW - 1, TW);
            offA = bsA - (endA - cA);
            offB = bsB - (endB - cB);
        }
        const int total = __shfl_sync(kFull, TW == 32 ? endA : endB, TW - 1, TW);
        // this lane's cursor: stream cell cur, its end and slot offset
        int cur = 0;
        int cend = __shfl_sync(kFull, endA, 0, TW), coff = __shfl_sync(kFull, offA, 0, TW);
        float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f, sz = 0.f, cz = 0.f, sp = 0.f, cp = 0.f;
        float bxs = 0.f, bys = 0.f, bzs = 0.f, bps = 0.f;  // terms of the current batch
        const int nch = (int)__reduce_max_sync(kFull, (unsigned)((total + TW - 1) / TW));
        for (int ch = 0; ch < nch; ++ch) {
            const int q = ch * TW + tl;
            // move the cursor to the cell holding stream position q (skipping empty cells)
            while (__any_sync(kFull, q < total && q >= cend)) {
                if (q < total && q >= cend) ++cur;
                const int src = cur < TW ? cur : cur - TW;
                const int eA = __shfl_sync(kFull, endA, src, TW), eB = __shfl_sync(kFull, endB, src, TW);
                const int fA = __shfl_sync(kFull, offA, src, TW), fB = __shfl_sync(kFull, offB, src, TW);
                cend = cur < TW ? eA : eB;
                coff = cur < TW ? fA : fB;
            }
            float4 sv = make_float4(kGravFar, kGravFar, kGravFar, 0.f);
            if (q < total) {
                const int j = coff + q;
                const float4 p = __ldg(a.pos4 + j);
                sv = make_float4(p.x + (float)(cur % 3 - 1) * L, p.y + (float)((cur / 3) % 3 - 1) * L,
                                 p.z + (float)(cur / 9 - 1) * L, __ldg(&a.vel4[j].w));
            }
            __syncwarp();
            sA[tl] = sv;
            __syncwarp();
#pragma unroll 8
            for (int k = 0; k < TW; ++k) {
                const float4 qk = sA[k];
                const float dx = qk.x - pi.x, dy = qk.y - pi.y, dz = qk.z - pi.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, a.eps2)));
                float inv = rsqrt_mufu(r2);
                if (!SOFT) inv = r2 > kGravMinR2 ? inv : 0.f;
                const float mi = qk.w * inv;
                bps += mi;
                const float mi3 = mi * inv * inv;
                bxs = fmaf(mi3, dx, bxs);
                bys = fmaf(mi3, dy, bys);
                bzs = fmaf(mi3, dz, bzs);
            }
            if ((ch + 1) % kFlush == 0 || ch == nch - 1) {
                kahan_add(sx, cx, bxs);
                kahan_add(sy, cy, bys);
                kahan_add(sz, cz, bzs);
                kahan_add(sp, cp, bps);
                bxs = bys = bzs = bps = 0.f;
            }
        }
        if (!valid) continue;
        // the target's own term: zero separation, so exactly m_i rsqrt(eps^2) in phi
        // and nothing in a
        if (SOFT) kahan_add(sp, cp, -(__ldg(&a.vel4[i].w) * rsqrt_mufu(a.eps2)));
        acc_pairs += (unsigned long long)(total - 1);
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
    const bool soft = a.eps2 >= kGravMinR2;
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
