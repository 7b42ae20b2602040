// sph_pairs.cu -- the two neighbour-sum passes of Theuns et al. 2015, Sec. 2-3.1:
//   density: Eq. 1 with the smoothing-length criterion (Newton on N_w(h) = N_ngb),
//            the velocity divergence/curl, and the per-particle quantities needed
//            before the pressure gradient (EOS, grad-h factor, Balsara switch);
//   force:   Eq. 2 in the Gadget-2 form with signal-velocity viscosity.
//
// Work decomposition (replaces the paper's self/pair tasks and task scheduler):
// one warp owns a tile of up to 32 target particles of one cell (one lane per
// target) and gathers from its own cell and the 26 adjacent cells (cells are no
// smaller than any h, Sec. 3.1).  Sources of each adjacent cell are read 32 at a
// time with one coalesced float4 load; a warp-parallel box test against the
// tile's bounding box (grown by the largest cutoff) stands in for the paper's
// sort-and-sweep pruning (Sec. 3.1, "sorting"): only sources that can reach some
// target survive the ballot, and each survivor is broadcast to all lanes by
// register shuffles.  Each target is written by exactly one lane, so the passes
// need no locks or atomics on particle data (the paper resolves the same write
// conflicts between tasks with locks).  Pair arithmetic is FP32 on cell-relative
// positions with compensated sums; distance tests within a few ulps of the
// cutoff are re-decided in FP64 so that neighbour sets are exact.
#include <algorithm>

#include "sph_internal.cuh"

namespace sph {

struct DensityArgs {
    const float4 *__restrict__ pos4;
    const float4 *__restrict__ vel4;
    const int *__restrict__ cell_start;
    const int4 *__restrict__ tiles;
    const int *__restrict__ n_tiles;
    const double *__restrict__ x;
    const double *__restrict__ y;
    const double *__restrict__ z;
    const int64_t *__restrict__ ids;
    const float *__restrict__ upred;
    uint8_t *active;
    float *h;
    float *rho, *P, *c, *f, *divv, *curl;
    int32_t *n_ngb;
    float4 *thermo4;
    uint64_t *ngb_hash;
    unsigned long long *counters;
    int nc;
    float L32;
    double box;
    float n_ngb_target, h_tol, gamma, h_cell_limit;
    int use_balsara;
    int last_pass;
};

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum_ull(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int wrapc(int j, int nc) { return j < 0 ? j + nc : (j >= nc ? j - nc : j); }

template <bool HASH>
__global__ void __launch_bounds__(256) k_density(DensityArgs a)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int ntiles = *a.n_tiles;
    const int nc = a.nc;
    const float L = a.L32;
    for (int t = gw; t < ntiles; t += nw) {
        const int4 tile = a.tiles[t];
        const int ca = tile.x, i = tile.y + lane;
        const bool valid = lane < tile.z;
        const bool act = valid && a.active[i];
        const unsigned amask = __ballot_sync(kFull, act);
        if (!amask) continue;
        float4 pi = valid ? a.pos4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float hi = act ? a.h[i] : 0.f;
        const float4 vi = act ? a.vel4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float inf = __int_as_float(0x7f800000);
        const float lox = warp_min(act ? pi.x : inf), hix = warp_max(act ? pi.x : -inf);
        const float loy = warp_min(act ? pi.y : inf), hiy = warp_max(act ? pi.y : -inf);
        const float loz = warp_min(act ? pi.z : inf), hiz = warp_max(act ? pi.z : -inf);
        const float hmax = warp_max(hi);
        // grown so that pairs the FP64 band re-decision may accept are never pruned
        const float reach2 = hmax * hmax * (1.f + kPruneMargin) + 2.f * kBandK * hmax * (hmax + L);
        const float hi2 = hi * hi;
        const float band = kBandK * hi * (hi + L);
        const float hinv = act ? 1.f / hi : 0.f;
        const int ix = ca % nc, iy = (ca / nc) % nc, iz = ca / (nc * nc);

        // sums; the self term (q = 0: w = sigma, w' = 0) starts them
        const float mi = vi.w;
        float rho_s = mi * kSigma, rho_c = 0.f;  // sum m_j w_j
        float sw_s = kSigma, sw_c = 0.f;          // sum w_j
        float sqdw = 0.f;                         // sum q_j w'_j
        float drho = 3.f * mi * kSigma;           // sum m_j (3 w_j + q_j w'_j)
        float dv = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
        int cnt = 0;
        uint64_t hh = 0;
        unsigned long long cand = 0;

        for (int oz = -1; oz <= 1; ++oz) {
            const int jz = wrapc(iz + oz, nc);
            for (int oy = -1; oy <= 1; ++oy) {
                const int jy = wrapc(iy + oy, nc);
                for (int ox = -1; ox <= 1; ++ox) {
                    const int jx = wrapc(ix + ox, nc);
                    const int cb = (jz * nc + jy) * nc + jx;
                    const float shx = (float)ox * L, shy = (float)oy * L, shz = (float)oz * L;
                    const int bs = a.cell_start[cb], be = a.cell_start[cb + 1];
                    for (int base = bs; base < be; base += 32) {
                        const int j = base + lane;
                        const bool has = j < be;
                        float sx = 0.f, sy = 0.f, sz = 0.f;
                        bool keep = false;
                        if (has) {
                            const float4 pj = __ldg(a.pos4 + j);
                            sx = pj.x + shx;
                            sy = pj.y + shy;
                            sz = pj.z + shz;
                            const float ex = fmaxf(fmaxf(lox - sx, sx - hix), 0.f);
                            const float ey = fmaxf(fmaxf(loy - sy, sy - hiy), 0.f);
                            const float ez = fmaxf(fmaxf(loz - sz, sz - hiz), 0.f);
                            keep = ex * ex + ey * ey + ez * ez < reach2;
                        }
                        unsigned mask = __ballot_sync(kFull, keep);
                        cand += (unsigned long long)__popc(mask);
                        while (mask) {
                            const int k = __ffs(mask) - 1;
                            mask &= mask - 1;
                            const float qx = __shfl_sync(kFull, sx, k);
                            const float qy = __shfl_sync(kFull, sy, k);
                            const float qz = __shfl_sync(kFull, sz, k);
                            const int jj = base + k;
                            if (act && jj != i) {
                                const float dx = pi.x - qx, dy = pi.y - qy, dz = pi.z - qz;
                                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                                bool in = r2 < hi2;
                                if (fabsf(r2 - hi2) <= band)
                                    in = within64(sep2_64(a.x, a.y, a.z, i, jj, a.box), hi);
                                if (in) {
                                    const float4 vj = __ldg(a.vel4 + jj);
                                    const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                                    const float q = r2 * rinv * hinv;
                                    float w, dw;
                                    spline(q, w, dw);
                                    const float mj = vj.w;
                                    kahan_add(rho_s, rho_c, mj * w);
                                    kahan_add(sw_s, sw_c, w);
                                    sqdw = fmaf(q, dw, sqdw);
                                    drho = fmaf(mj, fmaf(q, dw, 3.f * w), drho);
                                    const float fr = mj * dw * rinv;
                                    const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
                                    dv = fmaf(fr, fmaf(vx, dx, fmaf(vy, dy, vz * dz)), dv);
                                    cx = fmaf(fr, fmaf(vy, dz, -vz * dy), cx);
                                    cy = fmaf(fr, fmaf(vz, dx, -vx * dz), cy);
                                    cz = fmaf(fr, fmaf(vx, dy, -vy * dx), cz);
                                    ++cnt;
                                    if (HASH) hh += mix64((uint64_t)a.ids[jj]);
                                }
                            }
                        }
                    }
                }
            }
        }

        // counters (one atomic per warp)
        unsigned long long pairs = warp_sum_ull((unsigned long long)cnt);
        if (lane == 0) {
            atomicAdd(a.counters + C_DPAIRS, pairs);
            atomicAdd(a.counters + C_DCAND, cand * (unsigned long long)__popc(amask));
            atomicAdd(a.counters + C_DTARGETS, (unsigned long long)__popc(amask));
        }
        if (!act) continue;

        const float hinv3 = hinv * hinv * hinv, hinv4 = hinv3 * hinv;
        const float rho = hinv3 * (rho_s - rho_c);
        const float nw_ = kFourPi3 * (sw_s - sw_c);
        const float dnw_dh = -kFourPi3 * sqdw * hinv;
        const float drho_dh = -hinv4 * drho;
        const float divv = -hinv4 * dv / rho;
        const float curl = hinv4 * sqrtf(cx * cx + cy * cy + cz * cz) / rho;
        const float g = nw_ - a.n_ngb_target;
        const bool conv = fabsf(g) <= a.h_tol * a.n_ngb_target;
        if (!conv && !a.last_pass) {
            float hn = dnw_dh > 0.f ? hi - g / dnw_dh : (g < 0.f ? 2.f * hi : 0.5f * hi);
            hn = fminf(fmaxf(hn, 0.5f * hi), 2.f * hi);
            a.h[i] = hn;
            atomicAdd(a.counters + C_UNCONV, 1ull);
            if (hn > a.h_cell_limit) atomicOr(a.counters + C_HFLAG, 1ull);
            continue;
        }
        if (!conv) atomicAdd(a.counters + C_UNCONV, 1ull);
        a.active[i] = 0;
        // quantities needed before the pressure gradient (EOS, grad-h, Balsara)
        const float u = a.upred[i];
        const float gam = a.gamma;
        const float P = (gam - 1.f) * rho * u;
        const float cs = sqrtf(gam * (gam - 1.f) * u);
        const float fgh = 1.f / (1.f + hi / (3.f * rho) * drho_dh);
        float B = 1.f;
        if (a.use_balsara) {
            const float ad = fabsf(divv);
            const float den = ad + curl + 1e-4f * cs * hinv;
            B = den > 0.f ? ad / den : 0.f;
        }
        a.thermo4[i] = make_float4(rho, fgh * P / (rho * rho), cs, B);
        a.rho[i] = rho;
        a.P[i] = P;
        a.c[i] = cs;
        a.f[i] = fgh;
        a.divv[i] = divv;
        a.curl[i] = curl;
        a.n_ngb[i] = cnt;
        if (HASH) a.ngb_hash[i] = hh;
    }
}

struct ForceArgs {
    const float4 *__restrict__ pos4;
    const float4 *__restrict__ vel4;
    const float4 *__restrict__ thermo4;
    const int *__restrict__ cell_start;
    const int4 *__restrict__ tiles;
    const int *__restrict__ n_tiles;
    const double *__restrict__ x;
    const double *__restrict__ y;
    const double *__restrict__ z;
    const float *__restrict__ hmax_global;
    float *ax, *ay, *az, *dudt, *vsig;
    unsigned long long *counters;
    int nc;
    float L32;
    double box;
    float alpha;
};

__global__ void __launch_bounds__(256) k_force(ForceArgs a)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int ntiles = *a.n_tiles;
    const int nc = a.nc;
    const float L = a.L32;
    const float hglob = *a.hmax_global;
    for (int t = gw; t < ntiles; t += nw) {
        const int4 tile = a.tiles[t];
        const int ca = tile.x, i = tile.y + lane;
        const bool act = lane < tile.z;
        const unsigned amask = __ballot_sync(kFull, act);
        const float4 pi = act ? a.pos4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 vi = act ? a.vel4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 ti = act ? a.thermo4[i] : make_float4(1.f, 0.f, 0.f, 0.f);
        const float inf = __int_as_float(0x7f800000);
        const float lox = warp_min(act ? pi.x : inf), hix = warp_max(act ? pi.x : -inf);
        const float loy = warp_min(act ? pi.y : inf), hiy = warp_max(act ? pi.y : -inf);
        const float loz = warp_min(act ? pi.z : inf), hiz = warp_max(act ? pi.z : -inf);
        const float hi = pi.w;
        const float H = fmaxf(warp_max(hi), hglob);
        const float reach2 = H * H * (1.f + kPruneMargin) + 2.f * kBandK * H * (H + L);
        const float hi2 = hi * hi;
        const float hinv = act ? 1.f / hi : 0.f;
        const float hinv4 = hinv * hinv * hinv * hinv;
        const float band_i = kBandK * hi * (hi + L);
        const int ix = ca % nc, iy = (ca / nc) % nc, iz = ca / (nc * nc);
        const float rhoi = ti.x, Ai = ti.y, ci = ti.z, Bi = ti.w;
        float sx_ = 0.f, sxc = 0.f, sy_ = 0.f, syc = 0.f, sz_ = 0.f, szc = 0.f, su = 0.f, suc = 0.f;
        float vs = 0.f;
        int cnt = 0;
        unsigned long long cand = 0;
        for (int oz = -1; oz <= 1; ++oz) {
            const int jz = wrapc(iz + oz, nc);
            for (int oy = -1; oy <= 1; ++oy) {
                const int jy = wrapc(iy + oy, nc);
                for (int ox = -1; ox <= 1; ++ox) {
                    const int jx = wrapc(ix + ox, nc);
                    const int cb = (jz * nc + jy) * nc + jx;
                    const float shx = (float)ox * L, shy = (float)oy * L, shz = (float)oz * L;
                    const int bs = a.cell_start[cb], be = a.cell_start[cb + 1];
                    for (int base = bs; base < be; base += 32) {
                        const int j = base + lane;
                        const bool has = j < be;
                        float sx = 0.f, sy = 0.f, sz = 0.f, sh = 0.f;
                        bool keep = false;
                        if (has) {
                            const float4 pj = __ldg(a.pos4 + j);
                            sx = pj.x + shx;
                            sy = pj.y + shy;
                            sz = pj.z + shz;
                            sh = pj.w;
                            const float ex = fmaxf(fmaxf(lox - sx, sx - hix), 0.f);
                            const float ey = fmaxf(fmaxf(loy - sy, sy - hiy), 0.f);
                            const float ez = fmaxf(fmaxf(loz - sz, sz - hiz), 0.f);
                            keep = ex * ex + ey * ey + ez * ez < reach2;
                        }
                        unsigned mask = __ballot_sync(kFull, keep);
                        cand += (unsigned long long)__popc(mask);
                        while (mask) {
                            const int k = __ffs(mask) - 1;
                            mask &= mask - 1;
                            const float qx = __shfl_sync(kFull, sx, k);
                            const float qy = __shfl_sync(kFull, sy, k);
                            const float qz = __shfl_sync(kFull, sz, k);
                            const float hj = __shfl_sync(kFull, sh, k);
                            const int jj = base + k;
                            if (act && jj != i) {
                                const float dx = pi.x - qx, dy = pi.y - qy, dz = pi.z - qz;
                                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                                const float hj2 = hj * hj;
                                bool in_i = r2 < hi2, in_j = r2 < hj2;
                                const float band_j = kBandK * hj * (hj + L);
                                if (fabsf(r2 - hi2) <= band_i || fabsf(r2 - hj2) <= band_j) {
                                    const double r64 = sep2_64(a.x, a.y, a.z, i, jj, a.box);
                                    in_i = within64(r64, hi);
                                    in_j = within64(r64, hj);
                                }
                                if ((in_i || in_j) && r2 > 0.f) {
                                    const float4 vj = __ldg(a.vel4 + jj);
                                    const float4 tj = __ldg(a.thermo4 + jj);
                                    const float rinv = rsqrtf(r2);
                                    const float r = r2 * rinv;
                                    const float hjinv = __fdividef(1.f, hj);
                                    const float hj2inv = hjinv * hjinv;
                                    const float dWi = in_i ? spline_dw(r * hinv) * hinv4 : 0.f;
                                    const float dWj = in_j ? spline_dw(r * hjinv) * (hj2inv * hj2inv) : 0.f;
                                    const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
                                    const float mu = fmaf(vx, dx, fmaf(vy, dy, vz * dz)) * rinv;
                                    float Pi = 0.f;
                                    if (mu < 0.f)
                                        Pi = -a.alpha * (ci + tj.z - 3.f * mu) * mu * (0.5f * (Bi + tj.w)) /
                                             (rhoi + tj.x);
                                    const float dWbar = 0.5f * (dWi + dWj);
                                    const float mj = vj.w;
                                    const float s = mj * fmaf(Ai, dWi, fmaf(tj.y, dWj, Pi * dWbar)) * rinv;
                                    kahan_add(sx_, sxc, -s * dx);
                                    kahan_add(sy_, syc, -s * dy);
                                    kahan_add(sz_, szc, -s * dz);
                                    kahan_add(su, suc, mj * mu * fmaf(Ai, dWi, 0.5f * Pi * dWbar));
                                    vs = fmaxf(vs, ci + tj.z - 3.f * fminf(mu, 0.f));
                                    ++cnt;
                                } else if (in_i || in_j) {
                                    ++cnt;  // coincident pair: counted, no direction (w'(0) = 0)
                                }
                            }
                        }
                    }
                }
            }
        }
        unsigned long long pairs = warp_sum_ull((unsigned long long)cnt);
        if (lane == 0) {
            atomicAdd(a.counters + C_FPAIRS, pairs);
            atomicAdd(a.counters + C_FCAND, cand * (unsigned long long)__popc(amask));
        }
        if (!act) continue;
        a.ax[i] = sx_ - sxc;
        a.ay[i] = sy_ - syc;
        a.az[i] = sz_ - szc;
        a.dudt[i] = su - suc;
        a.vsig[i] = vs;
    }
}

__global__ void k_sync_h(const float *__restrict__ h, float4 *__restrict__ pos4, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pos4[i].w = h[i];
}

static int pair_grid(sph_ctx *ctx)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (sms <= 0) sms = 148;
    // persistent grid: 8 blocks of 8 warps per SM, warps stride over the tiles
    int64_t want = ((int64_t)ctx->n / kTile + ctx->grid.n_cells) / 8 + 1;
    int64_t g = std::min<int64_t>((int64_t)sms * 8, want);
    return (int)std::max<int64_t>(g, 1);
}

int run_density_pass(sph_ctx *ctx, sph_particles *parts, bool last_pass)
{
    DensityArgs a;
    a.pos4 = ctx->pos4;
    a.vel4 = ctx->vel4;
    a.cell_start = ctx->cell_start;
    a.tiles = ctx->tiles;
    a.n_tiles = ctx->n_tiles;
    a.x = parts->x;
    a.y = parts->y;
    a.z = parts->z;
    a.ids = ctx->ids;
    a.upred = ctx->upred;
    a.active = ctx->active;
    a.h = parts->h;
    a.rho = parts->rho;
    a.P = parts->P;
    a.c = parts->c;
    a.f = parts->f;
    a.divv = parts->divv;
    a.curl = parts->curl;
    a.n_ngb = parts->n_ngb;
    a.thermo4 = ctx->thermo4;
    a.ngb_hash = ctx->ngb_hash;
    a.counters = ctx->counters;
    a.nc = ctx->grid.nc;
    a.L32 = ctx->grid.L32;
    a.box = ctx->p.box_size;
    a.n_ngb_target = ctx->p.n_ngb;
    a.h_tol = ctx->p.h_tol;
    a.gamma = ctx->p.gamma;
    // largest h the current cells can hold (cells are no smaller than any h)
    a.h_cell_limit = (float)(ctx->grid.L64 * (1.0 - 1e-6));
    a.use_balsara = ctx->p.use_balsara;
    a.last_pass = last_pass ? 1 : 0;
    int g = pair_grid(ctx);
    cudaEvent_t end = nullptr;
    timer_begin(ctx, 0, &end);
    if (ctx->p.flags & SPH_FLAG_NGB_HASH)
        k_density<true><<<g, 256, 0, ctx->stream>>>(a);
    else
        k_density<false><<<g, 256, 0, ctx->stream>>>(a);
    timer_end(ctx, end);
    SPH_LAUNCH(ctx, "density kernel");
    ctx->st.density_passes++;
    return SPH_OK;
}

int run_force_pass(sph_ctx *ctx, sph_particles *parts)
{
    ForceArgs a;
    a.pos4 = ctx->pos4;
    a.vel4 = ctx->vel4;
    a.thermo4 = ctx->thermo4;
    a.cell_start = ctx->cell_start;
    a.tiles = ctx->tiles;
    a.n_tiles = ctx->n_tiles;
    a.x = parts->x;
    a.y = parts->y;
    a.z = parts->z;
    a.hmax_global = ctx->d_scalars;
    a.ax = parts->ax;
    a.ay = parts->ay;
    a.az = parts->az;
    a.dudt = parts->dudt;
    a.vsig = parts->vsig;
    a.counters = ctx->counters;
    a.nc = ctx->grid.nc;
    a.L32 = ctx->grid.L32;
    a.box = ctx->p.box_size;
    a.alpha = ctx->p.alpha_visc;
    int g = pair_grid(ctx);
    cudaEvent_t end = nullptr;
    timer_begin(ctx, 1, &end);
    k_force<<<g, 256, 0, ctx->stream>>>(a);
    timer_end(ctx, end);
    SPH_LAUNCH(ctx, "force kernel");
    ctx->st.force_passes++;
    return SPH_OK;
}

int sync_h(sph_ctx *ctx, sph_particles *parts)
{
    int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    k_sync_h<<<(n + 255) / 256, 256, 0, ctx->stream>>>(parts->h, ctx->pos4, n);
    SPH_LAUNCH(ctx, "sync h");
    return SPH_OK;
}

}  // namespace sph
