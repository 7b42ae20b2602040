// sph_cells.cu -- cubic cells no smaller than the smoothing length (Theuns et al.
// 2015, Sec. 3.1): periodic wrap, cell keys, a stable LSD radix sort of the
// particles by cell, the in-place permutation of the caller's arrays into cell
// order (particles of a cell contiguous in memory, Sec. 3.1), cell ranges and the
// warp work items (tiles of up to 16 or 32 targets of one cell).
#include <math.h>

#include <algorithm>

#include "sph_internal.cuh"

namespace sph {

// ----------------------------------------------------------------- exclusive scan

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread over the block; returns the block total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sh_warp, uint32_t &total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) sh_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < nw ? sh_warp[lane] : 0u;
        uint32_t ti = warp_incl_scan(t);
        if (lane < nw) sh_warp[lane] = ti - t;
        if (lane == 31) sh_warp[32] = ti;
    }
    __syncthreads();
    uint32_t r = sh_warp[w] + inc - v;
    total = sh_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in, int64_t n,
                                                              uint32_t *__restrict__ bsum)
{
    __shared__ uint32_t sh[33];
    int64_t base = (int64_t)blockIdx.x * kScanChunk;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    uint32_t tot;
    block_excl_scan(s, sh, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: in-place exclusive scan of nb block sums, in chunks with a carry
__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint32_t *bsum, int64_t nb)
{
    __shared__ uint32_t sh[33];
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        int64_t i = base + threadIdx.x;
        uint32_t v = i < nb ? bsum[i] : 0u;
        uint32_t tot;
        uint32_t e = block_excl_scan(v, sh, tot);
        if (i < nb) bsum[i] = carry + e;
        carry += tot;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t *in, uint32_t *out, int64_t n,
                                                            const uint32_t *__restrict__ bsum)
{
    __shared__ uint32_t sh[33];
    int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? in[i] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t e = block_excl_scan(s, sh, tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = e;
        e += v[k];
    }
}

int exclusive_scan_u32(sph_ctx *ctx, const uint32_t *in, uint32_t *out, int64_t n)
{
    if (n <= 0) return SPH_OK;
    int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb > kScanAuxCap) return fail(ctx, SPH_ERR_CAPACITY, "prefix sum longer than its block-sum scratch");
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(in, n, ctx->scan_aux);
    SPH_LAUNCH(ctx, "scan reduce");
    k_scan_top<<<1, kScanThreads, 0, ctx->stream>>>(ctx->scan_aux, nb);
    SPH_LAUNCH(ctx, "scan top");
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(in, out, n, ctx->scan_aux);
    SPH_LAUNCH(ctx, "scan down");
    return SPH_OK;
}

// ------------------------------------------------------------ LSD radix sort
// Keys are cell indices; 8-bit digits; one tile = 256 threads x 16 keys.  Ranks
// inside a tile are stable: warp w owns the contiguous sub-tile [w*512, w*512+512)
// and visits it in rounds of 32 consecutive keys; equal digits in a round are
// ranked by lane (match_any), rounds in order, warps in order.

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;  // 4096
constexpr int kRsWarps = kRsThreads / 32;

// dmask: the bits of the digit that take part (255, or fewer in the last pass of a
// sort whose key_bits is not a multiple of 8)
template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_radix_hist(const K *__restrict__ keys, int n, int shift,
                                                           uint32_t *__restrict__ hist, int ntiles,
                                                           uint32_t dmask = 255u)
{
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int k = 0; k < kRsItems; ++k) {
        int64_t i = base + k * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & dmask], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_radix_scatter(const K *__restrict__ kin,
                                                              const uint32_t *__restrict__ vin,
                                                              K *__restrict__ kout,
                                                              uint32_t *__restrict__ vout, int n, int shift,
                                                              const uint32_t *__restrict__ offs, int ntiles,
                                                              uint32_t dmask = 255u)
{
    __shared__ uint32_t wcnt[kRsWarps][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)w * (kRsItems * 32);
    const unsigned lt = (1u << lane) - 1u;
    K key[kRsItems];
    uint32_t val[kRsItems];
    uint16_t rank[kRsItems];
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        int64_t i = base + it * 32 + lane;
        bool ok = i < n;
        K k = ok ? kin[i] : (K)0;
        key[it] = k;
        val[it] = ok ? (vin ? vin[i] : (uint32_t)i) : 0u;
        uint32_t d = ok ? ((uint32_t)(k >> shift) & dmask) : 256u;
        unsigned peers = __match_any_sync(kFull, d);
        uint32_t before = ok ? wcnt[w][d] : 0u;
        rank[it] = (uint16_t)(before + __popc(peers & lt));
        __syncwarp();
        int leader = 31 - __clz(peers);
        if (ok && lane == leader) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix of the per-warp counts, per digit, in warp order
    __shared__ uint32_t woff[kRsWarps][256];
    {
        int d = threadIdx.x;  // 256 threads = 256 digits
        uint32_t s = 0;
#pragma unroll
        for (int ww = 0; ww < kRsWarps; ++ww) {
            woff[ww][d] = s;
            s += wcnt[ww][d];
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        int64_t i = base + it * 32 + lane;
        if (i < n) {
            uint32_t d = (uint32_t)(key[it] >> shift) & dmask;
            uint32_t dst = offs[(int64_t)d * ntiles + blockIdx.x] + woff[w][d] + rank[it];
            kout[dst] = key[it];
            vout[dst] = val[it];
        }
    }
}

// The same pass written through shared memory: the tile's keys are first placed in
// their order within the tile (the digit runs one after another, each run in the
// stable order above), then written out run by run, consecutive threads writing
// consecutive addresses (the plain scatter writes each key where it ranks, 256 runs
// interleaved).  Every key lands where k_radix_scatter puts it.
template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_radix_scatter_c(const K *__restrict__ kin,
                                                                const uint32_t *__restrict__ vin,
                                                                K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                                int n, int shift, const uint32_t *__restrict__ offs,
                                                                int ntiles)
{
    extern __shared__ __align__(16) unsigned char rs_smem[];
    K *sk = reinterpret_cast<K *>(rs_smem);                     // kRsTile keys in tile order
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kRsTile);  // and their values
    __shared__ uint32_t wcnt[kRsWarps][256];
    __shared__ uint32_t woff[kRsWarps][256];
    __shared__ uint32_t dstart[256];  // tile-local start of each digit's run
    __shared__ uint32_t gbase[256];   // global start of this tile's run of each digit
    __shared__ uint32_t wtot[kRsWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)w * (kRsItems * 32);
    const unsigned lt = (1u << lane) - 1u;
    K key[kRsItems];
    uint32_t val[kRsItems];
    uint16_t rank[kRsItems];
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        int64_t i = base + it * 32 + lane;
        bool ok = i < n;
        K k = ok ? kin[i] : (K)0;
        key[it] = k;
        val[it] = ok ? (vin ? vin[i] : (uint32_t)i) : 0u;
        uint32_t d = ok ? ((uint32_t)(k >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(kFull, d);
        uint32_t before = ok ? wcnt[w][d] : 0u;
        rank[it] = (uint16_t)(before + __popc(peers & lt));
        __syncwarp();
        int leader = 31 - __clz(peers);
        if (ok && lane == leader) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        // per digit (one thread each): warp-order offsets, the tile's count, and an
        // exclusive prefix of the counts over the digits (warp scans, then the warps')
        const int d = threadIdx.x;
        uint32_t c = 0;
#pragma unroll
        for (int ww = 0; ww < kRsWarps; ++ww) {
            woff[ww][d] = c;
            c += wcnt[ww][d];
        }
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wtot[w] = incl;
        __syncthreads();
        uint32_t before = 0;
        for (int ww = 0; ww < w; ++ww) before += wtot[ww];
        dstart[d] = before + incl - c;
        gbase[d] = offs[(int64_t)d * ntiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        int64_t i = base + it * 32 + lane;
        if (i < n) {
            const uint32_t d = (uint32_t)(key[it] >> shift) & 255u;
            const uint32_t p = dstart[d] + woff[w][d] + rank[it];
            sk[p] = key[it];
            sv[p] = val[it];
        }
    }
    __syncthreads();
    const int m = (int)min((int64_t)kRsTile, (int64_t)n - (int64_t)blockIdx.x * kRsTile);
    for (int p = threadIdx.x; p < m; p += kRsThreads) {
        const K k = sk[p];
        const uint32_t d = (uint32_t)(k >> shift) & 255u;
        const uint32_t dst = gbase[d] + ((uint32_t)p - dstart[d]);
        kout[dst] = k;
        vout[dst] = sv[p];
    }
}

template <typename K>
static size_t scatter_c_smem() { return (size_t)kRsTile * (sizeof(K) + sizeof(uint32_t)); }

// Stable LSD sort of keys[] (n entries, key_bits significant) with source slots as
// values (identity at the start); the sorted keys and slots end in keys[] / vals[]
// (the buffers are swapped on the host when the pass count is odd).
template <typename K>
static int radix_sort_any(sph_ctx *ctx, int n, int key_bits, K *&keys, K *&keys_alt)
{
    int ntiles = (n + kRsTile - 1) / kRsTile;
    static bool optin = false;  // (per function, once per process)
    if (!optin) {
        SPH_CUDA(ctx, cudaFuncSetAttribute(k_radix_scatter_c<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)scatter_c_smem<uint32_t>()));
        SPH_CUDA(ctx, cudaFuncSetAttribute(k_radix_scatter_c<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)scatter_c_smem<uint64_t>()));
        optin = true;
    }
    K *kin = keys, *kout = keys_alt;
    uint32_t *vin = nullptr, *vout = ctx->vals_alt;
    int passes = std::max(1, (key_bits + 7) / 8);
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_radix_hist<K><<<ntiles, kRsThreads, 0, ctx->stream>>>(kin, n, shift, ctx->hist, ntiles);
        SPH_LAUNCH(ctx, "radix histogram");
        int rc = exclusive_scan_u32(ctx, ctx->hist, ctx->hist, (int64_t)256 * ntiles);
        if (rc) return rc;
        k_radix_scatter_c<K><<<ntiles, kRsThreads, scatter_c_smem<K>(), ctx->stream>>>(kin, vin, kout, vout, n, shift,
                                                                                   ctx->hist, ntiles);
        SPH_LAUNCH(ctx, "radix scatter");
        std::swap(kin, kout);
        vin = vout;
        vout = (vin == ctx->vals_alt) ? ctx->vals : ctx->vals_alt;
    }
    if (kin != keys) std::swap(keys, keys_alt);
    if (vin != ctx->vals) std::swap(ctx->vals, ctx->vals_alt);
    return SPH_OK;
}

static int radix_sort(sph_ctx *ctx, int n, int key_bits) { return radix_sort_any(ctx, n, key_bits, ctx->keys, ctx->keys_alt); }

int radix_sort64(sph_ctx *ctx, int n, int key_bits)
{
    return radix_sort_any(ctx, n, key_bits, ctx->keys64, ctx->keys64_alt);
}

// -------------------------------------------------------- wrap, key, gather

// Wrap into [0, box): positions already inside (the common case) are returned
// unchanged without the FP64 division; others are shifted by box*floor(v/box) and
// corrected by one box if rounding left them just outside.
__device__ __forceinline__ double wrap64(double v, double box)
{
    if (v >= 0.0 && v < box) return v;
    double w = __dsub_rn(v, __dmul_rn(box, floor(__ddiv_rn(v, box))));
    if (w < 0.0) w = __dadd_rn(w, box);
    if (w >= box) w = __dsub_rn(w, box);
    if (w < 0.0 || w >= box) w = 0.0;
    return w;
}

// centre of cell index c along one axis, (c + 1/2) * L
__device__ __forceinline__ double centre64(int c, double L64) { return __dmul_rn(__dadd_rn((double)c, 0.5), L64); }

__device__ __forceinline__ int cell_of(double v, double s, int nc)
{
    int c = (int)floor(__dmul_rn(v, s));
    return c < 0 ? 0 : (c > nc - 1 ? nc - 1 : c);
}

// box owning particle slot p / global cell c (boxes are contiguous in both)
__device__ __forceinline__ int box_of_slot(int p, const BoxDev *__restrict__ bx, int nb)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bx[mid].p_begin <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int box_of_cell(int c, const BoxDev *__restrict__ bx, int nb)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bx[mid].cell_off <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// max h of every box (blockIdx.y = box, blockIdx.x strides its particles; the
// result is an atomic max of bit patterns into a zeroed slot).  h must be finite
// and > 0: NaN and negative values surface as NaN bits, which order above +inf.
__global__ void k_box_max_h(const float *__restrict__ h, const int64_t *__restrict__ off, unsigned *__restrict__ out)
{
    const int b = blockIdx.y;
    const int64_t lo = off[b], hi = off[b + 1];
    unsigned m = 0;
    for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned v = __float_as_uint(h[i]);
        if ((int)v < 0) v = 0x7fc00000u;
        m = max(m, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out + b, m);
}

int box_max_h(sph_ctx *ctx, const float *h)
{
    if (ctx->n <= 0) return SPH_OK;
    int64_t most = 0;
    for (int b = 0; b < ctx->n_boxes; ++b) most = std::max(most, ctx->box_off[b + 1] - ctx->box_off[b]);
    const unsigned bpb = (unsigned)std::min<int64_t>(512, std::max<int64_t>(1, most / 8192));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->d_box_hmax, 0, sizeof(float) * ctx->n_boxes, ctx->stream));
    k_box_max_h<<<dim3(bpb, ctx->n_boxes), 256, 0, ctx->stream>>>(h, ctx->d_box_off, (unsigned *)ctx->d_box_hmax);
    SPH_LAUNCH(ctx, "box max h");
    return SPH_OK;
}

struct WrapArgs {
    double *x, *y, *z;
    int n, nb;
    double box;
    const BoxDev *bx;
    uint32_t *keys;
};

// Wrap of one coordinate: positions already inside the box (FP32 test with a margin)
// are returned as they are; the others take the FP64 wrap.  Written back only if
// it moved.
__device__ __forceinline__ double wrap_coord(double *p, double box, float box_in)
{
    const double v = *p;
    const float vf = (float)v;
    if (vf > 0.f && vf < box_in) return v;
    const double w = wrap64(v, box);
    if (w != v) *p = w;
    return w;
}

// Cell index along one axis, floor(v s) clamped, and whether v lies in the upper half
// of that cell, v >= (c + 1/2) L -- as the FP64 forms cell_of / centre64 give them.
// The FP32 product t carries a relative error below 2e-7; where t lies further than
// eps = 1e-6 (t + 1) from an integer and from a half-integer both answers are those of
// the FP64 forms, else they are computed in FP64.
__device__ __forceinline__ int cell_half(double v, const BoxDev &g, float sf, unsigned &upper)
{
    const float t = __fmul_rn((float)v, sf);
    const float fl = floorf(t);
    const float fr = t - fl;
    const float eps = fmaf(t, 1e-6f, 1e-6f);
    if (fr > eps && fr < 1.f - eps && fabsf(fr - 0.5f) > eps && fl < (float)g.nc) {
        upper = fr >= 0.5f ? 1u : 0u;
        return (int)fl;
    }
    const int c = cell_of(v, g.s, g.nc);
    upper = v >= centre64(c, g.L64) ? 1u : 0u;
    return c;
}

__global__ void k_wrap_key(WrapArgs a)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const BoxDev g = a.bx[a.nb == 1 ? 0 : box_of_slot(i, a.bx, a.nb)];
    const float box_in = (float)a.box * (1.f - 1e-6f);
    const double x = wrap_coord(a.x + i, a.box, box_in), y = wrap_coord(a.y + i, a.box, box_in),
                 z = wrap_coord(a.z + i, a.box, box_in);
    const float sf = (float)g.s;
    unsigned ux, uy, uz;
    const int ix = cell_half(x, g, sf, ux), iy = cell_half(y, g, sf, uy), iz = cell_half(z, g, sf, uz);
    // key = cell * 8 + octant: inside a cell particles are grouped by octant (z
    // slowest), so the tiles of a cell split in two are each about half a cell
    const unsigned oct = ux | (uy << 1) | (uz << 2);
    a.keys[i] = ((uint32_t)(g.cell_off + (iz * g.nc + iy) * g.nc + ix) << 3) | oct;
}

struct GatherArgs {
    sph_particles P;
    const uint32_t *perm, *skeys;
    double *s64;
    float *s32;
    int64_t cap;
    const int64_t *ids_in;
    int64_t *ids_out;
    int ids_valid;
    float4 *pos4, *vel4;
    float *upred;
    const double *d_dt;  // non-null inside a step: predict v, u by d_dt/2
    int n, nb;
    const BoxDev *bx;
};

__global__ void k_gather(GatherArgs a)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n) return;
    int src = (int)a.perm[p];
    const sph_particles &P = a.P;
    double x = P.x[src], y = P.y[src], z = P.z[src];
    double vx = P.vx[src], vy = P.vy[src], vz = P.vz[src];
    float m = P.m[src], u = P.u[src], h = P.h[src];
    float ax = P.ax[src], ay = P.ay[src], az = P.az[src], du = P.dudt[src], vs = P.vsig[src];
    if (a.skeys) {
        const BoxDev g = a.bx[a.nb == 1 ? 0 : box_of_slot(p, a.bx, a.nb)];
        const int cell = (int)(a.skeys[p] >> 3) - g.cell_off;
        const int nc = g.nc;
        const int ix = cell % nc, iy = (cell / nc) % nc, iz = cell / (nc * nc);
        const double cx = centre64(ix, g.L64), cy = centre64(iy, g.L64), cz = centre64(iz, g.L64);
        a.pos4[p] = make_float4((float)(x - cx), (float)(y - cy), (float)(z - cz), h);
    }
    if (a.d_dt) {
        const double ph = 0.5 * *a.d_dt;
        a.vel4[p] = make_float4((float)(vx + (double)ax * ph), (float)(vy + (double)ay * ph),
                                (float)(vz + (double)az * ph), m);
        const double up = (double)u + (double)du * ph;
        a.upred[p] = (float)(up > 0.0 ? up : 0.0);
    } else {
        a.vel4[p] = make_float4((float)vx, (float)vy, (float)vz, m);
        a.upred[p] = u;
    }
    int64_t c = a.cap;
    a.s64[p] = x;
    a.s64[c + p] = y;
    a.s64[2 * c + p] = z;
    a.s64[3 * c + p] = vx;
    a.s64[4 * c + p] = vy;
    a.s64[5 * c + p] = vz;
    a.s32[p] = m;
    a.s32[c + p] = u;
    a.s32[2 * c + p] = h;
    a.s32[3 * c + p] = ax;
    a.s32[4 * c + p] = ay;
    a.s32[5 * c + p] = az;
    a.s32[6 * c + p] = du;
    a.s32[7 * c + p] = vs;
    // the previous hydro pass's divergence and neighbour count travel along (inputs
    // of the learned h guess)
    a.s32[8 * c + p] = P.divv[src];
    a.s32[9 * c + p] = __int_as_float(P.n_ngb[src]);
    a.ids_out[p] = a.ids_valid ? a.ids_in[src] : (int64_t)src;
}

// Copy the gathered arrays back into place (no pointer swaps: a captured step must
// read and write the same buffers on every replay).
__global__ void k_copy_back(sph_particles P, const double *__restrict__ s64, const float *__restrict__ s32,
                            const int64_t *__restrict__ ids_tmp, int64_t *__restrict__ ids, int64_t cap, int n)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t c = cap;
    ids[p] = ids_tmp[p];
    P.x[p] = s64[p];
    P.y[p] = s64[c + p];
    P.z[p] = s64[2 * c + p];
    P.vx[p] = s64[3 * c + p];
    P.vy[p] = s64[4 * c + p];
    P.vz[p] = s64[5 * c + p];
    P.m[p] = s32[p];
    P.u[p] = s32[c + p];
    P.h[p] = s32[2 * c + p];
    P.ax[p] = s32[3 * c + p];
    P.ay[p] = s32[4 * c + p];
    P.az[p] = s32[5 * c + p];
    P.dudt[p] = s32[6 * c + p];
    P.vsig[p] = s32[7 * c + p];
    P.divv[p] = s32[8 * c + p];
    P.n_ngb[p] = __float_as_int(s32[9 * c + p]);
}

// cell_start[c] = first slot with cell >= c (lower bound), c in [0, n_cells]
__global__ void k_cell_start(const uint32_t *__restrict__ skeys, int n, int64_t ncells, int *__restrict__ cs)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncells) return;
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((int64_t)(skeys[mid] >> 3) < c) lo = mid + 1;
        else hi = mid;
    }
    cs[c] = lo;
}

__global__ void k_cell_tiles(const int *__restrict__ cs, int64_t ncells, int tw, uint32_t *__restrict__ nt)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int cnt = cs[c + 1] - cs[c];
    nt[c] = (uint32_t)((cnt + tw - 1) / tw);
}

// tile = {global cell, first slot, count, box}
__global__ void k_tiles_write(const int *__restrict__ cs, int64_t ncells, int tw, const uint32_t *__restrict__ toff,
                              const BoxDev *__restrict__ bx, int nb, int4 *__restrict__ tiles,
                              int *__restrict__ n_tiles)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int s = cs[c], cnt = cs[c + 1] - s;
    uint32_t off = toff[c];
    const int box = nb == 1 ? 0 : box_of_cell((int)c, bx, nb);
    int k = 0;
    for (int b = 0; b < cnt; b += tw, ++k) tiles[off + k] = make_int4((int)c, s + b, min(tw, cnt - b), box);
    if (c == ncells - 1) *n_tiles = (int)(off + k);
}

__global__ void k_cell_of_key(const uint32_t *__restrict__ skeys, int n, int32_t *__restrict__ out)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) out[p] = (int32_t)(skeys[p] >> 3);
}

int cell_keys_out(sph_ctx *ctx, int32_t *dev_keys)
{
    const int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    k_cell_of_key<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->keys, n, dev_keys);
    SPH_LAUNCH(ctx, "cell keys");
    return SPH_OK;
}

// Largest h that can reach each cell: the max h of its particles, then the max of
// that over the 5 x 5 x 5 block of cells around it (periodic, within its box), done
// as three one-axis passes.  Any particle whose support reaches a cell lies in that
// block as long as every h is within two cell sides (beyond that the density pass
// flags the grid for re-planning).
__global__ void k_cell_hmax(const int *__restrict__ cs, const float4 *__restrict__ pos4, int64_t ncells,
                            float *__restrict__ out)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    float m = 0.f;
    for (int p = cs[c]; p < cs[c + 1]; ++p) m = fmaxf(m, pos4[p].w);
    out[c] = m;
}

__global__ void k_cell_max_axis(const float *__restrict__ in, float *__restrict__ out, int64_t ncells,
                                const BoxDev *__restrict__ bx, int nb, int axis)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const BoxDev g = bx[nb == 1 ? 0 : box_of_cell((int)c, bx, nb)];
    const int nc = g.nc, loc = (int)c - g.cell_off;
    int i3[3] = {loc % nc, (loc / nc) % nc, loc / (nc * nc)};
    float m = 0.f;
    for (int d = -2; d <= 2; ++d) {
        int j3[3] = {i3[0], i3[1], i3[2]};
        int v = i3[axis] + d;
        v = v < 0 ? v + nc : (v >= nc ? v - nc : v);
        v = v < 0 ? v + nc : (v >= nc ? v - nc : v);  // nc >= 3: two corrections suffice
        j3[axis] = v;
        m = fmaxf(m, in[g.cell_off + (j3[2] * nc + j3[1]) * nc + j3[0]]);
    }
    out[c] = m;
}

int cell_reach(sph_ctx *ctx)
{
    const int64_t nc = ctx->grid.n_cells;
    const unsigned blocks = (unsigned)((nc + 255) / 256);
    k_cell_hmax<<<blocks, 256, 0, ctx->stream>>>(ctx->cell_start, ctx->pos4, nc, ctx->cell_hmax);
    SPH_LAUNCH(ctx, "cell max h");
    k_cell_max_axis<<<blocks, 256, 0, ctx->stream>>>(ctx->cell_hmax, ctx->cell_tmp, nc, ctx->d_boxes, ctx->n_boxes, 0);
    SPH_LAUNCH(ctx, "cell reach x");
    k_cell_max_axis<<<blocks, 256, 0, ctx->stream>>>(ctx->cell_tmp, ctx->cell_hmax, nc, ctx->d_boxes, ctx->n_boxes, 1);
    SPH_LAUNCH(ctx, "cell reach y");
    k_cell_max_axis<<<blocks, 256, 0, ctx->stream>>>(ctx->cell_hmax, ctx->cell_tmp, nc, ctx->d_boxes, ctx->n_boxes, 2);
    SPH_LAUNCH(ctx, "cell reach z");  // result in cell_tmp
    return SPH_OK;
}

static int ensure_cells(sph_ctx *ctx, int64_t ncells)
{
    if (ncells + 1 > ctx->cell_cap) {
        cudaFree(ctx->cell_start);
        cudaFree(ctx->cell_tiles);
        cudaFree(ctx->cell_hmax);
        cudaFree(ctx->cell_tmp);
        ctx->cell_start = nullptr;
        ctx->cell_tiles = nullptr;
        ctx->cell_hmax = nullptr;
        ctx->cell_tmp = nullptr;
        int64_t cap = ncells + 1 + 1024;
        SPH_CUDA(ctx, cudaMalloc(&ctx->cell_start, sizeof(int) * cap));
        SPH_CUDA(ctx, cudaMalloc(&ctx->cell_tiles, sizeof(uint32_t) * cap));
        SPH_CUDA(ctx, cudaMalloc(&ctx->cell_hmax, sizeof(float) * cap));
        SPH_CUDA(ctx, cudaMalloc(&ctx->cell_tmp, sizeof(float) * cap));
        ctx->cell_cap = cap;
    }
    // the scan of per-cell tile counts needs ceil(ncells / chunk) block sums
    int64_t nb = (ncells + kScanChunk - 1) / kScanChunk + 1;
    if (nb > kScanAuxCap) return fail(ctx, SPH_ERR_INVALID_ARG, "cell grid too large for scan scratch");
    return SPH_OK;
}

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Plan the cell grid of every box from its largest h (one host read): the cell
// side is the smallest L = box / nc with L >= cell_factor * max h and nc >= 3 (cells
// no smaller than the smoothing length, Sec. 3.1), nc capped near (8 n_box)^(1/3).
// max h of every box into ctx->h_box_hmax (one host read)
int read_box_max_h(sph_ctx *ctx, sph_particles *parts)
{
    if (ctx->n <= 0) return SPH_OK;
    int rc = box_max_h(ctx, parts->h);
    if (rc) return rc;
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_box_hmax, ctx->d_box_hmax, sizeof(float) * ctx->n_boxes,
                                  cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SPH_OK;
}

// True while the current plan still suits the particles: every box's max h within
// 1.8 cell sides (the radius-2 stencil reaches two) and not far below the side the
// cell factor asks for (cells much larger than needed cost candidates).
bool plan_still_good(sph_ctx *ctx)
{
    if (!ctx->planned) return false;
    for (int b = 0; b < ctx->n_boxes; ++b) {
        if (ctx->box_off[b + 1] == ctx->box_off[b]) continue;
        const double h = ctx->h_box_hmax[b], L = ctx->h_boxes[b].L64;
        if (!(h > 0) || h > 1.8 * L || h * ctx->p.cell_factor < 0.6 * L) return false;
    }
    return true;
}

int plan_cells(sph_ctx *ctx, sph_particles *parts)
{
    int rc = read_box_max_h(ctx, parts);
    if (rc) return rc;
    return plan_from_hmax(ctx);
}

int plan_from_hmax(sph_ctx *ctx)
{
    const double box = ctx->p.box_size;
    const int nb = ctx->n_boxes;
    BoxDev *hb = ctx->h_boxes;
    int64_t cells = 0;
    for (int b = 0; b < nb; ++b) {
        const int64_t np = ctx->box_off[b + 1] - ctx->box_off[b];
        float hmax = np > 0 ? ctx->h_box_hmax[b] : (float)(box / 4.0);  // empty box: coarsest grid
        if (!(hmax > 0.f) || !isfinite(hmax)) return fail(ctx, SPH_ERR_NAN, "smoothing lengths must be finite and > 0");
        int nc = (int)floor(box / ((double)hmax * (double)ctx->p.cell_factor));
        const int cap_n = (int)floor(cbrt(8.0 * (double)std::max<int64_t>(np, 1)));
        if (ctx->adaptive) {
            // the leaf lists take every periodic image of the 27 top cells around a
            // leaf, so one or two top cells per side are fine; the minimum-image
            // convention still needs h below half the box
            if ((double)hmax >= 0.5 * box * (1.0 - 1e-6))
                return fail(ctx, SPH_ERR_H_EXCEEDS_CELL, "max h reaches box/2: no unique periodic image");
            nc = std::max(1, std::min(nc, std::min(kMaxNc, std::max(1, cap_n))));
        } else {
            if ((double)hmax > box / 3.0)
                return fail(ctx, SPH_ERR_H_EXCEEDS_CELL, "max h exceeds box/3: no periodic grid with >= 3 cells");
            nc = std::min(nc, std::min(kMaxNc, std::max(3, cap_n)));
            if (nc < 3) nc = 3;  // hmax <= box/3 guarantees cells of side box/3 hold the support
        }
        hb[b].p_begin = (int)ctx->box_off[b];
        hb[b].p_end = (int)ctx->box_off[b + 1];
        hb[b].cell_off = (int)cells;
        hb[b].nc = nc;
        hb[b].L64 = box / nc;
        hb[b].s = (double)nc / box;
        hb[b].L32 = (float)hb[b].L64;
        hb[b].hplan = hmax;
        cells += (int64_t)nc * nc * nc;
        if (cells * 8 >= (1ll << 32)) return fail(ctx, SPH_ERR_INVALID_ARG, "too many cells for 32-bit keys");
    }
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->d_boxes, hb, sizeof(BoxDev) * nb, cudaMemcpyHostToDevice, ctx->stream));
    Grid &g = ctx->grid;
    g.nc = hb[0].nc;
    g.n_cells = cells;
    g.L64 = hb[0].L64;
    int bits = 1;
    while ((1ll << bits) < g.n_cells) ++bits;
    g.key_bits = bits + 3;  // octant within the cell
    int rc = ensure_cells(ctx, g.n_cells);
    if (rc) return rc;
    ctx->planned = true;
    ctx->st.nc = g.nc;
    ctx->st.n_cells = g.n_cells;
    ctx->st.cell_size = g.L64;
    return SPH_OK;
}

// Gather every particle array into the sorted order held in ctx->vals and copy it
// back in place; cell_pos: also write pos4 relative to the uniform cell centres
// (keys in ctx->keys), else pos4 is written by the caller.
int permute_particles(sph_ctx *ctx, sph_particles *parts, bool cell_pos)
{
    const int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    GatherArgs ga{};
    ga.P = *parts;
    ga.perm = ctx->vals;
    ga.skeys = cell_pos ? ctx->keys : nullptr;
    ga.s64 = ctx->s64;
    ga.s32 = ctx->s32;
    ga.cap = ctx->cap;
    ga.ids_in = ctx->ids;
    ga.ids_out = ctx->ids_tmp;
    ga.ids_valid = ctx->ids_valid ? 1 : 0;
    ga.pos4 = ctx->pos4;
    ga.vel4 = ctx->vel4;
    ga.upred = ctx->upred;
    ga.d_dt = ctx->predict ? ctx->d_dt : nullptr;
    ga.n = n;
    ga.nb = ctx->n_boxes;
    ga.bx = ctx->d_boxes;
    k_gather<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(ga);
    SPH_LAUNCH(ctx, "gather");
    k_copy_back<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(*parts, ctx->s64, ctx->s32, ctx->ids_tmp, ctx->ids,
                                                             ctx->cap, n);
    SPH_LAUNCH(ctx, "copy back");
    ctx->ids_valid = true;
    // individual time-steps: bins, kept density outputs and per-particle prediction
    if (ctx->bin_mode) return bin_permute(ctx, parts);
    return SPH_OK;
}

// Bin, sort and permute with the current plan: no host synchronisation.
int build_planned(sph_ctx *ctx, sph_particles *parts)
{
    if (!ctx->planned) return fail(ctx, SPH_ERR_STATE, "no cell plan");
    if (ctx->adaptive) return build_tree(ctx, parts);
    const int n = (int)ctx->n;
    const Grid &g = ctx->grid;
    int rc;
    if (n > 0) {
        WrapArgs wa{parts->x, parts->y, parts->z, n, ctx->n_boxes, ctx->p.box_size, ctx->d_boxes, ctx->keys};
        k_wrap_key<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(wa);
        SPH_LAUNCH(ctx, "wrap/key");
        rc = radix_sort(ctx, n, g.key_bits);
        if (rc) return rc;
        rc = permute_particles(ctx, parts, true);
        if (rc) return rc;
    }
    k_cell_start<<<blocks_for(g.n_cells + 1, 256), 256, 0, ctx->stream>>>(ctx->keys, n, g.n_cells, ctx->cell_start);
    SPH_LAUNCH(ctx, "cell start");
    k_cell_tiles<<<blocks_for(g.n_cells, 256), 256, 0, ctx->stream>>>(ctx->cell_start, g.n_cells, ctx->tile_w,
                                                                     ctx->cell_tiles);
    SPH_LAUNCH(ctx, "cell tiles");
    rc = exclusive_scan_u32(ctx, ctx->cell_tiles, ctx->cell_tiles, g.n_cells);
    if (rc) return rc;
    k_tiles_write<<<blocks_for(g.n_cells, 256), 256, 0, ctx->stream>>>(
        ctx->cell_start, g.n_cells, ctx->tile_w, ctx->cell_tiles, ctx->d_boxes, ctx->n_boxes, ctx->tiles,
        ctx->n_tiles);
    SPH_LAUNCH(ctx, "tiles");
    if ((ctx->p.flags & SPH_FLAG_AXIS_SWEEP) && n > 0) {
        rc = axis_sort(ctx);
        if (rc) return rc;
    }
    ctx->built = true;
    ctx->density_valid = false;
    return SPH_OK;
}

// ------------------------------------------------------ per-axis cell orders
// Sec. 3.1 ("sorting"): the particles of a cell, sorted by their projection on the
// axis joining it to a neighbour, let a pair sweep stop once the projected distance
// exceeds the cutoff.  The 13 directions of a half stencil cover all 26 neighbours
// (a neighbour in direction -d reads the order of d backwards).

__constant__ signed char kAxisDir[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0},  {1, -1, 0},
                                            {1, 0, 1},  {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},
                                            {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
constexpr int kAxisMax = 256;  // cells above this keep slot order (their sweep never stops early)
constexpr int kAxisWarps = 4;

// one warp per cell: projections (cell-relative FP32 positions, unit directions) and
// their ranks (ties by slot); a cell too large for the shared buffer is written in
// slot order with projections -inf, so that no sweep stops inside it
__global__ void __launch_bounds__(32 * kAxisWarps) k_axis_sort(const int *__restrict__ cs, int64_t ncells,
                                                                const float4 *__restrict__ pos4, int64_t cap,
                                                                float2 *__restrict__ axis)
{
    __shared__ float sp[kAxisWarps][kAxisMax];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * kAxisWarps + wib;
    if (c >= ncells) return;  // warp-uniform
    const int b = cs[c], cnt = cs[c + 1] - b;
    for (int d = 0; d < 13; ++d) {
        const float dx = kAxisDir[d][0], dy = kAxisDir[d][1], dz = kAxisDir[d][2];
        const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        float2 *out = axis + (size_t)d * cap + b;
        if (cnt > kAxisMax) {
            for (int k = lane; k < cnt; k += 32) out[k] = make_float2(-INFINITY, __int_as_float(b + k));
            continue;
        }
        for (int k = lane; k < cnt; k += 32) {
            const float4 p = pos4[b + k];
            sp[wib][k] = (p.x * dx + p.y * dy + p.z * dz) * inv;
        }
        __syncwarp();
        for (int k = lane; k < cnt; k += 32) {
            const float sk = sp[wib][k];
            int rank = 0;
            for (int m = 0; m < cnt; ++m) {
                const float sm = sp[wib][m];
                rank += (sm < sk || (sm == sk && m < k)) ? 1 : 0;
            }
            out[rank] = make_float2(sk, __int_as_float(b + k));
        }
        __syncwarp();
    }
}

int axis_sort(sph_ctx *ctx)
{
    const int64_t need = 13 * std::max<int64_t>(ctx->cap, 1);
    if (ctx->axis_cap < need) {
        cudaFree(ctx->axis);
        ctx->axis = nullptr;
        ctx->axis_cap = 0;
        SPH_CUDA(ctx, cudaMalloc(&ctx->axis, sizeof(float2) * need));
        ctx->axis_cap = need;
    }
    const int64_t nc = ctx->grid.n_cells;
    k_axis_sort<<<(unsigned)((nc + kAxisWarps - 1) / kAxisWarps), 32 * kAxisWarps, 0, ctx->stream>>>(
        ctx->cell_start, nc, ctx->pos4, std::max<int64_t>(ctx->cap, 1), ctx->axis);
    SPH_LAUNCH(ctx, "axis sort");
    return SPH_OK;
}

int build_cells(sph_ctx *ctx, sph_particles *parts)
{
    int rc = plan_cells(ctx, parts);
    if (rc) return rc;
    return build_planned(ctx, parts);
}

}  // namespace sph

// ------------------------------------------------- sort without allocation
// sph_sort_keys_static: the stable LSD radix sort above, for callers that cannot
// allocate device memory.  Its scratch (one ping-pong set of keys and source
// slots, the per-tile digit histograms and the scan's block sums) is a
// file-scope static device array of fixed size, so any process that loads
// libsph holds it on every GPU it uses, until exit.

namespace sph {

constexpr int64_t kStaticSortTiles = (SPH_SORT_STATIC_MAX_N + kRsTile - 1) / kRsTile;
constexpr int64_t kStaticHist = 256 * kStaticSortTiles;
constexpr int64_t kStaticAux = (kStaticHist + kScanChunk - 1) / kScanChunk + 1;
constexpr int64_t kStaticWords = 2 * SPH_SORT_STATIC_MAX_N + kStaticHist + kStaticAux;

static __device__ __align__(256) uint32_t g_sort_scratch[kStaticWords];

// Device address of g_sort_scratch on the current device.  The host-side symbol is
// only a stand-in and must never reach a kernel.  The lookup runs on every call (it
// is a table lookup once the module is loaded), so an address can never outlive a
// cudaDeviceReset; the first call on a device loads the module.
static cudaError_t static_scratch(uint32_t **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    *out = (uint32_t *)p;
    return cudaSuccess;
}

// [a, a + bytes) and [b, b + bytes) share a byte
static bool overlap(const void *a, const void *b, size_t bytes)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bytes && y < x + bytes;
}

}  // namespace sph

extern "C" int sph_sort_keys_static(const uint32_t *keys_in, uint32_t *keys_out, uint32_t *perm_out, int64_t n,
                                    int32_t key_bits, void *cuda_stream)
{
    using namespace sph;
    if (n < 0 || n > SPH_SORT_STATIC_MAX_N || key_bits < 1 || key_bits > 32) return SPH_ERR_INVALID_ARG;
    if (n == 0) return SPH_OK;
    if (!keys_in || !keys_out || !perm_out) return SPH_ERR_INVALID_ARG;
    // a pass reads keys that other blocks of the same pass may already have overwritten
    // if the outputs alias the input or each other
    const size_t bytes = sizeof(uint32_t) * (size_t)n;
    if (overlap(keys_in, keys_out, bytes) || overlap(keys_in, perm_out, bytes) || overlap(keys_out, perm_out, bytes))
        return SPH_ERR_INVALID_ARG;
    // an error left pending by earlier, unrelated work is not this call's to report or
    // to clear: refuse to run on top of it
    if (cudaPeekAtLastError() != cudaSuccess) return SPH_ERR_CUDA;
    uint32_t *scratch = nullptr;
    if (static_scratch(&scratch) != cudaSuccess) return SPH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint32_t *sk = scratch, *sv = scratch + SPH_SORT_STATIC_MAX_N;
    uint32_t *hist = scratch + 2 * SPH_SORT_STATIC_MAX_N, *aux = hist + kStaticHist;
    const int nn = (int)n;
    const int ntiles = (nn + kRsTile - 1) / kRsTile;
    const int passes = (key_bits + 7) / 8;
    const int64_t nh = (int64_t)256 * ntiles;
    const int64_t nb = (nh + kScanChunk - 1) / kScanChunk;
    // ping-pong between the static buffers and the outputs so that the last
    // pass writes the outputs; every histogram and block sum is rewritten each
    // pass, so nothing left by an earlier call is read
    const uint32_t *kin = keys_in, *vin = nullptr;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t *kout = to_out ? keys_out : sk, *vout = to_out ? perm_out : sv;
        const int shift = 8 * p;
        // the last digit keeps only the bits below key_bits: higher bits take no part
        const int top = key_bits - shift;  // 1..8 in the last pass
        const uint32_t dmask = top >= 8 ? 255u : (1u << top) - 1u;
        k_radix_hist<uint32_t><<<ntiles, kRsThreads, 0, st>>>(kin, nn, shift, hist, ntiles, dmask);
        if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
        k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(hist, nh, aux);
        if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
        k_scan_top<<<1, kScanThreads, 0, st>>>(aux, nb);
        if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
        k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(hist, hist, nh, aux);
        if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
        k_radix_scatter<uint32_t><<<ntiles, kRsThreads, 0, st>>>(kin, vin, kout, vout, nn, shift, hist, ntiles, dmask);
        if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
        kin = kout;
        vin = vout;
    }
    return SPH_OK;
}
