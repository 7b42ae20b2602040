// sph_pairs.cu -- the two neighbour-sum passes of Theuns et al. 2015, Sec. 2-3.1:
//   density: Eq. 1 with the smoothing-length criterion (Newton on N_w(h) = N_ngb),
//            the velocity divergence/curl, and the per-particle quantities needed
//            before the pressure gradient (EOS, grad-h factor, Balsara switch);
//   force:   Eq. 2 in the Gadget-2 form with signal-velocity viscosity.
//
// Work decomposition (replaces the paper's self/pair tasks and task scheduler):
// a tile is up to TW (16 or 32) target particles of one cell, one lane per
// target; a warp holds 32/TW tiles.  Each tile gathers from its own cell and the
// 26 adjacent cells (cells are no smaller than any h, Sec. 3.1), so every target
// is written by exactly one lane: no locks or atomics on particle data (the paper
// resolves the same write conflicts between tasks with locks).
//
// Per tile, sources arrive TW at a time by one coalesced float4 load and are
// tested against the tile's bounding box grown by the cutoff -- the warp-parallel
// stand-in for the paper's sort-and-sweep pruning (Sec. 3.1, "sorting").  The
// survivors are compacted into a per-tile batch in shared memory.  A full batch
// is processed in two phases:
//   1. distance tests: every lane tests its target against each staged source
//      (broadcast shared-memory reads) and records its hits in a 64-bit mask;
//   2. interactions: every lane walks only its own hits.
// so the interaction body never runs for a lane that does not need it.
// Pair arithmetic is FP32 on cell-relative positions; the terms of one staged batch
// are summed plainly and the batch sums are accumulated with Kahan compensation;
// distance tests within a few ulps of the cutoff are re-decided in FP64 so that
// neighbour sets are exact.
#include <algorithm>

#include "sph_internal.cuh"

namespace sph {

constexpr int kBatchD = 128;  // staged survivors per tile, density (4 hit-mask words)
constexpr int kBatchF = 128;  // staged survivors per tile, force
constexpr int kSlotF = 132;   // floats per staged-coordinate array (>= kBatchD, even: 8-byte aligned pairs)
constexpr int kPairThreads = 256;
// Adaptive cells (leaf lists): the tiles' targets span a range of h, so their hit
// counts in a batch differ widely.  The density and force passes therefore cut a
// batch's hits into equal contiguous ranges, one per lane (the balanced walk of
// k_density and k_force), with the tile's targets in shared memory for the lanes that
// move from one target's hits to the next; measured on the 512 uneven boxes against
// the earlier walk (lane by lane while enough lanes had a hit left, then one
// compacted warp-wide list with a segmented scan): force 7.5 % faster.  The uniform
// grid's batches mix cells on both sides of the tile, so their hits spread over the
// lanes: its kernels walk lane by lane only.
constexpr int kWalkBytesD = 148;  // density pass, list mode: the balanced walk's scratch per target
constexpr int kWalkBytes = 148;   // force pass, list mode: the balanced walk's scratch per target
constexpr int kDensityBlocks = 2;  // resident blocks per SM the density kernel is compiled for
constexpr int kForceBlocks = 2;      // leaf lists (adaptive cells): 3 would spill (328 B at 80 registers)
constexpr int kForceBlocksU = 3;     // uniform grid: a third block per SM outweighs a few spilled values
// Padding sources sit at -kFar and target-less lanes at +kFar: the squared distance
// between either and anything else overflows to +inf, so no test can pass.
constexpr float kFar = 1e30f;
// an h bracket end at or above this is open (the bytes 0x7f7f7f7f read 3.39e38)
constexpr float kHUnbounded = 3e38f;
// relative width of an h bracket at which the iteration stops refining (2^-21: 4 to 8
// FP32 ulps of h); near the root the FP32 neighbour sums are noisy at about this level
// of h, so that for particles whose N_w is very sensitive to h a tolerance far below
// 1e-5 may have no FP32 h that meets it
constexpr float kHResolution = 4.76837158e-7f;

// Neighbour cells in visiting order: the own cell, then each of the 13 directions
// of a half stencil followed by its opposite, so that every staged batch mixes
// cells on both sides of the tile and the lanes' hit counts stay balanced.
__constant__ signed char kOrder[27][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},   {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},    {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},   {1, 1, 1},  {-1, -1, -1},
    {1, 1, -1},  {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},   {1, -1, -1}};

// Radius-2 stencils visit the 27 cells above, in that order, then the 98 cells at
// distance two (z, y, x lexicographic), so a tile's summation order never depends
// on which stencil its warp runs.
__constant__ signed char kOuter[98][3] = {
    {-2, -2, -2}, {-1, -2, -2}, {0, -2, -2}, {1, -2, -2}, {2, -2, -2}, {-2, -1, -2}, {-1, -1, -2},
    {0, -1, -2}, {1, -1, -2}, {2, -1, -2}, {-2, 0, -2}, {-1, 0, -2}, {0, 0, -2}, {1, 0, -2},
    {2, 0, -2}, {-2, 1, -2}, {-1, 1, -2}, {0, 1, -2}, {1, 1, -2}, {2, 1, -2}, {-2, 2, -2},
    {-1, 2, -2}, {0, 2, -2}, {1, 2, -2}, {2, 2, -2}, {-2, -2, -1}, {-1, -2, -1}, {0, -2, -1},
    {1, -2, -1}, {2, -2, -1}, {-2, -1, -1}, {2, -1, -1}, {-2, 0, -1}, {2, 0, -1}, {-2, 1, -1},
    {2, 1, -1}, {-2, 2, -1}, {-1, 2, -1}, {0, 2, -1}, {1, 2, -1}, {2, 2, -1}, {-2, -2, 0},
    {-1, -2, 0}, {0, -2, 0}, {1, -2, 0}, {2, -2, 0}, {-2, -1, 0}, {2, -1, 0}, {-2, 0, 0},
    {2, 0, 0}, {-2, 1, 0}, {2, 1, 0}, {-2, 2, 0}, {-1, 2, 0}, {0, 2, 0}, {1, 2, 0},
    {2, 2, 0}, {-2, -2, 1}, {-1, -2, 1}, {0, -2, 1}, {1, -2, 1}, {2, -2, 1}, {-2, -1, 1},
    {2, -1, 1}, {-2, 0, 1}, {2, 0, 1}, {-2, 1, 1}, {2, 1, 1}, {-2, 2, 1}, {-1, 2, 1},
    {0, 2, 1}, {1, 2, 1}, {2, 2, 1}, {-2, -2, 2}, {-1, -2, 2}, {0, -2, 2}, {1, -2, 2},
    {2, -2, 2}, {-2, -1, 2}, {-1, -1, 2}, {0, -1, 2}, {1, -1, 2}, {2, -1, 2}, {-2, 0, 2},
    {-1, 0, 2}, {0, 0, 2}, {1, 0, 2}, {2, 0, 2}, {-2, 1, 2}, {-1, 1, 2}, {0, 1, 2},
    {1, 1, 2}, {2, 1, 2}, {-2, 2, 2}, {-1, 2, 2}, {0, 2, 2}, {1, 2, 2}, {2, 2, 2},};

// SPH_FLAG_AXIS_SWEEP: for stencil cell o (kOrder index) the direction d of the 13
// half-stencil axes with kOrder[o] = sign * axis d, and |axis d| (1, sqrt 2, sqrt 3)
__constant__ signed char kOrderAxis[27][2] = {
    {-1, 0}, {0, 1},  {0, -1}, {1, 1},  {1, -1}, {2, 1},   {2, -1},  {3, 1},  {3, -1},
    {4, 1},  {4, -1}, {5, 1},  {5, -1}, {6, 1},  {6, -1},  {7, 1},   {7, -1}, {8, 1},
    {8, -1}, {9, 1},  {9, -1}, {10, 1}, {10, -1}, {11, 1}, {11, -1}, {12, -1}, {12, 1}};
__constant__ float kAxisLen[13] = {1.f, 1.f, 1.f, 1.41421356f, 1.41421356f, 1.41421356f, 1.41421356f,
                                   1.41421356f, 1.41421356f, 1.73205081f, 1.73205081f, 1.73205081f, 1.73205081f};

// Sweep bound of a neighbour cell: a source whose projection on the unit vector u from
// the tile's cell towards it (relative to the neighbour's centre; = sign x its stored
// projection on axis d) reaches lim or more is farther than rlim from every target of
// the tile, whose box is [lo, hi] -- projected distance never exceeds distance.  The
// bound is loosened by 1e-5 L against FP32 rounding.
__device__ __forceinline__ float sweep_limit(int o, float L, float rlim, float lox, float hix, float loy, float hiy,
                                             float loz, float hiz)
{
    const float len = kAxisLen[kOrderAxis[o][0]];
    // u points from the tile's cell to the neighbour (kOrder[o] = sign * axis d)
    const float ux = kOrder[o][0] / len, uy = kOrder[o][1] / len, uz = kOrder[o][2] / len;
    const float tmax = fmaxf(lox * ux, hix * ux) + fmaxf(loy * uy, hiy * uy) + fmaxf(loz * uz, hiz * uz);
    return rlim + tmax - len * L + 1e-5f * L;
}

// The sources of a tile's leaf list as one stream (adaptive cells).  The TW entries
// of a window are fetched at once (lane tl: entry wb + tl), their particle counts are
// prefix-summed across the TW lanes, and chunk ch of the window covers stream
// positions [ch TW, ch TW + TW): leaves much smaller than TW share a chunk instead of
// each leaving lanes idle.  The stream order -- entries in list order, particles in
// slot order -- is that of the entries taken one by one.
template <int TW>
struct ListStream {
    int wb = -TW;  // first entry of the window (warp-uniform)
    int incl = 0;  // prefix count of the window's entries up to this lane's, inclusive
    int st = 0;    // stream position of this lane's entry (its first particle)
    int sb = 0;    // first slot of this lane's entry minus its stream position
    int tot = 0;   // particles in this tile's window
    float px = 0.f, py = 0.f, pz = 0.f;  // offset of this lane's entry

    // next window (warp-uniform); false once the longest list of the warp is done;
    // *nchunk = the warp's largest chunk count of the window.  An entry whose leaf box
    // (moved by the entry's offset) lies beyond reach of the tile's box contributes no
    // sources: the staging would reject every one of them.  Reach: sqrt(reach2) for the
    // density (targets' h); for the force (FORCE) the larger of the targets' h and the
    // leaf's largest current h (set before the force pass).
    template <bool FORCE>
    __device__ __forceinline__ bool next(const float4 *__restrict__ list, const int2 *__restrict__ rng,
                                         const float4 *__restrict__ blo, const float4 *__restrict__ bhi, uint32_t e0,
                                         int ne, int ncell, int tl, int &nchunk, float lox, float hix, float loy,
                                         float hiy, float loz, float hiz, float reach2, float H, float L)
    {
        wb += TW;
        if (wb >= ncell) return false;
        int c = 0, b = 0;
        px = py = pz = 0.f;
        if (wb + tl < ne) {
            const float4 en = list[e0 + (uint32_t)(wb + tl)];
            const int lf = __float_as_int(en.w);
            const int2 r = rng[lf];
            b = r.x;
            c = r.y - r.x;
            px = en.x;
            py = en.y;
            pz = en.z;
            const float4 lo = blo[lf], hi = bhi[lf];
            const float gx = fmaxf(fmaxf(lo.x + px - hix, lox - (hi.x + px)), 0.f);
            const float gy = fmaxf(fmaxf(lo.y + py - hiy, loy - (hi.y + py)), 0.f);
            const float gz = fmaxf(fmaxf(lo.z + pz - hiz, loz - (hi.z + pz)), 0.f);
            float r2 = reach2;
            if (FORCE) {
                const float m = fmaxf(H, lo.w);
                r2 = m * m * (1.f + kPruneMargin) + 2.f * kBandK * m * (m + L);
            }
            if (fmaf(gx, gx, fmaf(gy, gy, gz * gz)) > r2 * 1.00001f) c = 0;
        }
        // the window's non-empty entries moved to the front (list order kept), so that
        // the lookup below meets no empty entry before the last non-empty one
        {
            const int g = TW == 32 ? 0 : (int)(threadIdx.x & 31) / TW;
            const unsigned gm = TW == 32 ? kFull : (((1u << TW) - 1u) << (TW * g));
            const unsigned mine = __ballot_sync(kFull, c > 0) & gm;
            const unsigned src = __fns(mine, (unsigned)(TW * g), tl + 1);
            const bool has = src < 32u;
            const int sl = has ? (int)src : (int)(threadIdx.x & 31);
            c = __shfl_sync(kFull, c, sl);
            b = __shfl_sync(kFull, b, sl);
            px = __shfl_sync(kFull, px, sl);
            py = __shfl_sync(kFull, py, sl);
            pz = __shfl_sync(kFull, pz, sl);
            if (!has) c = 0;
        }
        incl = c;
#pragma unroll
        for (int d = 1; d < TW; d <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, d, TW);
            if (tl >= d) incl += v;
        }
        st = incl - c;
        sb = b - st;
        tot = __shfl_sync(kFull, incl, TW - 1, TW);
        nchunk = (int)__reduce_max_sync(kFull, (unsigned)((tot + TW - 1) / TW));
        return true;
    }

    // slot j, validity and entry offset of the stream position base + tl of chunk
    // base (every lane calls it): the entry holding position base is the number of
    // entries that end at or before it; each entry that starts inside the chunk, at
    // or before the lane's position, adds one
    __device__ __forceinline__ void slot(int base, int tl, int &j, bool &v, float &sx, float &sy,
                                         float &sz) const
    {
        const int g = TW == 32 ? 0 : (int)(threadIdx.x & 31) / TW;  // tile of the lane within the warp
        const unsigned gm = TW == 32 ? kFull : (((1u << TW) - 1u) << (TW * g));
        const bool inside = st > base && st < base + TW && st < incl;
        const unsigned starts = __reduce_or_sync(kFull, inside ? 1u << (TW * g + st - base) : 0u) >> (TW * g);
        const int eb = __popc(__ballot_sync(kFull, incl <= base) & gm);
        const int e = min(eb + __popc(starts & ((2u << tl) - 2u)), TW - 1);
        const int q = base + tl;
        j = __shfl_sync(kFull, sb, e, TW) + q;
        sx = __shfl_sync(kFull, px, e, TW);
        sy = __shfl_sync(kFull, py, e, TW);
        sz = __shfl_sync(kFull, pz, e, TW);
        v = q < tot;
    }
};

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
    float *h_lo, *h_hi;  // bracket of the root of N_w(h) = N_ngb
    float *rho, *P, *c, *f, *divv, *curl;
    int32_t *n_ngb;
    float4 *thermo4;
    uint64_t *ngb_hash;
    unsigned long long *counters;
    const BoxDev *__restrict__ boxes;
    // adaptive cells: tile.x is a leaf, sources come from its neighbour list
    const uint32_t *__restrict__ list_off;
    const float4 *__restrict__ list;
    const int2 *__restrict__ leaf_rng;
    const float *__restrict__ leaf_scale;
    const float4 *__restrict__ leaf_lo, *__restrict__ leaf_hi;  // adaptive: leaf boxes (leaf frame)
    const float *__restrict__ leaf_hb;
    int hold_cells;  // list mode: the cells cannot be rebuilt during this iteration
    const int *__restrict__ tord;  // adaptive: targets of a leaf in ascending h (tiles index this)
    const float2 *__restrict__ axis;  // SPH_FLAG_AXIS_SWEEP orders (uniform grid), or null
    int64_t axis_stride;
    double box;
    float n_ngb_target, h_tol, gamma;
    int use_balsara;
    int last_pass;
};

// reductions over the TW lanes of a tile (xor offsets < TW stay inside the tile)
template <int TW>
__device__ __forceinline__ float tile_min(float v)
{
#pragma unroll
    for (int o = TW / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
template <int TW>
__device__ __forceinline__ float tile_max(float v)
{
#pragma unroll
    for (int o = TW / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum_ull(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int wrapc(int j, int nc) { return j < 0 ? j + nc : (j >= nc ? j - nc : j); }

// Pop the lowest set bit of a 128-bit mask held in four words; returns its index.
__device__ __forceinline__ int pop_bit(unsigned &m0, unsigned &m1, unsigned &m2, unsigned &m3)
{
    const bool a = m0 != 0, b = m1 != 0, c = m2 != 0;
    const unsigned m = a ? m0 : (b ? m1 : (c ? m2 : m3));
    const int base = a ? 0 : (b ? 32 : (c ? 64 : 96));
    const unsigned r = m & (m - 1u);
    if (a) m0 = r;
    else if (b) m1 = r;
    else if (c) m2 = r;
    else m3 = r;
    return base + __ffs(m) - 1;
}

// Clear the r lowest set bits of the 128-bit mask M (r below its population).
__device__ __forceinline__ unsigned keep_after(unsigned w, int r)
{
    return r == 0 ? w : w & ~((1u << __fns(w, 0u, r + 1)) - 1u);
}
__device__ __forceinline__ void drop_hits(uint4 &M, int r)
{
    int c = __popc(M.x);
    if (r < c) { M.x = keep_after(M.x, r); return; }
    r -= c;
    M.x = 0u;
    c = __popc(M.y);
    if (r < c) { M.y = keep_after(M.y, r); return; }
    r -= c;
    M.y = 0u;
    c = __popc(M.z);
    if (r < c) { M.z = keep_after(M.z, r); return; }
    r -= c;
    M.z = 0u;
    M.w = keep_after(M.w, r);
}

// Cubic spline of support 1 without its normalisation sigma, in truncated-power form:
// w/sigma = 2(1-q)^3_+ - 8(1/2-q)^3_+,  (dw/dq)/sigma = -6(1-q)^2_+ + 24(1/2-q)^2_+
// (identical to the piecewise polynomial; branch-free).
__device__ __forceinline__ void spline_u(float q, float &w, float &dw)
{
    const float a = fmaxf(1.f - q, 0.f), b = fmaxf(0.5f - q, 0.f);
    const float a2 = a * a, b2 = b * b;
    w = fmaf(-8.f * b2, b, 2.f * a2 * a);
    dw = fmaf(24.f, b2, -6.f * a2);
}
__device__ __forceinline__ float spline_dw_u(float q)
{
    const float a = fmaxf(1.f - q, 0.f), b = fmaxf(0.5f - q, 0.f);
    return fmaf(24.f * b, b, -6.f * a * a);
}

// Partial force sums of one target: a, du/dt and the largest v_sig.
struct ForceSum {
    float x = 0.f, y = 0.f, z = 0.f, u = 0.f, v = 0.f;
    // store into slot idx (sums into the float4, v_sig beside) and start again
    __device__ __forceinline__ void put(float4 *s4, float *sv, int idx)
    {
        s4[idx] = make_float4(x, y, z, u);
        sv[idx] = v;
        x = y = z = u = v = 0.f;
    }
};

// Partial density sums of one target: {sum m w, sum w, sum q w', sum m (3 w + q w')}
// and {sum (v_ij . d) m w'/r, the three components of the curl sum}.
struct DensSum {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
    // store into slot idx (two float4) and start again
    __device__ __forceinline__ void put(float4 *s, int idx)
    {
        s[2 * idx] = a;
        s[2 * idx + 1] = b;
        a = b = make_float4(0.f, 0.f, 0.f, 0.f);
    }
};

// The pair term of the force pass (Sec. 2: the grad-h pressure force with the
// Monaghan viscosity and its Balsara switch, and du/dt) of target i (1/h_i, 1/h_i^4,
// v_i, thermo_i = {rho, f P / rho^2, c, B}) and source j (h_j, {v_j, m_j}, thermo_j)
// at d = p_i - p_j, r2 = |d|^2 > 0; in_i, in_j: r < h_i, r < h_j.
__device__ __forceinline__ void force_term(float dx, float dy, float dz, float r2, bool in_i, bool in_j, float hinv,
                                           float hinv4, const float4 vi, const float4 ti, float hj, const float4 vj,
                                           const float4 tj, float alpha, ForceSum &f)
{
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float hjinv = __fdividef(1.f, hj);
    const float hj2inv = hjinv * hjinv;
    const float dWi = in_i ? kSigma * spline_dw_u(r * hinv) * hinv4 : 0.f;
    const float dWj = in_j ? kSigma * spline_dw_u(r * hjinv) * (hj2inv * hj2inv) : 0.f;
    const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
    const float mu = fmaf(vx, dx, fmaf(vy, dy, vz * dz)) * rinv;
    // viscosity only on approach (mu < 0): branch-free, Pi = 0 otherwise
    const float muc = fminf(mu, 0.f);
    const float vsig_ij = ti.z + tj.z - 3.f * muc;
    const float Pi = -alpha * vsig_ij * muc * (0.5f * (ti.w + tj.w)) * __fdividef(1.f, ti.x + tj.x);
    const float dWbar = 0.5f * (dWi + dWj);
    const float mj = vj.w;
    const float sc = mj * fmaf(ti.y, dWi, fmaf(tj.y, dWj, Pi * dWbar)) * rinv;
    f.x = fmaf(-sc, dx, f.x);
    f.y = fmaf(-sc, dy, f.y);
    f.z = fmaf(-sc, dz, f.z);
    f.u = fmaf(mj * mu, fmaf(ti.y, dWi, 0.5f * Pi * dWbar), f.u);
    f.v = fmaxf(f.v, vsig_ij);
}

// MODE: 0 = uniform grid, 1 = adaptive cells (leaf lists), 2 = uniform grid with the
// per-axis sweep (SPH_FLAG_AXIS_SWEEP)
template <int TW, bool HASH, int MODE>
__global__ void __launch_bounds__(kPairThreads, kDensityBlocks) k_density(DensityArgs a)
{
    constexpr bool LIST = MODE == 1, SWEEP = MODE == 2;
    constexpr int TPW = 32 / TW;
    constexpr int B = kBatchD;
    constexpr int SLOT = B + 1;  // one float4 of padding: the tiles of a warp hit different banks
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int sub = lane / TW, tl = lane % TW;
    float4 *sA = smem + (size_t)wib * (2 * TPW * SLOT) + sub * SLOT;  // {x, y, z, j} in target frame
    float4 *sB = sA + TPW * SLOT;                                      // {vx, vy, vz, m}
    // list mode, the balanced hit walk's scratch per tile (kWalkBytesD x TW): the
    // targets' hit masks, the partial sums (two float4) of each lane's first target (F),
    // last target (E) and of the targets inside its range (D), the tile's targets
    // ({x, y, z, 1/h}, {v, m}) and their first hit's position
    char *const wt = reinterpret_cast<char *>(smem + (size_t)(blockDim.x >> 5) * (2 * TPW * SLOT)) +
                     ((size_t)wib * TPW + sub) * TW * kWalkBytesD;
    uint4 *wM = reinterpret_cast<uint4 *>(wt);
    float4 *wF = reinterpret_cast<float4 *>(wt + TW * 16), *wE = wF + 2 * TW, *wD = wE + 2 * TW;
    float4 *wP = wD + 2 * TW, *wV = wP + TW;
    int *wOff = reinterpret_cast<int *>(wV + TW);
    const unsigned gmask = TW == 32 ? kFull : (((1u << TW) - 1u) << (sub * TW));
    const unsigned lt = (1u << lane) - 1u;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int ntiles = *a.n_tiles;
    const int ngroups = (ntiles + TPW - 1) / TPW;
    const float inf = __int_as_float(0x7f800000);

    // statistics and flags, kept per lane over all tile groups of this warp and added
    // to the global counters once at the end (one atomic per warp and counter)
    unsigned acc_pairs = 0u, acc_cand = 0u, acc_targets = 0u, acc_unc = 0u, acc_hf = 0u;
    unsigned acc_stream = 0u, acc_staged = 0u;  // sources read from the cells / lists, and staged
    // tile groups: the warp's first one by its index, the others handed out by a ticket
    // counter (taken one group ahead, so that its latency hides behind a tile), so
    // that warps that met costly tiles take fewer
    unsigned *ticket = reinterpret_cast<unsigned *>(a.counters + C_TICKET);  // its low word
    unsigned tk = 0u;
    if (lane == 0) tk = atomicAdd(ticket, 1u);
    for (int grp = gw, g_after = 0; grp < ngroups; grp = g_after) {
        g_after = nw + (int)__shfl_sync(kFull, tk, 0);
        if (lane == 0 && g_after < ngroups) tk = atomicAdd(ticket, 1u);
        const int t = grp * TPW + sub;
        const int4 tile = t < ntiles ? a.tiles[t] : make_int4(0, 0, 0, 0);
        const bool valid = tl < tile.z;
        const int i = LIST ? (valid ? a.tord[tile.y + tl] : 0) : tile.y + tl;
        const bool act = valid && a.active[i];
        const unsigned amask = __ballot_sync(kFull, act);
        if (!amask) continue;
        const bool live = (amask & gmask) != 0;  // uniform within the tile

        float4 pi = make_float4(0.f, 0.f, 0.f, 0.f), vi = pi;
        float hi = 0.f;
        if (act) {
            pi = a.pos4[i];
            vi = a.vel4[i];
            hi = a.h[i];
        }
        const float lox = tile_min<TW>(act ? pi.x : inf), hix = tile_max<TW>(act ? pi.x : -inf);
        const float loy = tile_min<TW>(act ? pi.y : inf), hiy = tile_max<TW>(act ? pi.y : -inf);
        const float loz = tile_min<TW>(act ? pi.z : inf), hiz = tile_max<TW>(act ? pi.z : -inf);
        const float hmax = tile_max<TW>(hi);
        const BoxDev bx = a.boxes[tile.w];
        const int nc = bx.nc;
        // coordinate scale of the FP32 arithmetic: the cell side, or the leaf's scale
        const float L = LIST ? a.leaf_scale[tile.x] : bx.L32;
        // stencil radius (cells) that holds the tile's cutoff; warp-uniform
        const int R = LIST ? 1 : (int)__reduce_max_sync(kFull, hmax * (1.f + kPruneMargin) > L ? 2u : 1u);
        // grown so that pairs the FP64 band re-decision may accept are never pruned
        const float reach2 = hmax * hmax * (1.f + kPruneMargin) + 2.f * kBandK * hmax * (hmax + L);
        // r^2 below lob: neighbour; above hib: not; in between: decided in FP64.
        // Lanes without an active target get thresholds no distance can pass.
        const float band = kBandK * hi * (hi + L);
        const float hi2 = act ? hi * hi : -1.f;
        const float lob = hi2 - band, hib = hi2 + band;
        const float hinv = act ? 1.f / hi : 0.f;
        if constexpr (LIST) {  // for the balanced walk (read after the flush's first __syncwarp)
            wP[tl] = make_float4(pi.x, pi.y, pi.z, hinv);
            wV[tl] = vi;
        }
        const int ca = tile.x - bx.cell_off;
        const int ix = ca % nc, iy = (ca / nc) % nc, iz = ca / (nc * nc);

        // sums without the kernel normalisation (applied at the end); the pair
        // (i, i) is met in the own cell and supplies the self term of Eq. 1
        float rho_s = 0.f, rho_c = 0.f;  // sum m_j w_j
        float sw_s = 0.f, sw_c = 0.f;    // sum w_j
        float sqdw = 0.f;                // sum q_j w'_j
        float drho = 0.f;                // sum m_j (3 w_j + q_j w'_j)
        float dv = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
        int cnt = 0;
        uint64_t hh = 0;
        unsigned cand = 0;
        int nst = 0;  // staged survivors of this tile (uniform within the tile)

        auto flush = [&]() {
            // pad this tile's batch up to the warp's longest one, rounded up to a
            // multiple of 4 (index 0 is a valid particle; the pads are far away)
            const int nmax = (int)((__reduce_max_sync(kFull, (unsigned)nst) + 3u) & ~3u);
            for (int k = nst + tl; k < nmax; k += TW) sA[k] = make_float4(-kFar, -kFar, -kFar, __int_as_float(0));
            __syncwarp();
            cand += (unsigned)nst;
            // phase 1: distance tests, broadcast reads of the staged sources
            unsigned m0 = 0u, m1 = 0u, m2 = 0u, m3 = 0u;
            const int nwords = (nmax + 31) >> 5;
#pragma unroll 1
            for (int wd = 0; wd < nwords; ++wd) {
                const int kend = min(32, nmax - 32 * wd);  // a multiple of 4
                const float4 *sw = sA + 32 * wd;
                unsigned mw = 0u, bw = 0u;  // hits; pairs in the FP32 band, decided below
                for (int k4 = 0; k4 < kend; k4 += 4) {
                    unsigned mn = 0u, bn = 0u;  // the four tests of this group
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 s = sw[k4 + u];
                        const float dx = pi.x - s.x, dy = pi.y - s.y, dz = pi.z - s.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        mn |= (unsigned)(r2 < lob) << u;
                        bn |= (unsigned)(r2 < hib) << u;  // (below the band's top; the hits are removed after)
                    }
                    mw |= mn << k4;
                    bw |= bn << k4;
                }
                // (rare) band pairs in FP64, out of the branch-free loop above: below the
                // band's top and not a hit
                bw &= ~mw;
                while (bw) {
                    const int kk = __ffs(bw) - 1;
                    bw &= bw - 1u;
                    if (band_decide(a.x, a.y, a.z, i, __float_as_int(sw[kk].w), a.box, hi, hi) & 1u) mw |= 1u << kk;
                }
                m0 = wd == 0 ? mw : m0;
                m1 = wd == 1 ? mw : m1;
                m2 = wd == 2 ? mw : m2;
                m3 = wd == 3 ? mw : m3;
            }
            // phase 2: each lane walks its own hits; the batch's terms are summed plainly
            // (at most kBatchD of them) and the batch sums are added with compensation
            float rb = 0.f, wb = 0.f;
            // one pair term, evaluated for staged source k
            auto term = [&](int k, float &w, float &dw, float &q, float &fr, float &mj, float3 &d, float3 &v) {
                const float4 sk = sA[k];
                const float4 vj = sB[k];
                d = make_float3(pi.x - sk.x, pi.y - sk.y, pi.z - sk.z);
                const float r2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
                const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                q = r2 * rinv * hinv;
                spline_u(q, w, dw);
                mj = vj.w;
                fr = mj * dw * rinv;
                v = make_float3(vi.x - vj.x, vi.y - vj.y, vi.z - vj.z);
            };
            auto accumulate = [&](float w, float dw, float q, float fr, float mj, float3 d, float3 v) {
                rb = fmaf(mj, w, rb);
                wb += w;
                sqdw = fmaf(q, dw, sqdw);
                drho = fmaf(mj, fmaf(q, dw, 3.f * w), drho);
                dv = fmaf(fr, fmaf(v.x, d.x, fmaf(v.y, d.y, v.z * d.z)), dv);
                cx = fmaf(fr, fmaf(v.y, d.z, -v.z * d.y), cx);
                cy = fmaf(fr, fmaf(v.z, d.x, -v.x * d.z), cy);
                cz = fmaf(fr, fmaf(v.x, d.y, -v.y * d.x), cz);
            };
            if constexpr (LIST) {
                // Balanced walk, as in the force pass (k_force): the tile's H hits, in lane
                // order, cut into TW contiguous ranges, one per lane; each lane sums its
                // targets' terms in order, and a target whose hits cross ranges adds the
                // pieces in lane order (the same order on every run).
                const int nh = __popc(m0) + __popc(m1) + __popc(m2) + __popc(m3);
                int hincl = nh;
#pragma unroll
                for (int dd = 1; dd < TW; dd <<= 1) {
                    const int v = __shfl_up_sync(kFull, hincl, dd, TW);
                    if (tl >= dd) hincl += v;
                }
                const int H = __shfl_sync(kFull, hincl, TW - 1, TW);
                const int hoff = hincl - nh;
                cnt += nh;
                if (HASH) {  // integer sums: any order gives the same bits
                    unsigned h0 = m0, h1 = m1, h2 = m2, h3 = m3;
                    while (h0 | h1 | h2 | h3) hh += mix64((uint64_t)a.ids[__float_as_int(sA[pop_bit(h0, h1, h2, h3)].w)]);
                }
                wM[tl] = make_uint4(m0, m1, m2, m3);
                wOff[tl] = hoff;
                __syncwarp();
                const int rb_ = (tl * H) / TW, re_ = ((tl + 1) * H) / TW;
                if (rb_ < re_) {
                    int o = 0;
#pragma unroll
                    for (int st = TW / 2; st > 0; st >>= 1)
                        if (wOff[o + st] <= rb_) o += st;
                    uint4 M = wM[o];
                    drop_hits(M, rb_ - wOff[o]);  // those belong to the ranges before
                    float4 po = wP[o];            // {x, y, z, 1/h}
                    float4 vo = wV[o];
                    DensSum part;
                    bool first = true;
                    for (int p = rb_; p < re_; ++p) {
                        if ((M.x | M.y | M.z | M.w) == 0u) {  // the owner's hits end here
                            if (first) part.put(wF, tl);
                            else part.put(wD, o);  // a target inside this range: only this lane
                            first = false;
                            do {
                                ++o;
                                M = wM[o];
                            } while ((M.x | M.y | M.z | M.w) == 0u);
                            po = wP[o];
                            vo = wV[o];
                        }
                        const int k = pop_bit(M.x, M.y, M.z, M.w);
                        const float4 sk = sA[k];
                        const float4 vj = sB[k];
                        const float dx = po.x - sk.x, dy = po.y - sk.y, dz = po.z - sk.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                        const float q = r2 * rinv * po.w;
                        float w, dw;
                        spline_u(q, w, dw);
                        const float mj = vj.w;
                        const float fr = mj * dw * rinv;
                        const float vx = vo.x - vj.x, vy = vo.y - vj.y, vz = vo.z - vj.z;
                        part.a.x = fmaf(mj, w, part.a.x);
                        part.a.y += w;
                        part.a.z = fmaf(q, dw, part.a.z);
                        part.a.w = fmaf(mj, fmaf(q, dw, 3.f * w), part.a.w);
                        part.b.x = fmaf(fr, fmaf(vx, dx, fmaf(vy, dy, vz * dz)), part.b.x);
                        part.b.y = fmaf(fr, fmaf(vy, dz, -vz * dy), part.b.y);
                        part.b.z = fmaf(fr, fmaf(vz, dx, -vx * dz), part.b.z);
                        part.b.w = fmaf(fr, fmaf(vx, dy, -vy * dx), part.b.w);
                    }
                    if (first) {
                        part.put(wF, tl);
                        wE[2 * tl] = wE[2 * tl + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
                    } else {
                        part.put(wE, tl);
                    }
                } else {
                    wF[2 * tl] = wF[2 * tl + 1] = wE[2 * tl] = wE[2 * tl + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                __syncwarp();
                if (nh > 0) {
                    // the ranges La..Lb hold this target's hits hoff..hoff + nh - 1
                    const int p0 = hoff, p1 = hoff + nh - 1;
                    const int La = min(TW - 1, ((p0 + 1) * TW - 1) / H);
                    const int Lb = min(TW - 1, ((p1 + 1) * TW - 1) / H);
                    const int bA = (La * H) / TW, eA = ((La + 1) * H) / TW;
                    const float4 *src = (La == Lb && p0 != bA && p1 + 1 != eA) ? wD + 2 * tl
                                        : (p0 == bA ? wF + 2 * La : wE + 2 * La);
                    float4 ta = src[0], tb = src[1];
                    for (int Lx = La + 1; Lx <= Lb; ++Lx) {  // ranges that start inside its hits
                        const float4 fa = wF[2 * Lx], fb = wF[2 * Lx + 1];
                        ta.x += fa.x;
                        ta.y += fa.y;
                        ta.z += fa.z;
                        ta.w += fa.w;
                        tb.x += fb.x;
                        tb.y += fb.y;
                        tb.z += fb.z;
                        tb.w += fb.w;
                    }
                    rb += ta.x;
                    wb += ta.y;
                    sqdw += ta.z;
                    drho += ta.w;
                    dv += tb.x;
                    cx += tb.y;
                    cy += tb.z;
                    cz += tb.w;
                }
                __syncwarp();  // the scratch is rewritten by the next batch
                m0 = m1 = m2 = m3 = 0u;
            } else {
                // Lane-by-lane rounds, two hits per round (independent instruction streams;
                // a lane's terms are still added in ascending staged order, so its sums are
                // those of one at a time).
                for (;;) {
                    const unsigned busy = __ballot_sync(kFull, (m0 | m1 | m2 | m3) != 0u);
                    if (busy == 0u) break;
                    if (m0 | m1 | m2 | m3) {
                        const int k1 = pop_bit(m0, m1, m2, m3);
                        const bool two = (m0 | m1 | m2 | m3) != 0u;
                        int k2 = k1;
                        if (two) k2 = pop_bit(m0, m1, m2, m3);
                        float w1, dw1, q1, fr1, mj1, w2, dw2, q2, fr2, mj2;
                        float3 d1, v1, d2, v2;
                        term(k1, w1, dw1, q1, fr1, mj1, d1, v1);
                        term(k2, w2, dw2, q2, fr2, mj2, d2, v2);
                        accumulate(w1, dw1, q1, fr1, mj1, d1, v1);
                        if (two) accumulate(w2, dw2, q2, fr2, mj2, d2, v2);
                        cnt += two ? 2 : 1;
                        if (HASH) {
                            hh += mix64((uint64_t)a.ids[__float_as_int(sA[k1].w)]);
                            if (two) hh += mix64((uint64_t)a.ids[__float_as_int(sA[k2].w)]);
                        }
                    }
                }
            }
            kahan_add(rho_s, rho_c, rb);
            kahan_add(sw_s, sw_c, wb);
            nst = 0;
            __syncwarp();
        };

        // the 27 cell ranges of the tile, fetched at once: lane tl holds cells tl, tl + TW
        // (radius-2 stencils, for h beyond the planned cell, load ranges one by one)
        int cs0 = 0, ce0 = 0, cs1 = 0, ce1 = 0;
        if (!LIST && live && R == 1) {
            if (tl < 27) {
                const int cb = bx.cell_off +
                               (wrapc(iz + kOrder[tl][2], nc) * nc + wrapc(iy + kOrder[tl][1], nc)) * nc +
                               wrapc(ix + kOrder[tl][0], nc);
                cs0 = a.cell_start[cb];
                ce0 = a.cell_start[cb + 1];
            }
            if (tl + TW < 27) {
                const int o2 = tl + TW;
                const int cb = bx.cell_off +
                               (wrapc(iz + kOrder[o2][2], nc) * nc + wrapc(iy + kOrder[o2][1], nc)) * nc +
                               wrapc(ix + kOrder[o2][0], nc);
                cs1 = a.cell_start[cb];
                ce1 = a.cell_start[cb + 1];
            }
        }
        // stage chunk after chunk; one flush site (keeps the kernel small)
        // (adaptive cells: the tile's list entries, each a leaf and its offset)
        uint32_t e0 = 0;
        int ne = 0;
        if (LIST && live) {
            e0 = a.list_off[tile.x];
            ne = (int)(a.list_off[tile.x + 1] - e0);
        }
        int o = -1, ch = -1, nchunk = 0, bs = 0, be = 0;
        const int ncell = LIST ? (int)__reduce_max_sync(kFull, (unsigned)ne) : (R == 1 ? 27 : 125);
        float shx = 0.f, shy = 0.f, shz = 0.f;  // offset of the chunk's sources (list mode: per lane)
        // axis sweep of the cell at the cursor (SPH_FLAG_AXIS_SWEEP, radius-1 stencils)
        int sw_d = -1;
        float sw_sg = 0.f, sw_lim = 0.f;
        const float rlim = SWEEP ? sqrtf(reach2) : 0.f;
        // cursor over (cell or list entry o, chunk ch): moves to the next chunk, false at
        // the end (warp-uniform)
        ListStream<TW> ls;
        auto next_chunk = [&]() -> bool {
            ++ch;
            if (LIST) {
                while (ch >= nchunk) {
                    if (!ls.template next<false>(a.list, a.leaf_rng, a.leaf_lo, a.leaf_hi, e0, ne, ncell, tl, nchunk,
                                                 lox, hix, loy, hiy, loz, hiz, reach2, 0.f, L))
                        return false;
                    ch = 0;
                }
            } else {
                while (ch >= nchunk) {
                    if (o >= ncell - 1) return false;
                    ++o;
                    ch = 0;
                    {
                        int ox, oy, oz;
                        if (R == 1) {
                            const int src = o < TW ? o : o - TW;
                            bs = __shfl_sync(kFull, o < TW ? cs0 : cs1, src, TW);
                            be = __shfl_sync(kFull, o < TW ? ce0 : ce1, src, TW);
                            ox = kOrder[o][0];
                            oy = kOrder[o][1];
                            oz = kOrder[o][2];
                        } else {
                            ox = o < 27 ? kOrder[o][0] : kOuter[o - 27][0];
                            oy = o < 27 ? kOrder[o][1] : kOuter[o - 27][1];
                            oz = o < 27 ? kOrder[o][2] : kOuter[o - 27][2];
                            bs = be = 0;
                            if (live) {
                                const int cb = bx.cell_off + (wrapc(iz + oz, nc) * nc + wrapc(iy + oy, nc)) * nc +
                                               wrapc(ix + ox, nc);
                                bs = a.cell_start[cb];
                                be = a.cell_start[cb + 1];
                            }
                        }
                        shx = (float)ox * L;
                        shy = (float)oy * L;
                        shz = (float)oz * L;
                        sw_d = -1;
                        if (SWEEP && R == 1 && o > 0) {
                            sw_d = kOrderAxis[o][0];
                            sw_sg = (float)kOrderAxis[o][1];
                            sw_lim = sweep_limit(o, L, rlim, lox, hix, loy, hiy, loz, hiz);
                        }
                    }
                    nchunk = (int)__reduce_max_sync(kFull, (unsigned)((be - bs + TW - 1) / TW));
                }
            }
            return true;
        };
        // slot of this lane's source in the chunk at the cursor: slot order, or the
        // cell's order along the axis (backwards for the negative direction), dropping
        // sources at or beyond the sweep bound
        auto slot_at = [&](int &j, bool &v) {
            const int q = ch * TW + tl;
            v = q < be - bs;
            j = bs + q;
            if (SWEEP && sw_d >= 0 && v) {
                const float2 e = a.axis[(size_t)sw_d * a.axis_stride + bs + (sw_sg > 0.f ? q : be - bs - 1 - q)];
                j = __float_as_int(e.y);
                v = sw_sg * e.x < sw_lim;
            }
        };
        // software pipeline: the positions of the next chunk are loaded before the
        // current chunk is tested, so their latency overlaps the test, the staging
        // and a flush
        bool have = next_chunk();
        int jc = bs + ch * TW + tl;
        bool vc = have && jc < be;
        if (LIST && have) ls.slot(ch * TW, tl, jc, vc, shx, shy, shz);
        if (SWEEP && have) slot_at(jc, vc);
        float4 pc = vc ? __ldg(a.pos4 + jc) : make_float4(0.f, 0.f, 0.f, 0.f);
        float scx = shx, scy = shy, scz = shz;
        while (have) {
            if constexpr (LIST) acc_stream += vc ? 1u : 0u;
            const bool have_n = next_chunk();
            int jn = bs + ch * TW + tl;
            bool vn = have_n && jn < be;
            if (LIST && have_n) ls.slot(ch * TW, tl, jn, vn, shx, shy, shz);
            if (SWEEP && have_n) slot_at(jn, vn);
            const float4 pn = vn ? __ldg(a.pos4 + jn) : make_float4(0.f, 0.f, 0.f, 0.f);
            bool keep = false;
            if (vc) {
                pc.x += scx;
                pc.y += scy;
                pc.z += scz;
                const float ex = fmaxf(fmaxf(lox - pc.x, pc.x - hix), 0.f);
                const float ey = fmaxf(fmaxf(loy - pc.y, pc.y - hiy), 0.f);
                const float ez = fmaxf(fmaxf(loz - pc.z, pc.z - hiz), 0.f);
                keep = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < reach2;
            }
            const unsigned mine = __ballot_sync(kFull, keep) & gmask;
            if (keep) {
                const int pos = nst + __popc(mine & lt);
                sA[pos] = make_float4(pc.x, pc.y, pc.z, __int_as_float(jc));
                sB[pos] = __ldg(a.vel4 + jc);  // (only for the kept sources: 1.6 % faster on boxes)
            }
            nst += __popc(mine);
            const int mx = (int)__reduce_max_sync(kFull, (unsigned)nst);
            if (mx > B - TW || (!have_n && mx > 0)) flush();
            have = have_n;
            jc = jn;
            vc = vn;
            pc = pn;
            scx = shx;
            scy = shy;
            scz = shz;
        }

        const int nself = act ? 1 : 0;  // the (i, i) pair is not a neighbour
        acc_pairs += (unsigned)(cnt - nself);
        if (tl == 0) acc_cand += cand * (unsigned)__popc(amask & gmask);
        if (tl == 0) acc_staged += cand;
        if (lane == 0) acc_targets += (unsigned)__popc(amask);

        // bit 0: not converged; bit 1: h beyond what the cells hold (rebuild needed)
        unsigned flag = 0u;
        if (act) {
            const float hinv3 = hinv * hinv * hinv, hinv4 = hinv3 * hinv;
            const float rho = kSigma * hinv3 * (rho_s - rho_c);
            const float nw_ = kSigma * kFourPi3 * (sw_s - sw_c);
            const float dnw_dh = -kSigma * kFourPi3 * sqdw * hinv;
            const float drho_dh = -kSigma * hinv4 * drho;
            const float divv = -kSigma * hinv4 * dv / rho;
            const float curl = kSigma * hinv4 * sqrtf(cx * cx + cy * cy + cz * cz) / rho;
            const float g = nw_ - a.n_ngb_target;
            bool conv = fabsf(g) <= a.h_tol * a.n_ngb_target;
            float lo = 0.f, up = kHUnbounded;
            if (!conv) {
                // N_w is non-decreasing in h, so every evaluation narrows a bracket of
                // the root; once the bracket is a few FP32 ulps wide the FP32 sums
                // cannot place the root more finely and h is accepted
                lo = a.h_lo[i];
                up = a.h_hi[i];
                if (g < 0.f) lo = fmaxf(lo, hi);
                else up = fminf(up, hi);
                conv = lo > 0.f && up < kHUnbounded && up - lo <= kHResolution * lo;
            }
            if (!conv && !a.last_pass) {
                // Newton step, at most a factor 2 either way; a step that leaves a
                // two-sided bracket is replaced by its geometric middle
                float hn = dnw_dh > 0.f ? hi - g / dnw_dh : (g < 0.f ? 2.f * hi : 0.5f * hi);
                hn = fminf(fmaxf(hn, 0.5f * hi), 2.f * hi);
                if (lo > 0.f && up < kHUnbounded && !(hn > lo && hn < up)) hn = sqrtf(lo) * sqrtf(up);
                flag = 1u;
                if (LIST) {
                    // adaptive cells: h up to just below half the box (the minimum
                    // image); beyond what its leaf's list or the adjacent top cells hold
                    // the cells are built again -- or, where they cannot be (captured
                    // steps), the step is cut back to that limit and new cells are
                    // reported only once the iterate sits there with N_w still short
                    const float hb = a.leaf_hb[tile.x];
                    const float lim = fminf(fminf(kTreeReach * hb, bx.L32), (float)(0.5 * a.box));
                    hn = fminf(hn, (float)(0.5 * a.box) * (1.f - 1e-5f));
                    if (a.hold_cells) {
                        const float cap = lim * (1.f - 2e-6f);
                        if (hn > cap) {
                            if (g < 0.f && hi >= cap * (1.f - 1e-6f)) flag |= 2u;
                            hn = cap;
                        }
                    } else if (hn > lim * (1.f - 1e-6f)) {
                        flag |= 2u;
                    }
                } else if ((double)hn > 2.0 * bx.L64 * (1.0 - 1e-6)) {
                    flag |= 2u;  // beyond the radius-2 stencil of its cell
                }
                a.h[i] = hn;
                a.h_lo[i] = lo;
                a.h_hi[i] = up;
            } else {
                if (!conv) flag = 1u;
                // uniform grid: FP32 cell-relative positions resolve h only down to
                // cell side / SPH_FRAME_RATIO at the density tolerance
                if (!LIST && bx.L32 > (float)SPH_FRAME_RATIO * hi) flag |= 4u;
                a.active[i] = 0;
                // quantities needed before the pressure gradient (EOS, grad-h, Balsara)
                const float u = a.upred[i];
                const float gam = a.gamma;
                const float P = (gam - 1.f) * rho * u;
                const float cs = sqrtf(gam * (gam - 1.f) * u);
                const float fgh = 1.f / (1.f + hi / (3.f * rho) * drho_dh);
                float Bq = 1.f;
                if (a.use_balsara) {
                    const float ad = fabsf(divv);
                    const float den = ad + curl + 1e-4f * cs * hinv;
                    Bq = den > 0.f ? ad / den : 0.f;
                }
                a.thermo4[i] = make_float4(rho, fgh * P / (rho * rho), cs, Bq);
                a.rho[i] = rho;
                a.P[i] = P;
                a.c[i] = cs;
                a.f[i] = fgh;
                a.divv[i] = divv;
                a.curl[i] = curl;
                a.n_ngb[i] = cnt - 1;
                if (HASH) a.ngb_hash[i] = hh - mix64((uint64_t)a.ids[i]);
            }
        }
        acc_unc += flag & 1u;
        acc_hf |= flag & 6u;
    }
    const unsigned long long tp = warp_sum_ull(acc_pairs), tc = warp_sum_ull(acc_cand);  // 64-bit sums
    const unsigned tu = __reduce_add_sync(kFull, acc_unc), th = __reduce_or_sync(kFull, acc_hf);
    const unsigned long long ts = warp_sum_ull(acc_stream), tg = warp_sum_ull(acc_staged);
    if (lane == 0) {
        if (ts) atomicAdd(a.counters + C_DSTREAM, ts);
        if (tg) atomicAdd(a.counters + C_DSTAGED, tg);
        if (tp) atomicAdd(a.counters + C_DPAIRS, tp);
        if (tc) atomicAdd(a.counters + C_DCAND, tc);
        if (acc_targets) atomicAdd(a.counters + C_DTARGETS, (unsigned long long)acc_targets);
        if (tu) atomicAdd(a.counters + C_UNCONV, (unsigned long long)tu);
        if (th & 2u) atomicOr(a.counters + C_HFLAG, 1ull);
        if (th & 4u) atomicOr(a.counters + C_PREC, 1ull);
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
    const float *__restrict__ cell_reach;  // per cell: max h of anything that can reach it
    float *ax, *ay, *az, *dudt, *vsig;
    const uint8_t *__restrict__ fmask;  // individual time-steps: targets to update (null: all)
    const unsigned long long *__restrict__ run_if;  // non-null: run only if *run_if != 0
    unsigned long long *counters;
    const BoxDev *__restrict__ boxes;
    const uint32_t *__restrict__ list_off;
    const float4 *__restrict__ list;
    const int2 *__restrict__ leaf_rng;
    const float *__restrict__ leaf_scale;
    const float4 *__restrict__ leaf_lo, *__restrict__ leaf_hi;  // adaptive: leaf boxes (leaf frame)
    const int *__restrict__ tord;
    const float2 *__restrict__ axis;
    int64_t axis_stride;
    double box;
    float alpha;
};

template <int TW, int MODE>
__global__ void __launch_bounds__(kPairThreads, MODE == 1 ? kForceBlocks : kForceBlocksU) k_force(ForceArgs a)
{
    if (a.run_if && *a.run_if == 0ull) return;  // the symmetric pass ran instead
    constexpr bool LIST = MODE == 1, SWEEP = MODE == 2;
    constexpr int TPW = 32 / TW;
    constexpr int B = kBatchF;
    constexpr int SLOT = B + 1;
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int sub = lane / TW, tl = lane % TW;
    float4 *sA = smem + (size_t)wib * (3 * TPW * SLOT) + sub * SLOT;  // {x, y, z, h_j} in target frame
    float4 *sB = sA + TPW * SLOT;                                      // {vx, vy, vz, m}
    float4 *sC = sB + TPW * SLOT;                                      // {rho, A, c, B}
    int *sI = (int *)(smem + (size_t)(blockDim.x >> 5) * (3 * TPW * SLOT)) + (size_t)wib * TPW * SLOT +
              sub * SLOT;
    // list mode, for the distance tests, as arrays (pairs of sources per instruction):
    // the staged x, y, z, and each source's cutoff thresholds h_j^2 -/+ its FP32 band
    // (h spans decades within a list, so each pair has its own band)
    const size_t nwb = blockDim.x >> 5;
    float *sX = (float *)((int *)(smem + nwb * (3 * TPW * SLOT)) + nwb * TPW * SLOT) +
                ((size_t)wib * TPW + sub) * 5 * kSlotF;  // (list mode only: not allocated otherwise)
    float *sY = sX + kSlotF, *sZ = sY + kSlotF, *sLo = sZ + kSlotF, *sHi = sLo + kSlotF;
    // list mode, the balanced hit walk's scratch per tile (kWalkBytes x TW): the targets'
    // hit masks, their first hit's position, the partial sums of each lane's first
    // target (F), last target (E) and of the targets inside its range (D), and the
    // tile's targets ({x, y, z, h}, {v, m}, thermo, {1/h, 1/h^4, h^2, band}, index)
    char *const wt = reinterpret_cast<char *>(smem) + (size_t)nwb * (3 * TPW * SLOT) * sizeof(float4) +
                     (size_t)nwb * TPW * SLOT * sizeof(int) + (size_t)nwb * TPW * 5 * kSlotF * sizeof(float) +
                     ((size_t)wib * TPW + sub) * TW * kWalkBytes;
    uint4 *wM = reinterpret_cast<uint4 *>(wt);
    float4 *wF = reinterpret_cast<float4 *>(wt + TW * 16), *wE = wF + TW, *wD = wE + TW;
    int *wOff = reinterpret_cast<int *>(wt + TW * 64);
    float *wFv = reinterpret_cast<float *>(wOff + TW), *wEv = wFv + TW, *wDv = wEv + TW;
    float4 *wP = reinterpret_cast<float4 *>(wt + TW * 80), *wV = wP + TW, *wT = wV + TW;
    float4 *wQ = wT + TW;  // {1/h, 1/h^4, h^2, FP32 band of h}
    int *wI = reinterpret_cast<int *>(wQ + TW);
    const unsigned gmask = TW == 32 ? kFull : (((1u << TW) - 1u) << (sub * TW));
    const unsigned lt = (1u << lane) - 1u;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int ntiles = *a.n_tiles;
    const int ngroups = (ntiles + TPW - 1) / TPW;
    const float inf = __int_as_float(0x7f800000);

    unsigned acc_pairs = 0u, acc_cand = 0u;  // per lane; added to the counters at the end
    unsigned acc_stream = 0u, acc_staged = 0u;  // sources read from the cells / lists, and staged
    // tile groups: the warp's first one by its index, the others handed out by a ticket
    // counter (taken one group ahead, so that its latency hides behind a tile), so
    // that warps that met costly tiles take fewer
    unsigned *ticket = reinterpret_cast<unsigned *>(a.counters + C_TICKET);  // its low word
    unsigned tk = 0u;
    if (lane == 0) tk = atomicAdd(ticket, 1u);
    for (int grp = gw, g_after = 0; grp < ngroups; grp = g_after) {
        g_after = nw + (int)__shfl_sync(kFull, tk, 0);
        if (lane == 0 && g_after < ngroups) tk = atomicAdd(ticket, 1u);
        const int t = grp * TPW + sub;
        const int4 tile = t < ntiles ? a.tiles[t] : make_int4(0, 0, 0, 0);
        const bool inr = tl < tile.z;
        const int i = LIST ? (inr ? a.tord[tile.y + tl] : 0) : tile.y + tl;
        const bool act = inr && (a.fmask == nullptr || a.fmask[i]);
        const unsigned amask = __ballot_sync(kFull, act);
        const bool live = (amask & gmask) != 0;
        // lanes without a target sit far away so that no distance test passes
        float4 pi = make_float4(kFar, kFar, kFar, 0.f), vi = make_float4(0.f, 0.f, 0.f, 0.f),
               ti = make_float4(1.f, 0.f, 0.f, 0.f);
        if (act) {
            pi = a.pos4[i];
            vi = a.vel4[i];
            ti = a.thermo4[i];
        }
        if constexpr (LIST) {  // for the balanced walk (read after the flush's first __syncwarp)
            wP[tl] = pi;
            wV[tl] = vi;
            wT[tl] = ti;
            wI[tl] = i;
        }
        const float lox = tile_min<TW>(act ? pi.x : inf), hix = tile_max<TW>(act ? pi.x : -inf);
        const float loy = tile_min<TW>(act ? pi.y : inf), hiy = tile_max<TW>(act ? pi.y : -inf);
        const float loz = tile_min<TW>(act ? pi.z : inf), hiz = tile_max<TW>(act ? pi.z : -inf);
        const float hi = pi.w;
        const BoxDev bx = a.boxes[tile.w];
        const int nc = bx.nc;
        const float L = LIST ? a.leaf_scale[tile.x] : bx.L32;
        // cutoff reach of the tile: r < max(h_i, h_j) with h_j of any particle that can
        // reach its cell (a tile beyond the last has tile.x = 0, a valid cell)
        // (adaptive cells: the leaf's list holds every source in reach, and each source
        // is pruned with its own h below)
        const float H = LIST ? tile_max<TW>(hi) : fmaxf(tile_max<TW>(hi), a.cell_reach[tile.x]);
        const int R = LIST ? 1 : (int)__reduce_max_sync(kFull, H * (1.f + kPruneMargin) > L ? 2u : 1u);
        const float bandmax = 2.f * kBandK * H * (H + L);
        const float reach2 = H * H * (1.f + kPruneMargin) + bandmax;
        const float hi2 = hi * hi;
        const float hinv = act ? 1.f / hi : 0.f;
        const float hinv4 = hinv * hinv * hinv * hinv;
        const float band_i = kBandK * hi * (hi + L);
        // list mode: r^2 below max(tlo_i, tlo_j): neighbour; at or above max(thi_i, thi_j):
        // not; in between decided in FP64 (h^2 -/+ the band, of the pair's larger h: the
        // band grows with h, so the pair's thresholds are the larger of the two particles')
        const float tlo_i = act ? hi2 - band_i : -1.f, thi_i = act ? hi2 + band_i : -1.f;
        if constexpr (LIST) wQ[tl] = make_float4(hinv, hinv4, hi2, band_i);
        const int ca = tile.x - bx.cell_off;
        const int ix = ca % nc, iy = (ca / nc) % nc, iz = ca / (nc * nc);
        float sx_ = 0.f, sxc = 0.f, sy_ = 0.f, syc = 0.f, sz_ = 0.f, szc = 0.f, su = 0.f, suc = 0.f;
        float vs = 0.f;
        int cnt = 0;
        unsigned cand = 0;
        int nst = 0;

        // exact neighbour decision for the pair (i, j): r < h_i and r < h_j
        auto decide = [&](float r2, float hj, const int *jp, bool &in_i, bool &in_j) {
            const float hj2 = hj * hj;
            in_i = r2 < hi2;
            in_j = r2 < hj2;
            const float band_j = kBandK * hj * (hj + L);
            if (fabsf(r2 - hi2) <= band_i || fabsf(r2 - hj2) <= band_j) {
                const unsigned d = band_decide(a.x, a.y, a.z, i, *jp, a.box, hi, hj);
                in_i = d & 1u;
                in_j = d & 2u;
            }
        };

        auto flush = [&]() {
            // pad this tile's batch up to the warp's longest one, rounded up to a
            // multiple of 4 (index 0 is a valid particle; the pads are far away)
            const int nmax = (int)((__reduce_max_sync(kFull, (unsigned)nst) + 3u) & ~3u);
            for (int k = nst + tl; k < nmax; k += TW) {
                sA[k] = make_float4(-kFar, -kFar, -kFar, 0.f);
                sI[k] = 0;
                if constexpr (LIST) {
                    sX[k] = -kFar;
                    sY[k] = -kFar;
                    sZ[k] = -kFar;
                    sLo[k] = -1.f;
                    sHi[k] = -1.f;
                }
            }
            __syncwarp();
            cand += (unsigned)nst;
            unsigned m0 = 0u, m1 = 0u, m2 = 0u, m3 = 0u;
            const float2 px2 = make_float2(pi.x, pi.x), py2 = make_float2(pi.y, pi.y), pz2 = make_float2(pi.z, pi.z);
            const float2 mone = make_float2(-1.f, -1.f);
            const int nwords = (nmax + 31) >> 5;
#pragma unroll 1
            for (int wd = 0; wd < nwords; ++wd) {
                const int kend = min(32, nmax - 32 * wd);  // a multiple of 4
                const float4 *sw = sA + 32 * wd;
                unsigned mw = 0u, bw = 0u;  // hits; pairs in the FP32 band, decided below
#pragma unroll(LIST ? 2 : 1)  // list mode: two groups in flight (1.3 % faster; the uniform grid keeps one)
                for (int k4 = 0; k4 < kend; k4 += 4) {
                    unsigned mn = 0u, bn = 0u;  // the four tests of this group
                    if constexpr (!LIST) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float4 s = sw[k4 + u];
                            const float dx = pi.x - s.x, dy = pi.y - s.y, dz = pi.z - s.z;
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            const float d2 = r2 - fmaxf(hi2, s.w * s.w);
                            mn |= (unsigned)(d2 < -bandmax) << u;
                            bn |= (unsigned)(d2 < bandmax) << u;
                        }
                    } else {
#pragma unroll
                    for (int u = 0; u < 4; u += 2) {
                        const int k = 32 * wd + k4 + u;  // two sources per instruction (FP32x2)
                        const float2 x2 = *reinterpret_cast<const float2 *>(sX + k);
                        const float2 y2 = *reinterpret_cast<const float2 *>(sY + k);
                        const float2 z2 = *reinterpret_cast<const float2 *>(sZ + k);
                        const float2 lo2 = *reinterpret_cast<const float2 *>(sLo + k);
                        const float2 hi2v = *reinterpret_cast<const float2 *>(sHi + k);
                        const float2 dx2 = __ffma2_rn(x2, mone, px2), dy2 = __ffma2_rn(y2, mone, py2);
                        const float2 dz2 = __ffma2_rn(z2, mone, pz2);
                        const float2 r2 = __ffma2_rn(dx2, dx2, __ffma2_rn(dy2, dy2, __fmul2_rn(dz2, dz2)));
                        const float l0 = fmaxf(tlo_i, lo2.x), l1 = fmaxf(tlo_i, lo2.y);
                        const float h0 = fmaxf(thi_i, hi2v.x), h1 = fmaxf(thi_i, hi2v.y);
                        mn |= ((unsigned)(r2.x < l0) << u) | ((unsigned)(r2.y < l1) << (u + 1));
                        bn |= ((unsigned)(r2.x < h0) << u) | ((unsigned)(r2.y < h1) << (u + 1));
                    }
                    }
                    mw |= mn << k4;
                    bw |= bn << k4;
                }
                // (rare) band pairs in FP64, out of the branch-free loop above: below the
                // band's top and not a hit
                bw &= ~mw;
                while (bw) {
                    const int kk = __ffs(bw) - 1;
                    bw &= bw - 1u;
                    if (band_decide(a.x, a.y, a.z, i, sI[32 * wd + kk], a.box, hi, sw[kk].w) != 0u) mw |= 1u << kk;
                }
                m0 = wd == 0 ? mw : m0;
                m1 = wd == 1 ? mw : m1;
                m2 = wd == 2 ? mw : m2;
                m3 = wd == 3 ? mw : m3;
            }
            // batch sums plain, compensated across batches
            float bx = 0.f, by = 0.f, bz = 0.f, bu = 0.f;
            if constexpr (LIST) {
                // Balanced walk (adaptive cells, where a tile's targets span a range of h
                // and their hit counts differ widely): the tile's H hits, laid out in
                // lane order (each target's in ascending staged index), are cut into TW
                // contiguous ranges, one per lane; a lane walks its range, moving to the
                // next target where one's hits end, and sums each target's terms in
                // order.  A target whose hits lie inside one range takes its sum from that
                // lane; one whose hits cross ranges adds the pieces in lane order -- the
                // same order on every run.
                const int nh = __popc(m0) + __popc(m1) + __popc(m2) + __popc(m3);
                int hincl = nh;
#pragma unroll
                for (int dd = 1; dd < TW; dd <<= 1) {
                    const int v = __shfl_up_sync(kFull, hincl, dd, TW);
                    if (tl >= dd) hincl += v;
                }
                const int H = __shfl_sync(kFull, hincl, TW - 1, TW);
                const int hoff = hincl - nh;
                cnt += nh;
                wM[tl] = make_uint4(m0, m1, m2, m3);
                wOff[tl] = hoff;
                __syncwarp();
                const int rb = (tl * H) / TW, re = ((tl + 1) * H) / TW;
                if (rb < re) {
                    // owner of position rb: the last target whose hits start at or before it
                    int o = 0;
#pragma unroll
                    for (int st = TW / 2; st > 0; st >>= 1)
                        if (wOff[o + st] <= rb) o += st;
                    uint4 M = wM[o];
                    drop_hits(M, rb - wOff[o]);  // those belong to the ranges before
                    int io = 0;
                    float4 po, vo, to;
                    float ho = 0.f, hinv_o = 0.f, hinv4_o = 0.f, ho2 = 0.f, band_o = 0.f;
                    auto owner = [&]() {
                        io = wI[o];
                        po = wP[o];
                        vo = wV[o];
                        to = wT[o];
                        ho = po.w;
                        const float4 q = wQ[o];
                        hinv_o = q.x;
                        hinv4_o = q.y;
                        ho2 = q.z;
                        band_o = q.w;
                    };
                    owner();
                    ForceSum part;
                    bool first = true;
                    for (int p = rb; p < re;) {
                        if ((M.x | M.y | M.z | M.w) == 0u) {  // the owner's hits end here
                            if (first) part.put(wF, wFv, tl);
                            else part.put(wD, wDv, o);  // a target inside this range: only this lane
                            first = false;
                            do {
                                ++o;
                                M = wM[o];
                            } while ((M.x | M.y | M.z | M.w) == 0u);
                            owner();
                        }
                        // two hits of the owner at once where the range holds them (two
                        // instruction streams, added in order: the sums of one at a time)
                        const int k1 = pop_bit(M.x, M.y, M.z, M.w);
                        const bool two = p + 1 < re && (M.x | M.y | M.z | M.w) != 0u;
                        const int k2 = two ? pop_bit(M.x, M.y, M.z, M.w) : k1;
                        p += two ? 2 : 1;
                        auto add = [&](int k) {
                            const float4 s = sA[k];
                            const float dx = po.x - s.x, dy = po.y - s.y, dz = po.z - s.z;
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            if (r2 > 0.f) {  // the pair (i, i), and coincident pairs, have no direction
                                const float hj2 = s.w * s.w;
                                bool in_i = r2 < ho2, in_j = r2 < hj2;
                                if (fabsf(r2 - ho2) <= band_o || fabsf(r2 - hj2) <= kBandK * s.w * (s.w + L)) {
                                    const unsigned d = band_decide(a.x, a.y, a.z, io, sI[k], a.box, ho, s.w);
                                    in_i = d & 1u;
                                    in_j = d & 2u;
                                }
                                force_term(dx, dy, dz, r2, in_i, in_j, hinv_o, hinv4_o, vo, to, s.w, sB[k], sC[k],
                                           a.alpha, part);
                            }
                        };
                        add(k1);
                        if (two) add(k2);
                    }
                    if (first) {
                        part.put(wF, wFv, tl);
                        wE[tl] = make_float4(0.f, 0.f, 0.f, 0.f);
                        wEv[tl] = 0.f;
                    } else {
                        part.put(wE, wEv, tl);
                    }
                } else {
                    wF[tl] = wE[tl] = make_float4(0.f, 0.f, 0.f, 0.f);
                    wFv[tl] = wEv[tl] = 0.f;
                }
                __syncwarp();
                if (nh > 0) {
                    // the ranges La..Lb hold this target's hits hoff..hoff + nh - 1
                    const int p0 = hoff, p1 = hoff + nh - 1;
                    const int La = min(TW - 1, ((p0 + 1) * TW - 1) / H);
                    const int Lb = min(TW - 1, ((p1 + 1) * TW - 1) / H);
                    const int bA = (La * H) / TW, eA = ((La + 1) * H) / TW;
                    float4 t4;
                    float tv;
                    if (La == Lb && p0 != bA && p1 + 1 != eA) {
                        t4 = wD[tl];
                        tv = wDv[tl];
                    } else if (p0 == bA) {  // the first target of range La
                        t4 = wF[La];
                        tv = wFv[La];
                    } else {  // the last one
                        t4 = wE[La];
                        tv = wEv[La];
                    }
                    for (int Lx = La + 1; Lx <= Lb; ++Lx) {  // ranges that start inside its hits
                        const float4 f = wF[Lx];
                        t4.x += f.x;
                        t4.y += f.y;
                        t4.z += f.z;
                        t4.w += f.w;
                        tv = fmaxf(tv, wFv[Lx]);
                    }
                    bx = t4.x;
                    by = t4.y;
                    bz = t4.z;
                    bu = t4.w;
                    vs = fmaxf(vs, tv);
                }
                __syncwarp();  // the scratch is rewritten by the next batch
                m0 = m1 = m2 = m3 = 0u;
            } else {
                // lane by lane (uniform grid: a cell's targets have similar hit counts)
                for (;;) {
                    const unsigned busy = __ballot_sync(kFull, (m0 | m1 | m2 | m3) != 0u);
                    if (busy == 0u) break;
                    if (m0 | m1 | m2 | m3) {
                        const int k = pop_bit(m0, m1, m2, m3);
                        const float4 s = sA[k];
                        const float4 vj = sB[k];
                        const float4 tj = sC[k];
                        const float dx = pi.x - s.x, dy = pi.y - s.y, dz = pi.z - s.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        ++cnt;
                        if (r2 > 0.f) {  // the pair (i, i), and coincident pairs, have no direction
                            bool in_i, in_j;
                            decide(r2, s.w, sI + k, in_i, in_j);
                            const float rinv = rsqrtf(r2);
                            const float r = r2 * rinv;
                            const float hjinv = __fdividef(1.f, s.w);
                            const float hj2inv = hjinv * hjinv;
                            const float dWi = in_i ? kSigma * spline_dw_u(r * hinv) * hinv4 : 0.f;
                            const float dWj = in_j ? kSigma * spline_dw_u(r * hjinv) * (hj2inv * hj2inv) : 0.f;
                            const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
                            const float mu = fmaf(vx, dx, fmaf(vy, dy, vz * dz)) * rinv;
                            // viscosity only on approach (mu < 0): branch-free, Pi = 0 otherwise
                            const float muc = fminf(mu, 0.f);
                            const float vsig_ij = ti.z + tj.z - 3.f * muc;
                            const float Pi = -a.alpha * vsig_ij * muc * (0.5f * (ti.w + tj.w)) *
                                             __fdividef(1.f, ti.x + tj.x);
                            const float dWbar = 0.5f * (dWi + dWj);
                            const float mj = vj.w;
                            const float sc = mj * fmaf(ti.y, dWi, fmaf(tj.y, dWj, Pi * dWbar)) * rinv;
                            bx = fmaf(-sc, dx, bx);
                            by = fmaf(-sc, dy, by);
                            bz = fmaf(-sc, dz, bz);
                            bu = fmaf(mj * mu, fmaf(ti.y, dWi, 0.5f * Pi * dWbar), bu);
                            vs = fmaxf(vs, vsig_ij);
                        }
                    }
                }
            }
            kahan_add(sx_, sxc, bx);
            kahan_add(sy_, syc, by);
            kahan_add(sz_, szc, bz);
            kahan_add(su, suc, bu);
            nst = 0;
            __syncwarp();
        };

        // the 27 cell ranges of the tile, fetched at once: lane tl holds cells tl, tl + TW
        // (radius-2 stencils, for h beyond the planned cell, load ranges one by one)
        int cs0 = 0, ce0 = 0, cs1 = 0, ce1 = 0;
        if (!LIST && live && R == 1) {
            if (tl < 27) {
                const int cb = bx.cell_off +
                               (wrapc(iz + kOrder[tl][2], nc) * nc + wrapc(iy + kOrder[tl][1], nc)) * nc +
                               wrapc(ix + kOrder[tl][0], nc);
                cs0 = a.cell_start[cb];
                ce0 = a.cell_start[cb + 1];
            }
            if (tl + TW < 27) {
                const int o2 = tl + TW;
                const int cb = bx.cell_off +
                               (wrapc(iz + kOrder[o2][2], nc) * nc + wrapc(iy + kOrder[o2][1], nc)) * nc +
                               wrapc(ix + kOrder[o2][0], nc);
                cs1 = a.cell_start[cb];
                ce1 = a.cell_start[cb + 1];
            }
        }
        // stage chunk after chunk; one flush site (keeps the kernel small)
        // (adaptive cells: the tile's list entries, each a leaf and its offset)
        uint32_t e0 = 0;
        int ne = 0;
        if (LIST && live) {
            e0 = a.list_off[tile.x];
            ne = (int)(a.list_off[tile.x + 1] - e0);
        }
        int o = -1, ch = 0, nchunk = 0, bs = 0, be = 0;
        const int ncell = LIST ? (int)__reduce_max_sync(kFull, (unsigned)ne) : (R == 1 ? 27 : 125);
        float shx = 0.f, shy = 0.f, shz = 0.f;  // offset of the chunk's sources (list mode: per lane)
        ListStream<TW> ls;
        int sw_d = -1;  // axis sweep of the current cell (SPH_FLAG_AXIS_SWEEP, radius 1)
        float sw_sg = 0.f, sw_lim = 0.f;
        const float rlim = SWEEP ? sqrtf(reach2) : 0.f;
        for (;;) {
            if (LIST) {
                while (ch >= nchunk && ls.template next<true>(a.list, a.leaf_rng, a.leaf_lo, a.leaf_hi, e0, ne, ncell, tl,
                                                              nchunk, lox, hix, loy, hiy, loz, hiz, reach2, H, L))
                    ch = 0;
            }
            while (!LIST && ch >= nchunk && o < ncell - 1) {
                ++o;
                ch = 0;
                int ox, oy, oz;
                if (R == 1) {
                    const int src = o < TW ? o : o - TW;
                    bs = __shfl_sync(kFull, o < TW ? cs0 : cs1, src, TW);
                    be = __shfl_sync(kFull, o < TW ? ce0 : ce1, src, TW);
                    ox = kOrder[o][0];
                    oy = kOrder[o][1];
                    oz = kOrder[o][2];
                } else {
                    ox = o < 27 ? kOrder[o][0] : kOuter[o - 27][0];
                    oy = o < 27 ? kOrder[o][1] : kOuter[o - 27][1];
                    oz = o < 27 ? kOrder[o][2] : kOuter[o - 27][2];
                    bs = be = 0;
                    if (live) {
                        const int cb = bx.cell_off + (wrapc(iz + oz, nc) * nc + wrapc(iy + oy, nc)) * nc +
                                       wrapc(ix + ox, nc);
                        bs = a.cell_start[cb];
                        be = a.cell_start[cb + 1];
                    }
                }
                nchunk = (int)__reduce_max_sync(kFull, (unsigned)((be - bs + TW - 1) / TW));
                shx = (float)ox * L;
                shy = (float)oy * L;
                shz = (float)oz * L;
                sw_d = -1;
                if (SWEEP && R == 1 && o > 0) {
                    sw_d = kOrderAxis[o][0];
                    sw_sg = (float)kOrderAxis[o][1];
                    sw_lim = sweep_limit(o, L, rlim, lox, hix, loy, hiy, loz, hiz);
                }
            }
            const bool more = ch < nchunk;  // warp-uniform
            if (more) {
                const int q = ch * TW + tl;
                int j = bs + q;
                bool vq = q < be - bs;
                if (LIST) ls.slot(ch * TW, tl, j, vq, shx, shy, shz);
                if (SWEEP && sw_d >= 0 && vq) {  // the cell's order along the axis, up to the sweep bound
                    const float2 e = a.axis[(size_t)sw_d * a.axis_stride + bs + (sw_sg > 0.f ? q : be - bs - 1 - q)];
                    j = __float_as_int(e.y);
                    vq = sw_sg * e.x < sw_lim;
                }
                // (no branch: a lane past the chunk's end reads slot 0 and keeps nothing)
                const int jj = vq ? j : 0;
                float4 pj = __ldg(a.pos4 + jj);
                const float4 vj = __ldg(a.vel4 + jj);
                const float4 tj = __ldg(a.thermo4 + jj);
                pj.x += shx;
                pj.y += shy;
                pj.z += shz;
                const float ex = fmaxf(fmaxf(lox - pj.x, pj.x - hix), 0.f);
                const float ey = fmaxf(fmaxf(loy - pj.y, pj.y - hiy), 0.f);
                const float ez = fmaxf(fmaxf(loz - pj.z, pj.z - hiz), 0.f);
                float r2max = reach2;
                if (LIST) {
                    const float m = fmaxf(H, pj.w);
                    r2max = m * m * (1.f + kPruneMargin) + 2.f * kBandK * m * (m + L);
                }
                if constexpr (LIST) acc_stream += vq ? 1u : 0u;
                const bool keep = vq && fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < r2max;
                const unsigned mine = __ballot_sync(kFull, keep) & gmask;
                if (keep) {
                    const int pos = nst + __popc(mine & lt);
                    sA[pos] = pj;
                    sB[pos] = vj;
                    sC[pos] = tj;
                    sI[pos] = jj;
                    if constexpr (LIST) {
                        sX[pos] = pj.x;
                        sY[pos] = pj.y;
                        sZ[pos] = pj.z;
                        const float hj2 = pj.w * pj.w, bj = kBandK * pj.w * (pj.w + L);
                        sLo[pos] = hj2 - bj;
                        sHi[pos] = hj2 + bj;
                    }
                }
                nst += __popc(mine);
                ++ch;
            }
            const int mx = (int)__reduce_max_sync(kFull, (unsigned)nst);
            if (mx > B - TW || (!more && mx > 0)) flush();
            if (!more) break;
        }

        const int nself = act ? 1 : 0;  // the (i, i) pair is not a neighbour
        acc_pairs += (unsigned)(cnt - nself);
        if (tl == 0) acc_cand += cand * (unsigned)__popc(amask & gmask);
        if (tl == 0) acc_staged += cand;
        if (!act) continue;
        a.ax[i] = sx_ - sxc;
        a.ay[i] = sy_ - syc;
        a.az[i] = sz_ - szc;
        a.dudt[i] = su - suc;
        a.vsig[i] = vs;
    }
    const unsigned long long tp = warp_sum_ull(acc_pairs), tc = warp_sum_ull(acc_cand);  // 64-bit sums
    const unsigned long long ts = warp_sum_ull(acc_stream), tg = warp_sum_ull(acc_staged);
    if (lane == 0) {
        if (tp) atomicAdd(a.counters + C_FPAIRS, tp);
        if (tc) atomicAdd(a.counters + C_FCAND, tc);
        if (ts) atomicAdd(a.counters + C_FSTREAM, ts);
        if (tg) atomicAdd(a.counters + C_FSTAGED, tg);
    }
}

// ------------------------------------------------ symmetric force pass (f4)
// Each unordered cell pair once (the paper's pair tasks, Sec. 3.1, which update both
// cells): one warp owns a cell, takes its particles as targets in groups of 32, and
// visits its own cell in gather form (every target sums over every other particle of
// the cell) and the 13 cells of a half stencil (kOrder[1], kOrder[3], ..., kOrder[25]:
// one of each pair +d, -d) symmetrically: each pair (i, j) with j in neighbour cell
// B = A + d is evaluated once, and its term goes to i (the target, in registers)
// and to j (the source).  Determinism without atomics on the sums: within a round of
// the hit walk, lanes that hit the same source form a group (match_any) whose terms
// the lowest lane adds in lane order into the batch's per-source sum; after the
// batch, the warp adds those into slot s of j (s = 1..13, the direction index), a
// slot only the warp of cell B - d_s ever writes, in a fixed order (groups, then
// batches).  A final pass adds the 13 slots to the target-side sums in slot order.
// v_sig is a maximum (order-free): an atomic max on its bits.
// Needs every cell's reach within one cell side (no radius-2 stencil): otherwise
// *need_gather is set beforehand and the gather kernel runs the pass instead.

constexpr int kSymSlots = 13;

struct ForceSymArgs {
    const float4 *__restrict__ pos4;
    const float4 *__restrict__ vel4;
    const float4 *__restrict__ thermo4;
    const int *__restrict__ cell_start;
    const double *__restrict__ x;
    const double *__restrict__ y;
    const double *__restrict__ z;
    const float *__restrict__ cell_reach;
    const BoxDev *__restrict__ boxes;
    float *ax, *ay, *az, *dudt, *vsig;    // target-side sums (plain stores)
    float4 *slot;                         // kSymSlots x n: source-side sums {a, du/dt}
    unsigned *vsig_src;                   // n: source-side max v_sig (float bits)
    const unsigned long long *need_gather;
    unsigned long long *counters;
    int64_t n_cells, n;
    int nb;
    double box;
    float alpha;
};

__device__ __forceinline__ int sym_box_of_cell(int c, const BoxDev *__restrict__ bx, int nb)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bx[mid].cell_off <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kPairThreads, kForceBlocks) k_force_sym(ForceSymArgs a)
{
    if (*a.need_gather) return;
    constexpr int TW = 32;
    constexpr int B = kBatchF;
    constexpr int SLOT = B + 1;
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwb = blockDim.x >> 5;
    float4 *sA = smem + (size_t)wib * (4 * SLOT);  // {x, y, z, h_j} in the target frame
    float4 *sB = sA + SLOT;                         // {vx, vy, vz, m}
    float4 *sC = sB + SLOT;                         // {rho, A, c, B}
    float4 *sS = sC + SLOT;                         // source-side sums of the batch
    int *sI = (int *)(smem + (size_t)nwb * (4 * SLOT)) + (size_t)wib * SLOT;  // slot * 16 + stencil index
    float *sV = (float *)(smem + (size_t)nwb * (4 * SLOT)) + (size_t)nwb * SLOT + (size_t)wib * SLOT;  // max v_sig
    const unsigned lt = (1u << lane) - 1u;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int ncells = (int)a.n_cells;
    const float inf = __int_as_float(0x7f800000);
    unsigned acc_pairs = 0u, acc_cand = 0u;
    unsigned *ticket = reinterpret_cast<unsigned *>(a.counters + C_TICKET);
    unsigned tk = 0u;
    if (lane == 0) tk = atomicAdd(ticket, 1u);
    for (int c = gw, c_after = 0; c < ncells; c = c_after) {
        c_after = nw + (int)__shfl_sync(kFull, tk, 0);
        if (lane == 0 && c_after < ncells) tk = atomicAdd(ticket, 1u);
        const int cs = a.cell_start[c], ce = a.cell_start[c + 1];
        if (cs == ce) continue;
        const BoxDev bx = a.boxes[a.nb == 1 ? 0 : sym_box_of_cell(c, a.boxes, a.nb)];
        const int nc = bx.nc;
        const float L = bx.L32;
        const int ca = c - bx.cell_off;
        const int ix = ca % nc, iy = (ca / nc) % nc, iz = ca / (nc * nc);
        // ranges of the 14 cells: lane s < 14 holds stencil entry s (0 = own cell,
        // s >= 1: kOrder[2 s - 1])
        int csl = 0, cel = 0;
        if (lane < 14) {
            const int o = lane == 0 ? 0 : 2 * lane - 1;
            const int cb = bx.cell_off + (wrapc(iz + kOrder[o][2], nc) * nc + wrapc(iy + kOrder[o][1], nc)) * nc +
                           wrapc(ix + kOrder[o][0], nc);
            csl = a.cell_start[cb];
            cel = a.cell_start[cb + 1];
        }
        const float hreach = a.cell_reach[c];
        for (int g0 = cs; g0 < ce; g0 += TW) {
            const int i = g0 + lane;
            const bool act = i < ce;
            float4 pi = make_float4(kFar, kFar, kFar, 0.f), vi = make_float4(0.f, 0.f, 0.f, 0.f),
                   ti = make_float4(1.f, 0.f, 0.f, 0.f);
            if (act) {
                pi = a.pos4[i];
                vi = a.vel4[i];
                ti = a.thermo4[i];
            }
            const float lox = tile_min<TW>(act ? pi.x : inf), hix = tile_max<TW>(act ? pi.x : -inf);
            const float loy = tile_min<TW>(act ? pi.y : inf), hiy = tile_max<TW>(act ? pi.y : -inf);
            const float loz = tile_min<TW>(act ? pi.z : inf), hiz = tile_max<TW>(act ? pi.z : -inf);
            const float hi = pi.w;
            const float H = fmaxf(tile_max<TW>(hi), hreach);
            const float bandmax = 2.f * kBandK * H * (H + L);
            const float reach2 = H * H * (1.f + kPruneMargin) + bandmax;
            const float hi2 = hi * hi;
            const float hinv = act ? 1.f / hi : 0.f;
            const float hinv4 = hinv * hinv * hinv * hinv;
            const float band_i = kBandK * hi * (hi + L);
            const float mi_ = vi.w;
            float sx_ = 0.f, sxc = 0.f, sy_ = 0.f, syc = 0.f, sz_ = 0.f, szc = 0.f, su = 0.f, suc = 0.f;
            float vs = 0.f;
            int cnt = 0;
            unsigned cand = 0;
            int nst = 0;

            auto flush = [&]() {
                const int nmax = (int)((__reduce_max_sync(kFull, (unsigned)nst) + 3u) & ~3u);
                for (int k = nst + lane; k < nmax; k += TW) {
                    sA[k] = make_float4(-kFar, -kFar, -kFar, 0.f);
                    sI[k] = 0;
                }
                for (int k = lane; k < nmax; k += TW) {
                    sS[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    sV[k] = 0.f;
                }
                __syncwarp();
                cand += (unsigned)nst;
                unsigned m0 = 0u, m1 = 0u, m2 = 0u, m3 = 0u;
                const int nwords = (nmax + 31) >> 5;
#pragma unroll 1
                for (int wd = 0; wd < nwords; ++wd) {
                    const int kend = min(32, nmax - 32 * wd);
                    const float4 *sw = sA + 32 * wd;
                    unsigned mw = 0u, bw = 0u;
                    for (int k4 = 0; k4 < kend; k4 += 4) {
                        unsigned mn = 0u, bn = 0u;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float4 s = sw[k4 + u];
                            const float dx = pi.x - s.x, dy = pi.y - s.y, dz = pi.z - s.z;
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            const float d2 = r2 - fmaxf(hi2, s.w * s.w);
                            mn |= (unsigned)(d2 < -bandmax) << u;
                            bn |= (unsigned)(d2 < bandmax) << u;
                        }
                        mw |= mn << k4;
                        bw |= bn << k4;
                    }
                    bw &= ~mw;  // below the band's top and not a hit
                    while (bw) {
                        const int kk = __ffs(bw) - 1;
                        bw &= bw - 1u;
                        if (band_decide(a.x, a.y, a.z, i, sI[32 * wd + kk] >> 4, a.box, hi, sw[kk].w) != 0u)
                            mw |= 1u << kk;
                    }
                    m0 = wd == 0 ? mw : m0;
                    m1 = wd == 1 ? mw : m1;
                    m2 = wd == 2 ? mw : m2;
                    m3 = wd == 3 ? mw : m3;
                }
                float bx_ = 0.f, by_ = 0.f, bz_ = 0.f, bu = 0.f;
                while (__any_sync(kFull, (m0 | m1 | m2 | m3) != 0u)) {
                    // this round: each lane's next hit (lowest staged index first)
                    int k = -1;
                    float cx = 0.f, cy = 0.f, cz = 0.f, cu = 0.f, cv = 0.f;
                    bool src = false;
                    if (m0 | m1 | m2 | m3) {
                        k = pop_bit(m0, m1, m2, m3);
                        const float4 s = sA[k];
                        const float4 vj = sB[k];
                        const float4 tj = sC[k];
                        const int code = sI[k];
                        const float dx = pi.x - s.x, dy = pi.y - s.y, dz = pi.z - s.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        src = (code & 15) != 0;
                        cnt += src ? 2 : 1;
                        if (r2 > 0.f) {
                            const float hj2 = s.w * s.w;
                            bool in_i = r2 < hi2, in_j = r2 < hj2;
                            const float band_j = kBandK * s.w * (s.w + L);
                            if (fabsf(r2 - hi2) <= band_i || fabsf(r2 - hj2) <= band_j) {
                                const unsigned dd = band_decide(a.x, a.y, a.z, i, code >> 4, a.box, hi, s.w);
                                in_i = dd & 1u;
                                in_j = dd & 2u;
                            }
                            const float rinv = rsqrtf(r2);
                            const float r = r2 * rinv;
                            const float hjinv = __fdividef(1.f, s.w);
                            const float hj2inv = hjinv * hjinv;
                            const float dWi = in_i ? kSigma * spline_dw_u(r * hinv) * hinv4 : 0.f;
                            const float dWj = in_j ? kSigma * spline_dw_u(r * hjinv) * (hj2inv * hj2inv) : 0.f;
                            const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
                            const float mu = fmaf(vx, dx, fmaf(vy, dy, vz * dz)) * rinv;
                            const float muc = fminf(mu, 0.f);
                            const float vsig_ij = ti.z + tj.z - 3.f * muc;
                            const float Pi = -a.alpha * vsig_ij * muc * (0.5f * (ti.w + tj.w)) *
                                             __fdividef(1.f, ti.x + tj.x);
                            const float pdw = 0.5f * Pi * (0.5f * (dWi + dWj));  // (1/2) Pi dW-bar
                            const float X = fmaf(ti.y, dWi, fmaf(tj.y, dWj, 2.f * pdw)) * rinv;
                            const float mj = vj.w;
                            bx_ = fmaf(-mj * X, dx, bx_);
                            by_ = fmaf(-mj * X, dy, by_);
                            bz_ = fmaf(-mj * X, dz, bz_);
                            bu = fmaf(mj * mu, fmaf(ti.y, dWi, pdw), bu);
                            vs = fmaxf(vs, vsig_ij);
                            if (src) {  // the same pair seen from j: d_ji = -d_ij, same mu
                                const float mX = mi_ * X;
                                cx = mX * dx;
                                cy = mX * dy;
                                cz = mX * dz;
                                cu = mi_ * mu * fmaf(tj.y, dWj, pdw);
                                cv = vsig_ij;
                            }
                        } else if (src) {
                            cv = 0.f;
                        }
                    }
                    // the lanes that hit the same source: the lowest adds the group's
                    // terms in lane order into the batch's sum for that source
                    const unsigned peers = __match_any_sync(kFull, src ? k : -1 - lane);
                    const int leader = __ffs(peers) - 1;
                    const unsigned others = peers & ~(1u << leader);
                    const int nothers = lane == leader ? __popc(others) : 0;
                    const int mo = (int)__reduce_max_sync(kFull, (unsigned)nothers);
                    float gx = cx, gy = cy, gz = cz, gu = cu, gv = cv;
                    for (int t = 0; t < mo; ++t) {
                        const int from = t < nothers ? (int)__fns(others, 0u, t + 1) : lane;
                        const float ox = __shfl_sync(kFull, cx, from), oy = __shfl_sync(kFull, cy, from);
                        const float oz = __shfl_sync(kFull, cz, from), ou = __shfl_sync(kFull, cu, from);
                        const float ov = __shfl_sync(kFull, cv, from);
                        if (t < nothers) {
                            gx += ox;
                            gy += oy;
                            gz += oz;
                            gu += ou;
                            gv = fmaxf(gv, ov);
                        }
                    }
                    if (src && lane == leader) {
                        float4 acc = sS[k];
                        acc.x += gx;
                        acc.y += gy;
                        acc.z += gz;
                        acc.w += gu;
                        sS[k] = acc;
                        sV[k] = fmaxf(sV[k], gv);
                    }
                    __syncwarp();
                }
                kahan_add(sx_, sxc, bx_);
                kahan_add(sy_, syc, by_);
                kahan_add(sz_, szc, bz_);
                kahan_add(su, suc, bu);
                // the batch's source sums into the slots of their particles (one writer
                // per slot: this warp, in batch order)
                for (int k = lane; k < nst; k += TW) {
                    const int code = sI[k];
                    const int s = code & 15;
                    if (s == 0) continue;
                    const int j = code >> 4;
                    const float4 v = sS[k];
                    float4 *dst = a.slot + (size_t)(s - 1) * (size_t)a.n + j;
                    float4 o = *dst;
                    o.x += v.x;
                    o.y += v.y;
                    o.z += v.z;
                    o.w += v.w;
                    *dst = o;
                    if (sV[k] > 0.f) atomicMax(a.vsig_src + j, __float_as_uint(sV[k]));
                }
                nst = 0;
                __syncwarp();
            };

            // stream the 14 cells, TW sources at a time; box-prune against the group
            for (int s = 0; s < 14; ++s) {
                const int bs = __shfl_sync(kFull, csl, s), be = __shfl_sync(kFull, cel, s);
                const int o = s == 0 ? 0 : 2 * s - 1;
                const float shx = (float)kOrder[o][0] * L, shy = (float)kOrder[o][1] * L,
                            shz = (float)kOrder[o][2] * L;
                for (int base = bs; base < be; base += TW) {
                    const int j = base + lane;
                    const bool vq = j < be;
                    const int jj = vq ? j : bs;
                    float4 pj = __ldg(a.pos4 + jj);
                    const float4 vj = __ldg(a.vel4 + jj);
                    const float4 tj = __ldg(a.thermo4 + jj);
                    pj.x += shx;
                    pj.y += shy;
                    pj.z += shz;
                    const float ex = fmaxf(fmaxf(lox - pj.x, pj.x - hix), 0.f);
                    const float ey = fmaxf(fmaxf(loy - pj.y, pj.y - hiy), 0.f);
                    const float ez = fmaxf(fmaxf(loz - pj.z, pj.z - hiz), 0.f);
                    const bool keep = vq && fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < reach2;
                    const unsigned mine = __ballot_sync(kFull, keep);
                    if (keep) {
                        const int pos = nst + __popc(mine & lt);
                        sA[pos] = pj;
                        sB[pos] = vj;
                        sC[pos] = tj;
                        sI[pos] = (jj << 4) | s;
                    }
                    nst += __popc(mine);
                    if (nst > B - TW) flush();
                }
            }
            if (nst > 0) flush();
            const int nself = act ? 1 : 0;
            acc_pairs += (unsigned)(cnt - nself);
            const unsigned am = __ballot_sync(kFull, act);
            if (lane == 0) acc_cand += cand * (unsigned)__popc(am);
            if (act) {
                a.ax[i] = sx_ - sxc;
                a.ay[i] = sy_ - syc;
                a.az[i] = sz_ - szc;
                a.dudt[i] = su - suc;
                a.vsig[i] = vs;
            }
        }
    }
    const unsigned long long tp = warp_sum_ull(acc_pairs), tc = warp_sum_ull(acc_cand);
    if (lane == 0) {
        if (tp) atomicAdd(a.counters + C_FPAIRS, tp);
        if (tc) atomicAdd(a.counters + C_FCAND, tc);
    }
}

// Whether some cell's reach exceeds its side (the symmetric pass covers one cell
// around each cell only): sets *flag.
__global__ void k_sym_check(const float *__restrict__ reach, const BoxDev *__restrict__ bx, int nb, int64_t ncells,
                            unsigned long long *flag)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const float L = bx[nb == 1 ? 0 : sym_box_of_cell((int)c, bx, nb)].L32;
    if (reach[c] * (1.f + kPruneMargin) > L) atomicOr(flag, 1ull);
}

// target-side sums + the 13 source-side slots (slot order) and the two v_sig maxima
__global__ void k_sym_reduce(const float4 *__restrict__ slot, const unsigned *__restrict__ vsig_src, int64_t n,
                             const unsigned long long *__restrict__ need_gather, float *ax, float *ay, float *az,
                             float *dudt, float *vsig)
{
    if (*need_gather) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x = ax[i], y = ay[i], z = az[i], u = dudt[i];
#pragma unroll
    for (int s = 0; s < kSymSlots; ++s) {
        const float4 v = slot[(size_t)s * (size_t)n + i];
        x += v.x;
        y += v.y;
        z += v.z;
        u += v.w;
    }
    ax[i] = x;
    ay[i] = y;
    az[i] = z;
    dudt[i] = u;
    vsig[i] = fmaxf(vsig[i], __uint_as_float(vsig_src[i]));
}

__global__ void k_sync_h(const float *__restrict__ h, float4 *__restrict__ pos4, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pos4[i].w = h[i];
}

template <int TW>
static size_t density_smem(bool list)
{
    return (size_t)(kPairThreads / 32) * 2 * (32 / TW) * (kBatchD + 1) * sizeof(float4) +
           (list ? (size_t)(kPairThreads / 32) * 32 * kWalkBytesD : 0);
}
template <int TW>
static size_t force_smem(bool list)
{
    const size_t slots = (size_t)(kPairThreads / 32) * (32 / TW) * (kBatchF + 1);
    const size_t tiles = (size_t)(kPairThreads / 32) * (32 / TW);
    return slots * (3 * sizeof(float4) + sizeof(int)) +
           (list ? tiles * (5 * kSlotF * sizeof(float) + (size_t)TW * kWalkBytes) : 0);
}

static size_t force_sym_smem()
{
    const size_t slots = (size_t)(kPairThreads / 32) * (kBatchF + 1);
    return slots * (4 * sizeof(float4) + sizeof(int) + sizeof(float));
}

// Opt the pair kernels into more than 48 KB of dynamic shared memory (once per process;
// the attribute is per function, not per device).
static int smem_optin(sph_ctx *ctx)
{
    static bool done = false;
    if (done) return SPH_OK;
    const int d16 = (int)density_smem<16>(true), d32 = (int)density_smem<32>(true);
    const int f16 = (int)force_smem<16>(true), f32 = (int)force_smem<32>(true);
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
#define SPH_OPT_D(M)                                                              \
    SPH_CUDA(ctx, cudaFuncSetAttribute(k_density<16, false, M>, at, d16));        \
    SPH_CUDA(ctx, cudaFuncSetAttribute(k_density<16, true, M>, at, d16));         \
    SPH_CUDA(ctx, cudaFuncSetAttribute(k_density<32, false, M>, at, d32));        \
    SPH_CUDA(ctx, cudaFuncSetAttribute(k_density<32, true, M>, at, d32));         \
    SPH_CUDA(ctx, cudaFuncSetAttribute(k_force<16, M>, at, f16));                 \
    SPH_CUDA(ctx, cudaFuncSetAttribute(k_force<32, M>, at, f32));
    SPH_OPT_D(0)
    SPH_OPT_D(1)
    SPH_OPT_D(2)
#undef SPH_OPT_D
    SPH_CUDA(ctx, cudaFuncSetAttribute(k_force_sym, at, (int)force_sym_smem()));
    done = true;
    return SPH_OK;
}

static int pair_grid(sph_ctx *ctx, int blocks_per_sm)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (sms <= 0) sms = 148;
    // persistent grid: warps stride over the tile groups
    const int64_t cells = ctx->adaptive ? ctx->tree.n_leaves : ctx->grid.n_cells;
    int64_t want = ((int64_t)ctx->n / ctx->tile_w + cells) / (kPairThreads / 32) + 1;
    int64_t g = std::min<int64_t>((int64_t)sms * blocks_per_sm, want);
    return (int)std::max<int64_t>(g, 1);
}

// Tiles that still hold an unconverged target, for the later density passes, kept
// in their original order (flags, exclusive prefix sum, scatter): which tiles share
// a warp, and so where a tile's staged batches end, is then the same on every run,
// and with it every rounding.
// (*unconv: the targets the last pass left active; none -- a captured step's passes
// after convergence -- leaves nothing to flag, and the scatter below runs no tile)
__global__ void k_tile_flags(const int4 *__restrict__ tiles, const int *__restrict__ n_tiles,
                             const uint8_t *__restrict__ active, const int *__restrict__ tord, int64_t cap,
                             const unsigned long long *__restrict__ unconv, uint32_t *__restrict__ flag)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cap || *unconv == 0ull) return;
    bool keep = false;
    if (t < *n_tiles) {
        const int4 tile = tiles[t];
        for (int k = 0; k < tile.z && !keep; ++k) keep = active[tord ? tord[tile.y + k] : tile.y + k] != 0;
    }
    flag[t] = keep ? 1u : 0u;
}

__global__ void k_tile_scatter(const int4 *__restrict__ tiles, const uint32_t *__restrict__ flag,
                               const uint32_t *__restrict__ pos, int64_t cap,
                               const unsigned long long *__restrict__ unconv, int4 *__restrict__ out,
                               int *__restrict__ n_out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cap) return;
    if (*unconv == 0ull) {
        if (t == 0) *n_out = 0;
        return;
    }
    if (flag[t]) out[pos[t]] = tiles[t];
    if (t == cap - 1) *n_out = (int)(pos[t] + flag[t]);
}

int compact_active_tiles(sph_ctx *ctx)
{
    // every tile holds <= tile_w targets of one cell: at most n / tile_w + n_cells
    // tiles (uniform grid), far fewer than the array's capacity
    int64_t cap = ctx->tile_cap;
    if (!ctx->adaptive) cap = std::min<int64_t>(cap, ctx->grid.n_cells + ctx->n / ctx->tile_w + 1);
    const unsigned blocks = (unsigned)((cap + 255) / 256);
    k_tile_flags<<<blocks, 256, 0, ctx->stream>>>(ctx->tiles, ctx->n_tiles, ctx->active,
                                                 ctx->adaptive ? ctx->tree.tord : nullptr, cap, ctx->counters + C_UNCONV,
                                                 ctx->tile_flag);
    SPH_LAUNCH(ctx, "tile flags");
    int rc = exclusive_scan_u32(ctx, ctx->tile_flag, ctx->tile_pos, cap);
    if (rc) return rc;
    k_tile_scatter<<<blocks, 256, 0, ctx->stream>>>(ctx->tiles, ctx->tile_flag, ctx->tile_pos, cap,
                                                   ctx->counters + C_UNCONV, ctx->act_tiles, ctx->n_act_tiles);
    SPH_LAUNCH(ctx, "compact tiles");
    return SPH_OK;
}

int run_density_pass(sph_ctx *ctx, sph_particles *parts, bool last_pass, bool active_list)
{
    DensityArgs a{};  // every field not set below is null / zero
    a.pos4 = ctx->pos4;
    a.vel4 = ctx->vel4;
    a.cell_start = ctx->cell_start;
    a.tiles = active_list ? ctx->act_tiles : ctx->tiles;
    a.n_tiles = active_list ? ctx->n_act_tiles : ctx->n_tiles;
    a.x = parts->x;
    a.y = parts->y;
    a.z = parts->z;
    a.ids = ctx->ids;
    a.upred = ctx->upred;
    a.active = ctx->active;
    a.h = parts->h;
    a.h_lo = ctx->h_lo;
    a.h_hi = ctx->h_hi;
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
    a.boxes = ctx->d_boxes;
    a.list_off = ctx->tree.list_off;
    a.list = ctx->tree.list;
    a.leaf_rng = ctx->tree.leaf_rng;
    a.leaf_scale = ctx->tree.leaf_scale;
    a.leaf_lo = ctx->tree.leaf_lo;
    a.leaf_hi = ctx->tree.leaf_hi;
    a.leaf_hb = ctx->tree.leaf_h;
    a.hold_cells = ctx->tree.device_sized ? 1 : 0;  // captured steps
    // adaptive cells: later passes run tiles of the active targets only (act_ord)
    a.tord = ctx->adaptive && active_list ? ctx->tree.act_ord : ctx->tree.tord;
    a.axis = (ctx->p.flags & SPH_FLAG_AXIS_SWEEP) && !ctx->adaptive ? ctx->axis : nullptr;
    a.axis_stride = std::max<int64_t>(ctx->cap, 1);
    a.box = ctx->p.box_size;
    a.n_ngb_target = ctx->p.n_ngb;
    a.h_tol = ctx->p.h_tol;
    a.gamma = ctx->p.gamma;
    a.use_balsara = ctx->p.use_balsara;
    a.last_pass = last_pass ? 1 : 0;
    int rc = smem_optin(ctx);
    if (rc) return rc;
    const int g = pair_grid(ctx, kDensityBlocks);
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_TICKET, 0, sizeof(unsigned long long), ctx->stream));
    const bool hash = (ctx->p.flags & SPH_FLAG_NGB_HASH) != 0;
    cudaEvent_t end = nullptr;
    timer_begin(ctx, 0, &end);
    const int mode = ctx->adaptive ? 1 : (a.axis ? 2 : 0);
    const size_t sm = ctx->tile_w == 32 ? density_smem<32>(ctx->adaptive) : density_smem<16>(ctx->adaptive);
#define SPH_LAUNCH_D(TWv, Hv, Mv) k_density<TWv, Hv, Mv><<<g, kPairThreads, sm, ctx->stream>>>(a)
    if (ctx->tile_w == 32) {
        if (mode == 1) { if (hash) SPH_LAUNCH_D(32, true, 1); else SPH_LAUNCH_D(32, false, 1); }
        else if (mode == 2) { if (hash) SPH_LAUNCH_D(32, true, 2); else SPH_LAUNCH_D(32, false, 2); }
        else { if (hash) SPH_LAUNCH_D(32, true, 0); else SPH_LAUNCH_D(32, false, 0); }
    } else {
        if (mode == 1) { if (hash) SPH_LAUNCH_D(16, true, 1); else SPH_LAUNCH_D(16, false, 1); }
        else if (mode == 2) { if (hash) SPH_LAUNCH_D(16, true, 2); else SPH_LAUNCH_D(16, false, 2); }
        else { if (hash) SPH_LAUNCH_D(16, true, 0); else SPH_LAUNCH_D(16, false, 0); }
    }
#undef SPH_LAUNCH_D
    timer_end(ctx, end);
    SPH_LAUNCH(ctx, "density kernel");
    ctx->st.density_passes++;
    return SPH_OK;
}

// active_list: the tiles compacted from ctx->active (individual time-steps)
int run_force_pass(sph_ctx *ctx, sph_particles *parts, bool active_list)
{
    ForceArgs a{};
    a.pos4 = ctx->pos4;
    a.vel4 = ctx->vel4;
    a.thermo4 = ctx->thermo4;
    a.cell_start = ctx->cell_start;
    a.tiles = active_list ? ctx->act_tiles : ctx->tiles;
    a.n_tiles = active_list ? ctx->n_act_tiles : ctx->n_tiles;
    a.x = parts->x;
    a.y = parts->y;
    a.z = parts->z;
    a.cell_reach = ctx->cell_tmp;  // uniform grid only
    a.list_off = ctx->tree.list_off;
    a.list = ctx->tree.list;
    a.leaf_rng = ctx->tree.leaf_rng;
    a.leaf_scale = ctx->tree.leaf_scale;
    a.leaf_lo = ctx->tree.leaf_lo;
    a.leaf_hi = ctx->tree.leaf_hi;
    a.tord = ctx->adaptive && active_list ? ctx->tree.act_ord : ctx->tree.tord;
    a.axis = (ctx->p.flags & SPH_FLAG_AXIS_SWEEP) && !ctx->adaptive ? ctx->axis : nullptr;
    a.axis_stride = std::max<int64_t>(ctx->cap, 1);
    a.ax = parts->ax;
    a.ay = parts->ay;
    a.az = parts->az;
    a.dudt = parts->dudt;
    a.vsig = parts->vsig;
    a.fmask = ctx->bin_mode ? ctx->bin_active : nullptr;
    a.counters = ctx->counters;
    a.boxes = ctx->d_boxes;
    a.box = ctx->p.box_size;
    a.alpha = ctx->p.alpha_visc;
    int rc = smem_optin(ctx);
    if (rc) return rc;
    const int g = pair_grid(ctx, ctx->adaptive ? kForceBlocks : kForceBlocksU);
    // symmetric variant (uniform grid, every target, radius-1 reach): the gather
    // kernel below then runs only if some cell needs the radius-2 stencil
    const bool sym = ctx->sym_force && !ctx->adaptive && !a.fmask && !a.axis && !active_list &&
                     ctx->n < ((int64_t)1 << 27);
    if (sym) {
        rc = ensure_sym(ctx);
        if (rc) return rc;
        const int64_t nc = ctx->grid.n_cells, n = ctx->n;
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_SYMGATHER, 0, sizeof(unsigned long long), ctx->stream));
        k_sym_check<<<(unsigned)((nc + 255) / 256), 256, 0, ctx->stream>>>(ctx->cell_tmp, ctx->d_boxes, ctx->n_boxes,
                                                                         nc, ctx->counters + C_SYMGATHER);
        SPH_LAUNCH(ctx, "symmetric force check");
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->sym_slot, 0, sizeof(float4) * kSymSlots * (size_t)n, ctx->stream));
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->sym_vsig, 0, sizeof(unsigned) * (size_t)n, ctx->stream));
        ForceSymArgs sa{};
        sa.pos4 = ctx->pos4;
        sa.vel4 = ctx->vel4;
        sa.thermo4 = ctx->thermo4;
        sa.cell_start = ctx->cell_start;
        sa.x = parts->x;
        sa.y = parts->y;
        sa.z = parts->z;
        sa.cell_reach = ctx->cell_tmp;
        sa.boxes = ctx->d_boxes;
        sa.ax = parts->ax;
        sa.ay = parts->ay;
        sa.az = parts->az;
        sa.dudt = parts->dudt;
        sa.vsig = parts->vsig;
        sa.slot = ctx->sym_slot;
        sa.vsig_src = ctx->sym_vsig;
        sa.need_gather = ctx->counters + C_SYMGATHER;
        sa.counters = ctx->counters;
        sa.n_cells = nc;
        sa.n = n;
        sa.nb = ctx->n_boxes;
        sa.box = ctx->p.box_size;
        sa.alpha = ctx->p.alpha_visc;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        if (sms <= 0) sms = 148;
        const int gs = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * kForceBlocks,
                                                                    nc / (kPairThreads / 32) + 1));
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_TICKET, 0, sizeof(unsigned long long), ctx->stream));
        cudaEvent_t end = nullptr;
        timer_begin(ctx, 1, &end);
        k_force_sym<<<gs, kPairThreads, force_sym_smem(), ctx->stream>>>(sa);
        timer_end(ctx, end);
        SPH_LAUNCH(ctx, "symmetric force kernel");
        a.run_if = ctx->counters + C_SYMGATHER;
    }
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_TICKET, 0, sizeof(unsigned long long), ctx->stream));
    cudaEvent_t end = nullptr;
    timer_begin(ctx, 1, &end);
    const int mode = ctx->adaptive ? 1 : (a.axis ? 2 : 0);
    const size_t smf = ctx->tile_w == 32 ? force_smem<32>(ctx->adaptive) : force_smem<16>(ctx->adaptive);
#define SPH_LAUNCH_F(TWv, Mv) k_force<TWv, Mv><<<g, kPairThreads, smf, ctx->stream>>>(a)
    if (ctx->tile_w == 32) {
        if (mode == 1) SPH_LAUNCH_F(32, 1); else if (mode == 2) SPH_LAUNCH_F(32, 2); else SPH_LAUNCH_F(32, 0);
    } else {
        if (mode == 1) SPH_LAUNCH_F(16, 1); else if (mode == 2) SPH_LAUNCH_F(16, 2); else SPH_LAUNCH_F(16, 0);
    }
#undef SPH_LAUNCH_F
    timer_end(ctx, end);
    SPH_LAUNCH(ctx, "force kernel");
    if (sym) {
        const int64_t n = ctx->n;
        k_sym_reduce<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
            ctx->sym_slot, ctx->sym_vsig, n, ctx->counters + C_SYMGATHER, parts->ax, parts->ay, parts->az,
            parts->dudt, parts->vsig);
        SPH_LAUNCH(ctx, "symmetric force sums");
    }
    ctx->st.force_passes++;
    return SPH_OK;
}

// slot arrays of the symmetric force pass (allocated on first use, outside captures)
int ensure_sym(sph_ctx *ctx)
{
    const int64_t need = std::max<int64_t>(ctx->cap, 1);
    if (ctx->sym_cap >= need) return SPH_OK;
    cudaFree(ctx->sym_slot);
    cudaFree(ctx->sym_vsig);
    ctx->sym_slot = nullptr;
    ctx->sym_vsig = nullptr;
    ctx->sym_cap = 0;
    SPH_CUDA(ctx, cudaMalloc(&ctx->sym_slot, sizeof(float4) * kSymSlots * (size_t)need));
    SPH_CUDA(ctx, cudaMalloc(&ctx->sym_vsig, sizeof(unsigned) * (size_t)need));
    ctx->sym_cap = need;
    return SPH_OK;
}

// Open brackets: lower end 0, upper end kHUnbounded (bytes 0x7f: 3.39e38).
int reset_h_brackets(sph_ctx *ctx)
{
    const int64_t n = ctx->n;
    if (n <= 0) return SPH_OK;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->h_lo, 0, sizeof(float) * n, ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->h_hi, 0x7f, sizeof(float) * n, ctx->stream));
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
