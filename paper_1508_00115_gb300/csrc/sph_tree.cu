// sph_tree.cu -- adaptive cells (Theuns et al. 2015, Sec. 3.1: the dynamic range of
// h calls for an adaptive mesh of cells; the tree is cut off at cells of ~100
// particles, and neighbouring cells are themselves found with a tree).
//
// Top-level cells are the uniform per-box grid (side >= cell_factor * max h), so a
// particle's neighbours always lie in the 27 top cells around it.  Inside each top
// cell particles are ordered by a 3 x 14-bit Morton code; every octree node is then
// a contiguous range of the sorted particles.  Nodes are refined top-down, one level
// per step, while they hold more than leaf_max particles (a parameter, 64 by default).
// Unlike the paper's cells, a leaf may be smaller than the h of its particles: its
// neighbours need not lie in the adjacent leaves, because every leaf carries an
// explicit list of the leaves within reach.  For every leaf the list
// holds every leaf met in the 27 surrounding top-cell subtrees whose bounding box
// comes within reach -- max of the two leaves' largest h, grown by kTreeReach so
// that h may grow during the density iteration -- and every entry carries the FP32
// offset between the two leaf centres (computed in FP64, periodic image included).
// Particle positions are stored relative to their leaf's centre, so FP32 keeps
// ~2^-24 of a leaf side even where h is 10^-3 of the top cell.
#include <math.h>

#include <string.h>

#include <algorithm>
#include <vector>

#include "sph_internal.cuh"

namespace sph {

constexpr int kMortonBits = 14;       // per axis, inside a top cell
constexpr int kBoundsW = 10;          // words per frontier node: 9 octant bounds + child starts
constexpr int kMortonShift = 3 * kMortonBits;

__device__ __forceinline__ uint64_t spread3(uint32_t v)  // 14 bits -> every third bit
{
    uint64_t x = v & 0x3fffu;
    x = (x | (x << 16)) & 0x0000ff0000ffull;
    x = (x | (x << 8)) & 0x00f00f00f00f00full;
    x = (x | (x << 4)) & 0x0c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x249249249249249ull;
    return x;
}
__device__ __forceinline__ uint32_t compact3(uint64_t x)  // inverse of spread3
{
    x &= 0x249249249249249ull;
    x = (x ^ (x >> 2)) & 0x0c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x00f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x3fffull;
    return (uint32_t)x;
}

__device__ __forceinline__ double twrap(double v, double box)
{
    if (v >= 0.0 && v < box) return v;
    double w = __dsub_rn(v, __dmul_rn(box, floor(__ddiv_rn(v, box))));
    if (w < 0.0) w = __dadd_rn(w, box);
    if (w >= box) w = __dsub_rn(w, box);
    if (w < 0.0 || w >= box) w = 0.0;
    return w;
}

__device__ __forceinline__ int tbox_of_slot(int p, const BoxDev *__restrict__ bx, int nb)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bx[mid].p_begin <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int tbox_of_cell(int c, const BoxDev *__restrict__ bx, int nb)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bx[mid].cell_off <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int tcell_of(double v, double s, int nc)
{
    int c = (int)floor(__dmul_rn(v, s));
    return c < 0 ? 0 : (c > nc - 1 ? nc - 1 : c);
}

// key = top cell << 42 | Morton code of the position inside the top cell
__global__ void k_tree_keys(double *x, double *y, double *z, int n, int nb, double box,
                            const BoxDev *__restrict__ bxs, uint64_t *__restrict__ keys)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const BoxDev g = bxs[nb == 1 ? 0 : tbox_of_slot(i, bxs, nb)];
    const double px = twrap(x[i], box), py = twrap(y[i], box), pz = twrap(z[i], box);
    x[i] = px;
    y[i] = py;
    z[i] = pz;
    const int ix = tcell_of(px, g.s, g.nc), iy = tcell_of(py, g.s, g.nc), iz = tcell_of(pz, g.s, g.nc);
    const double sub = (double)(1 << kMortonBits) * g.s;  // sub-cells per unit length
    auto subi = [&](double p, int c) {
        int v = (int)floor((p - (double)c * g.L64) * sub);
        return (uint32_t)(v < 0 ? 0 : (v > (1 << kMortonBits) - 1 ? (1 << kMortonBits) - 1 : v));
    };
    const uint64_t m = spread3(subi(px, ix)) | (spread3(subi(py, iy)) << 1) | (spread3(subi(pz, iz)) << 2);
    const uint64_t top = (uint64_t)(g.cell_off + (iz * g.nc + iy) * g.nc + ix);
    keys[i] = (top << kMortonShift) | m;
}

__global__ void k_top_start(const uint64_t *__restrict__ k, int n, int64_t ntop, int *__restrict__ cs)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ntop) return;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int64_t)(k[mid] >> kMortonShift) < c) lo = mid + 1;
        else hi = mid;
    }
    cs[c] = lo;
}

__global__ void k_nonempty(const int *__restrict__ cs, int64_t ntop, uint32_t *__restrict__ f)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ntop) f[c] = cs[c + 1] > cs[c] ? 1u : 0u;
}

// roots: one node per non-empty top cell, numbered in cell order
__global__ void k_roots(const int *__restrict__ cs, int64_t ntop, const uint32_t *__restrict__ off,
                        TreeNode *__restrict__ nodes, int *__restrict__ top_node, int *__restrict__ front)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ntop) return;
    if (cs[c + 1] == cs[c]) {
        top_node[c] = -1;
        return;
    }
    const int id = (int)off[c];
    TreeNode t;
    t.lo = cs[c];
    t.hi = cs[c + 1];
    t.child = -1;
    t.nchild = 0;
    t.top = (int)c;
    t.level = 0;
    t.prefix = 0;
    t.parent = -1;
    nodes[id] = t;
    top_node[c] = id;
    front[id] = id;
}

// Refinement decision of every frontier node (one thread per node): a node is split
// while it holds more than leaf_max particles (down to the Morton resolution); its
// non-empty octants' particle ranges come from binary searches on the next Morton
// digit.  Octants are joined along the Morton order into halves (4 octants, a slab)
// or quarters (2 octants, a bar) of the node while the part holds at most leaf_max
// particles (a leaf spanning several octants keeps its parent's cube), so that a node
// just above leaf_max gives two to four full leaves instead of up to eight sparse
// ones.  Word 9 of a node's bounds marks the octants that start a child.
// (Sizes: the host count, or -- builds inside captured steps -- the level's node range
// lvl[0] .. lvl[1] on the device, the kernel then covering cap entries and writing
// zero counts past the frontier.)
__global__ void k_node_split(const int *__restrict__ front, int nfront_h, const int *__restrict__ lvl, int cap,
                             const TreeNode *__restrict__ nodes, const uint64_t *__restrict__ keys, int leaf_max,
                             int *__restrict__ bounds, uint32_t *__restrict__ nkids)
{
    const int nfront = lvl ? lvl[1] - lvl[0] : nfront_h;
    const int end = lvl ? cap : nfront;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < end; w += gridDim.x * blockDim.x) {
        if (w >= nfront) {
            nkids[w] = 0u;
            continue;
        }
        const TreeNode t = nodes[front[w]];
        const bool split = (t.hi - t.lo) > leaf_max && t.level < kMortonBits;
        int cnt = 0;
        if (split) {
            // child boundaries: first slot whose next Morton digit is >= k (k = 1..7)
            const int sh = 3 * (kMortonBits - 1 - t.level);
            int b[9];
            b[0] = t.lo;
            b[8] = t.hi;
            for (int k = 1; k < 8; ++k) {
                int lo = b[k - 1], hi = t.hi;  // digits are sorted: search from the previous bound
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if ((int)((keys[mid] >> sh) & 7u) < k) lo = mid + 1;
                    else hi = mid;
                }
                b[k] = lo;
            }
            // children: a half of the cube (octants 4h .. 4h + 3) if it holds at most
            // leaf_max particles, else its quarters (octant pairs) that do, else octants
            int starts = 0;
            auto first_in = [&](int k0, int k1) {  // first non-empty octant of [k0, k1)
                int k = k0;
                while (k < k1 && b[k + 1] == b[k]) ++k;
                return k;
            };
            for (int q0 = 0; q0 < 8; q0 += 4) {
                const int qn = b[q0 + 4] - b[q0];
                if (qn <= leaf_max) {
                    if (qn > 0) starts |= 1 << first_in(q0, q0 + 4);
                    continue;
                }
                for (int p0 = q0; p0 < q0 + 4; p0 += 2) {
                    const int pn = b[p0 + 2] - b[p0];
                    if (pn <= leaf_max) {
                        if (pn > 0) starts |= 1 << first_in(p0, p0 + 2);
                        continue;
                    }
                    for (int k = p0; k < p0 + 2; ++k)
                        if (b[k + 1] > b[k]) starts |= 1 << k;
                }
            }
            cnt = __popc(starts);
            for (int k = 0; k < 9; ++k) bounds[kBoundsW * w + k] = b[k];
            bounds[kBoundsW * w + 9] = starts;
        }
        nkids[w] = (uint32_t)cnt;
    }
}

// Largest h and bounding box (relative to the top-cell centre) of every leaf, one warp
// per leaf node; the box is widened by one FP32 ulp of the top cell so that rounding of
// the positions never shrinks it.
__global__ void k_leaf_box(TreeNode *__restrict__ nodes, int n_nodes_h, const int *__restrict__ np,
                           const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                           const float *__restrict__ h, const BoxDev *__restrict__ bxs, int nb)
{
    const int n_nodes = np ? *np : n_nodes_h;
    const int lane = threadIdx.x & 31;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_nodes; w += (gridDim.x * blockDim.x) >> 5) {
        TreeNode t = nodes[w];
        if (t.child >= 0) continue;  // warp-uniform
        const BoxDev g = bxs[nb == 1 ? 0 : tbox_of_cell(t.top, bxs, nb)];
        const int loc = t.top - g.cell_off;
        const double cx = ((double)(loc % g.nc) + 0.5) * g.L64, cy = ((double)((loc / g.nc) % g.nc) + 0.5) * g.L64,
                     cz = ((double)(loc / (g.nc * g.nc)) + 0.5) * g.L64;
        float hm = 0.f, x0 = 1e30f, y0 = 1e30f, z0 = 1e30f, x1 = -1e30f, y1 = -1e30f, z1 = -1e30f;
        for (int p = t.lo + lane; p < t.hi; p += 32) {
            hm = fmaxf(hm, h[p]);
            const float px = (float)(x[p] - cx), py = (float)(y[p] - cy), pz = (float)(z[p] - cz);
            x0 = fminf(x0, px);
            x1 = fmaxf(x1, px);
            y0 = fminf(y0, py);
            y1 = fmaxf(y1, py);
            z0 = fminf(z0, pz);
            z1 = fmaxf(z1, pz);
        }
    #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            hm = fmaxf(hm, __shfl_xor_sync(kFull, hm, o));
            x0 = fminf(x0, __shfl_xor_sync(kFull, x0, o));
            x1 = fmaxf(x1, __shfl_xor_sync(kFull, x1, o));
            y0 = fminf(y0, __shfl_xor_sync(kFull, y0, o));
            y1 = fmaxf(y1, __shfl_xor_sync(kFull, y1, o));
            z0 = fminf(z0, __shfl_xor_sync(kFull, z0, o));
            z1 = fmaxf(z1, __shfl_xor_sync(kFull, z1, o));
        }
        if (lane == 0) {
            const float pad = g.L32 * 1.2e-7f;
            t.hmax = hm;
            t.bx0 = x0 - pad;
            t.by0 = y0 - pad;
            t.bz0 = z0 - pad;
            t.bx1 = x1 + pad;
            t.by1 = y1 + pad;
            t.bz1 = z1 + pad;
            nodes[w] = t;
        }
    }
}

// internal nodes of one level [first, last): union of their children's boxes and max h
__global__ void k_merge_children(TreeNode *__restrict__ nodes, int first_h, int last_h, const int *__restrict__ lb,
                                 int level)
{
    const int first = lb ? lb[level] : first_h, last = lb ? lb[level + 1] : last_h;
    for (int id = first + blockIdx.x * blockDim.x + threadIdx.x; id < last; id += gridDim.x * blockDim.x) {
        TreeNode t = nodes[id];
        if (t.child < 0) continue;
        float hm = 0.f, x0 = 1e30f, y0 = 1e30f, z0 = 1e30f, x1 = -1e30f, y1 = -1e30f, z1 = -1e30f;
        for (int c = t.child; c < t.child + t.nchild; ++c) {
            const TreeNode k = nodes[c];
            hm = fmaxf(hm, k.hmax);
            x0 = fminf(x0, k.bx0);
            y0 = fminf(y0, k.by0);
            z0 = fminf(z0, k.bz0);
            x1 = fmaxf(x1, k.bx1);
            y1 = fmaxf(y1, k.by1);
            z1 = fmaxf(z1, k.bz1);
        }
        t.hmax = hm;
        t.bx0 = x0;
        t.by0 = y0;
        t.bz0 = z0;
        t.bx1 = x1;
        t.by1 = y1;
        t.bz1 = z1;
        nodes[id] = t;
    }
}

// children of the refined frontier nodes, numbered in frontier order (deterministic)
// (device sizes: the frontier is level lvl[0] .. lvl[1], its children lvl[1] .. lvl[2];
// an empty child range -- nothing refined, or no room for the children -- makes none)
__global__ void k_make_children(const int *__restrict__ front, int nfront_h, TreeNode *__restrict__ nodes,
                                const int *__restrict__ bounds, const uint32_t *__restrict__ off, uint32_t total_h,
                                int base_h, const int *__restrict__ lvl, int *__restrict__ next)
{
    const int nfront = lvl ? lvl[1] - lvl[0] : nfront_h;
    const uint32_t total = lvl ? (uint32_t)(lvl[2] - lvl[1]) : total_h;
    const int base = lvl ? lvl[1] : base_h;
    if (total == 0u) return;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nfront; f += gridDim.x * blockDim.x) {
        const uint32_t first = off[f], end = f + 1 < nfront ? off[f + 1] : total;
        if (end == first) continue;  // not refined: a leaf
        const int id = front[f];
        const int *b = bounds + kBoundsW * f;
        const int starts = b[9];
        TreeNode &t = nodes[id];
        int c = 0;
        for (int k = 0; k < 8; ++k) {
            if (!((starts >> k) & 1)) continue;
            // the child runs from octant k up to the next starting octant
            int e = k + 1;
            int octants = 1;
            while (e < 8 && !((starts >> e) & 1)) {
                octants += b[e + 1] > b[e] ? 1 : 0;
                ++e;
            }
            TreeNode ch;
            ch.lo = b[k];
            ch.hi = b[e];
            ch.child = -1;
            ch.nchild = 0;
            ch.top = t.top;
            if (octants == 1) {  // one octant: its own cube
                ch.level = t.level + 1;
                ch.prefix = (t.prefix << 3) | (uint64_t)k;
            } else {  // joined octants: the parent's cube
                ch.level = t.level;
                ch.prefix = t.prefix;
            }
            ch.parent = id;
            const int cid = base + (int)first + c;
            nodes[cid] = ch;
            next[first + c] = cid;
            ++c;
        }
        t.child = base + (int)first;
        t.nchild = c;
    }
}

// Initial h from the tree: for every leaf, the smallest node around it (itself or an
// ancestor) that holds at least min_count particles gives a number density n =
// count / side^3, and h = (3 N_ngb / (4 pi n))^(1/3) -- the h at which a uniform
// medium of that density meets the criterion -- is written to the leaf's particles.
__global__ void k_h_guess(const TreeNode *__restrict__ nodes, int n_nodes, const BoxDev *__restrict__ bxs, int nb,
                          int min_count, float n_ngb, double box, float *__restrict__ h)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_nodes) return;
    const TreeNode t = nodes[id];
    if (t.child >= 0) return;
    TreeNode A = t;
    while (A.hi - A.lo < min_count && A.parent >= 0) A = nodes[A.parent];
    const BoxDev g = bxs[nb == 1 ? 0 : tbox_of_cell(A.top, bxs, nb)];
    const double side = ldexp(g.L64, -A.level);
    const double dens = (double)(A.hi - A.lo) / (side * side * side);
    double h0 = cbrt(3.0 * (double)n_ngb / (4.0 * 3.14159265358979323846 * dens));
    h0 = fmin(h0, 0.45 * box);
    for (int p = t.lo; p < t.hi; ++p) h[p] = (float)h0;
}

__global__ void k_sum_u32(const uint32_t *__restrict__ v, int n, unsigned long long *__restrict__ out)
{
    unsigned long long s = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// flags the first slot of every leaf (leaves partition the particles)
__global__ void k_leaf_marks(const TreeNode *__restrict__ nodes, int n_nodes_h, const int *__restrict__ np,
                             uint32_t *__restrict__ flag, int *__restrict__ node_at)
{
    const int n_nodes = np ? *np : n_nodes_h;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < n_nodes; id += gridDim.x * blockDim.x) {
        const TreeNode t = nodes[id];
        if (t.child >= 0) continue;
        flag[t.lo] = 1u;
        node_at[t.lo] = id;
    }
}

// leaves in particle (Morton) order: leaf id of slot p = (number of leaf starts <= p) - 1
__global__ void k_leaves(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ excl, int n,
                         const int *__restrict__ node_at, const TreeNode *__restrict__ nodes,
                         const BoxDev *__restrict__ bxs, int nb, int *__restrict__ leaf_of, int *__restrict__ leaf_node,
                         int *__restrict__ node_leaf, int2 *__restrict__ leaf_rng, double *__restrict__ leaf_cen,
                         float *__restrict__ leaf_h, float4 *__restrict__ leaf_lo, float4 *__restrict__ leaf_hi)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int lid = (int)excl[p] + (int)flag[p] - 1;
    leaf_of[p] = lid;
    if (!flag[p]) return;
    const int id = node_at[p];
    const TreeNode t = nodes[id];
    leaf_node[lid] = id;
    node_leaf[id] = lid;
    leaf_rng[lid] = make_int2(t.lo, t.hi);
    leaf_h[lid] = t.hmax;
    const BoxDev g = bxs[nb == 1 ? 0 : tbox_of_cell(t.top, bxs, nb)];
    const int loc = t.top - g.cell_off;
    const int ix = loc % g.nc, iy = (loc / g.nc) % g.nc, iz = loc / (g.nc * g.nc);
    // the leaf's cube: Morton prefix at its level gives its sub-cell coordinates
    const uint64_t pre = t.prefix << (3 * (kMortonBits - t.level));
    const double side = g.L64 / (double)(1 << t.level);
    const double fine = g.L64 / (double)(1 << kMortonBits);
    const double sx = (double)compact3(pre) * fine, sy = (double)compact3(pre >> 1) * fine,
                 sz = (double)compact3(pre >> 2) * fine;
    const double lx = (double)ix * g.L64 + sx + 0.5 * side, ly = (double)iy * g.L64 + sy + 0.5 * side,
                 lz = (double)iz * g.L64 + sz + 0.5 * side;
    leaf_cen[3 * lid + 0] = lx;
    leaf_cen[3 * lid + 1] = ly;
    leaf_cen[3 * lid + 2] = lz;
    // the node's box (relative to the top-cell centre) moved to the leaf centre, grown
    // by two more FP32 ulps of the top cell for the rounding of the move
    const float ox = (float)(((double)ix + 0.5) * g.L64 - lx), oy = (float)(((double)iy + 0.5) * g.L64 - ly),
                oz = (float)(((double)iz + 0.5) * g.L64 - lz);
    const float pad = g.L32 * 2.4e-7f;
    leaf_lo[lid] = make_float4(t.bx0 + ox - pad, t.by0 + oy - pad, t.bz0 + oz - pad, t.hmax);
    leaf_hi[lid] = make_float4(t.bx1 + ox + pad, t.by1 + oy + pad, t.bz1 + oz + pad, 0.f);
}

// positions relative to the leaf centre
__global__ void k_leaf_pos(const int *__restrict__ leaf_of, const double *__restrict__ leaf_cen,
                           const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                           const float *__restrict__ h, int n, float4 *__restrict__ pos4)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int l = leaf_of[p];
    pos4[p] = make_float4((float)(x[p] - leaf_cen[3 * l]), (float)(y[p] - leaf_cen[3 * l + 1]),
                          (float)(z[p] - leaf_cen[3 * l + 2]), h[p]);
}

// Targets of every leaf in ascending h (ties by slot), so that a tile holds targets of
// similar h: its reach -- and with it the candidates of every target -- is not set by
// one large-h particle among small ones.  One warp per leaf: a bitonic sort in shared
// memory of the keys (bits of h, which order as h does for h >= 0; slot within the leaf),
// padded to a power of two with keys above every real one.  Then each run of two tiles'
// worth (2 tw targets of similar h) is sorted along the longest side of its bounding box
// (the coordinate's FP32 bits: positions lie in [0, box)), so that each of its two tiles
// covers half of it: 2-3 % fewer pair-pass time on the uneven boxes (a second, finer
// split of runs of four tiles was slower).  Leaves above kSortMax particles keep their
// order.
constexpr int kSortMax = 256;
constexpr int kSortWarps = 4;
__global__ void __launch_bounds__(32 * kSortWarps) k_leaf_hsort(const int2 *__restrict__ rng, int nl_h,
                                                                const int *__restrict__ nlp,
                                                                const float *__restrict__ h, int *__restrict__ tord,
                                                                const double *__restrict__ x,
                                                                const double *__restrict__ y,
                                                                const double *__restrict__ z, int tw)
{
    __shared__ unsigned long long sk[kSortWarps][kSortMax];
    __shared__ unsigned long long sg[kSortWarps][64];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned long long *k2 = sk[wib];
    unsigned long long *g2 = sg[wib];
    const int nl = nlp ? *nlp : nl_h;
    for (int l = blockIdx.x * kSortWarps + wib; l < nl; l += gridDim.x * kSortWarps) {  // warp-uniform
        const int lo = rng[l].x, c = rng[l].y - lo;
        if (c > kSortMax) {
            for (int k = lane; k < c; k += 32) tord[lo + k] = lo + k;
            continue;
        }
        int P = 1;
        while (P < c) P <<= 1;
        __syncwarp();
        for (int k = lane; k < P; k += 32)
            k2[k] = k < c ? ((unsigned long long)__float_as_uint(h[lo + k]) << 32) | (unsigned)k : ~0ull;
        __syncwarp();
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = lane; t < (P >> 1); t += 32) {
                    const int i = 2 * t - (t & (stride - 1));  // lower element of the t-th pair
                    const unsigned long long a = k2[i], b = k2[i + stride];
                    if ((a > b) == ((i & size) == 0)) {  // ascending where (i & size) == 0
                        k2[i] = b;
                        k2[i + stride] = a;
                    }
                }
                __syncwarp();
            }
        }
        // groups of two tiles of similar h: each split in two halves along the longest
        // side of the group's box, so that each tile covers half of it
        const int gs = 2 * tw;
        for (int g0 = 0; g0 < c; g0 += gs) {
            const int gc = min(gs, c - g0);
            if (gc <= tw) break;
            float mn0 = 3e38f, mn1 = 3e38f, mn2 = 3e38f, mx0 = -3e38f, mx1 = -3e38f, mx2 = -3e38f;
            for (int k = lane; k < gc; k += 32) {
                const int s_ = lo + (int)(unsigned)(k2[g0 + k] & 0xffffffffull);
                const float px = (float)x[s_], py = (float)y[s_], pz = (float)z[s_];
                mn0 = fminf(mn0, px);
                mx0 = fmaxf(mx0, px);
                mn1 = fminf(mn1, py);
                mx1 = fmaxf(mx1, py);
                mn2 = fminf(mn2, pz);
                mx2 = fmaxf(mx2, pz);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn0 = fminf(mn0, __shfl_xor_sync(kFull, mn0, o));
                mx0 = fmaxf(mx0, __shfl_xor_sync(kFull, mx0, o));
                mn1 = fminf(mn1, __shfl_xor_sync(kFull, mn1, o));
                mx1 = fmaxf(mx1, __shfl_xor_sync(kFull, mx1, o));
                mn2 = fminf(mn2, __shfl_xor_sync(kFull, mn2, o));
                mx2 = fmaxf(mx2, __shfl_xor_sync(kFull, mx2, o));
            }
            const int ax = (mx0 - mn0 >= mx1 - mn1 && mx0 - mn0 >= mx2 - mn2) ? 0 : (mx1 - mn1 >= mx2 - mn2 ? 1 : 2);
            int P2 = 1;
            while (P2 < gc) P2 <<= 1;
            __syncwarp();
            for (int k = lane; k < P2; k += 32) {
                unsigned long long key = ~0ull;
                if (k < gc) {
                    const unsigned s_ = (unsigned)(k2[g0 + k] & 0xffffffffull);
                    const double v = ax == 0 ? x[lo + s_] : (ax == 1 ? y[lo + s_] : z[lo + s_]);
                    key = ((unsigned long long)__float_as_uint((float)v) << 32) | s_;
                }
                g2[k] = key;
            }
            __syncwarp();
            for (int size = 2; size <= P2; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int t = lane; t < (P2 >> 1); t += 32) {
                        const int i = 2 * t - (t & (stride - 1));
                        const unsigned long long a = g2[i], b = g2[i + stride];
                        if ((a > b) == ((i & size) == 0)) {
                            g2[i] = b;
                            g2[i + stride] = a;
                        }
                    }
                    __syncwarp();
                }
            }
            for (int k = lane; k < gc; k += 32) k2[g0 + k] = g2[k];
            __syncwarp();
        }
        for (int k = lane; k < c; k += 32) tord[lo + k] = lo + (int)(unsigned)(k2[k] & 0xffffffffull);
    }
}

// (device count: entries from nl up to cap are set to zero for the prefix sum)
__global__ void k_leaf_tiles_n(const int2 *__restrict__ rng, int nl_h, const int *__restrict__ nlp, int cap, int tw,
                               uint32_t *__restrict__ nt)
{
    const int nl = nlp ? *nlp : nl_h;
    const int end = nlp ? cap : nl;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < end; l += gridDim.x * blockDim.x)
        nt[l] = l < nl ? (uint32_t)((rng[l].y - rng[l].x + tw - 1) / tw) : 0u;
}

// tile = {leaf, first slot, count, box}
__global__ void k_leaf_tiles(const int2 *__restrict__ rng, const int *__restrict__ leaf_node,
                             const TreeNode *__restrict__ nodes, int nl_h, const int *__restrict__ nlp, int tw,
                             const uint32_t *__restrict__ off, const BoxDev *__restrict__ bxs, int nb,
                             int4 *__restrict__ tiles, int *__restrict__ ntiles)
{
    const int nl = nlp ? *nlp : nl_h;
    if (nl == 0 && blockIdx.x == 0 && threadIdx.x == 0) *ntiles = 0;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x) {
        const int s = rng[l].x, cnt = rng[l].y - s;
        const int box = nb == 1 ? 0 : tbox_of_cell(nodes[leaf_node[l]].top, bxs, nb);
        int k = 0;
        for (int b = 0; b < cnt; b += tw, ++k) tiles[off[l] + k] = make_int4(l, s + b, min(tw, cnt - b), box);
        if (l == nl - 1) *ntiles = (int)(off[l] + k);
    }
}

// Later density passes of adaptive cells: the still-active targets of every leaf,
// packed to the front of its range in act_ord (in tord order, one warp per leaf),
// and their tile counts; a tile then holds only targets that need the pass.
// (*unconv, when given: the targets the last pass left active; none -- a captured
// step's passes after convergence -- leaves nothing to do, and the tile kernel below
// runs no tile)
__global__ void k_leaf_active(const int2 *__restrict__ rng, int nl_h, const int *__restrict__ nlp, int cap,
                              const int *__restrict__ tord, const uint8_t *__restrict__ active, int tw,
                              const unsigned long long *__restrict__ unconv, int *__restrict__ act_ord,
                              uint32_t *__restrict__ ntiles_leaf, int *__restrict__ nact_leaf)
{
    if (unconv && *unconv == 0ull) return;
    const int lane = threadIdx.x & 31;
    const int nl = nlp ? *nlp : nl_h;
    for (int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; l < nl; l += (gridDim.x * blockDim.x) >> 5) {
        const int lo = rng[l].x, hi = rng[l].y;  // warp-uniform
        int c = 0;
        for (int q0 = lo; q0 < hi; q0 += 32) {
            const int q = q0 + lane;
            const int slot = q < hi ? tord[q] : 0;
            const bool a = q < hi && active[slot] != 0;
            const unsigned b = __ballot_sync(kFull, a);
            if (a) act_ord[lo + c + __popc(b & ((1u << lane) - 1u))] = slot;
            c += __popc(b);
        }
        if (lane == 0) {
            ntiles_leaf[l] = (uint32_t)((c + tw - 1) / tw);
            nact_leaf[l] = c;
        }
    }
    // device count: zero counts past the last leaf, up to cap, for the prefix sum
    if (nlp)
        for (int l = nl + blockIdx.x * blockDim.x + threadIdx.x; l < cap; l += gridDim.x * blockDim.x)
            ntiles_leaf[l] = 0u;
}

__global__ void k_leaf_active_tiles(const int2 *__restrict__ rng, const int *__restrict__ leaf_node,
                                    const TreeNode *__restrict__ nodes, int nl_h, const int *__restrict__ nlp, int tw,
                                    const uint32_t *__restrict__ off, const int *__restrict__ nact_leaf,
                                    const BoxDev *__restrict__ bxs, int nb, const int *__restrict__ err,
                                    const unsigned long long *__restrict__ unconv, int4 *__restrict__ tiles,
                                    int *__restrict__ ntiles)
{
    if ((err && *err) || (unconv && *unconv == 0ull)) {  // lists that did not fit, or nothing active
        if (blockIdx.x == 0 && threadIdx.x == 0) *ntiles = 0;
        return;
    }
    const int nl = nlp ? *nlp : nl_h;
    if (nl == 0 && blockIdx.x == 0 && threadIdx.x == 0) *ntiles = 0;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x) {
        const int s = rng[l].x, cnt = nact_leaf[l];
        const int box = nb == 1 ? 0 : tbox_of_cell(nodes[leaf_node[l]].top, bxs, nb);
        int k = 0;
        for (int b = 0; b < cnt; b += tw, ++k) tiles[off[l] + k] = make_int4(l, s + b, min(tw, cnt - b), box);
        if (l == nl - 1) *ntiles = (int)(off[l] + k);
    }
}

// Neighbour leaves of leaf `l`: walk the subtrees of the 27 top cells around its own,
// keeping nodes whose bounding box is within reach.  COUNT: only count; else write
// {offset between the leaf centres (FP32), neighbour leaf} from out[0].
template <bool COUNT>
__device__ int leaf_pairs(int l, const int *__restrict__ leaf_node, const TreeNode *__restrict__ nodes,
                          const int *__restrict__ top_node, const int *__restrict__ node_leaf,
                          const double *__restrict__ leaf_cen, const BoxDev *__restrict__ bxs, int nb, double box,
                          float4 *__restrict__ out, float *__restrict__ scale_out)
{
    const TreeNode A = nodes[leaf_node[l]];
    const BoxDev g = bxs[nb == 1 ? 0 : tbox_of_cell(A.top, bxs, nb)];
    const int nc = g.nc, loc = A.top - g.cell_off;
    const int ix = loc % nc, iy = (loc / nc) % nc, iz = loc / (nc * nc);
    const float hA = A.hmax * kTreeReach;
    // FP32 rounding of the boxes and offsets (a few ulps of the top cell) is covered
    // by a slack added to every reach
    const float slack = 4.8e-7f * g.L32;
    const double cAx = leaf_cen[3 * l], cAy = leaf_cen[3 * l + 1], cAz = leaf_cen[3 * l + 2];
    const double sideA = ldexp(g.L64, -A.level);
    double scale = sideA;
    int stack[8 * (kMortonBits + 1)];
    int cnt = 0;
    for (int o = 0; o < 27; ++o) {
        const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
        int jx = ix + ox, jy = iy + oy, jz = iz + oz;
        // periodic image: k_ * box added to the neighbour's absolute positions
        const int kx = jx < 0 ? -1 : (jx >= nc ? 1 : 0), ky = jy < 0 ? -1 : (jy >= nc ? 1 : 0),
                  kz = jz < 0 ? -1 : (jz >= nc ? 1 : 0);
        jx -= kx * nc;
        jy -= ky * nc;
        jz -= kz * nc;
        const int root = top_node[g.cell_off + (jz * nc + jy) * nc + jx];
        if (root < 0) continue;
        // offset of the neighbour top cell's centre relative to A's (FP32, multiples of L)
        const float dx = (float)ox * g.L32, dy = (float)oy * g.L32, dz = (float)oz * g.L32;
        int sp = 0;
        stack[sp++] = root;
        while (sp > 0) {
            const int id = stack[--sp];
            const TreeNode N = nodes[id];
            const float gx = fmaxf(fmaxf(N.bx0 + dx - A.bx1, A.bx0 - (N.bx1 + dx)), 0.f);
            const float gy = fmaxf(fmaxf(N.by0 + dy - A.by1, A.by0 - (N.by1 + dy)), 0.f);
            const float gz = fmaxf(fmaxf(N.bz0 + dz - A.bz1, A.bz0 - (N.bz1 + dz)), 0.f);
            const float reach = fmaxf(hA, N.hmax * kTreeReach) * (1.f + 1e-5f) + slack;
            if (gx * gx + gy * gy + gz * gz >= reach * reach) continue;
            if (N.child < 0) {
                if (!COUNT) {
                    const int b = node_leaf[id];
                    const double sx = leaf_cen[3 * b] + kx * box - cAx, sy = leaf_cen[3 * b + 1] + ky * box - cAy,
                                 sz = leaf_cen[3 * b + 2] + kz * box - cAz;
                    out[cnt] = make_float4((float)sx, (float)sy, (float)sz, __int_as_float(b));
                    // coordinates met in this pair's FP32 arithmetic are below
                    // |p_i| + |p_j| + |shift| <= (sides of both leaves + shift)
                    const double m = fmax(fabs(sx), fmax(fabs(sy), fabs(sz)));
                    scale = fmax(scale, 0.5 * (sideA + ldexp(g.L64, -N.level) + m));
                }
                ++cnt;
            } else {
                for (int c = N.nchild - 1; c >= 0; --c) stack[sp++] = N.child + c;
            }
        }
    }
    if (!COUNT) *scale_out = (float)scale;
    return cnt;
}

// (device count: runs only when *ovf reports an overflowed warp walk)
__global__ void k_pairs_count(int nl_h, const int *__restrict__ nlp, const unsigned long long *__restrict__ ovf,
                              const int *__restrict__ leaf_node, const TreeNode *__restrict__ nodes,
                              const int *__restrict__ top_node, const int *__restrict__ node_leaf,
                              const double *__restrict__ leaf_cen, const BoxDev *__restrict__ bxs, int nb, double box,
                              uint32_t *__restrict__ cnt)
{
    if (ovf && *ovf == 0ull) return;
    const int nl = nlp ? *nlp : nl_h;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x)
        cnt[l] = (uint32_t)leaf_pairs<true>(l, leaf_node, nodes, top_node, node_leaf, leaf_cen, bxs, nb, box, nullptr,
                                            nullptr);
}

// (device count: runs only when *ovf reports an overflowed warp walk and *err holds
// no list-capacity error)
__global__ void k_pairs_fill(int nl_h, const int *__restrict__ nlp, const unsigned long long *__restrict__ ovf,
                             const int *__restrict__ err, const int *__restrict__ leaf_node,
                             const TreeNode *__restrict__ nodes, const int *__restrict__ top_node,
                             const int *__restrict__ node_leaf, const double *__restrict__ leaf_cen,
                             const BoxDev *__restrict__ bxs, int nb, double box, const uint32_t *__restrict__ off,
                             float4 *__restrict__ list, float *__restrict__ scale)
{
    if (ovf && *ovf == 0ull) return;
    if (err && *err) return;
    const int nl = nlp ? *nlp : nl_h;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x)
        leaf_pairs<false>(l, leaf_node, nodes, top_node, node_leaf, leaf_cen, bxs, nb, box, list + off[l], scale + l);
}

// The same lists built by one warp per leaf: the warp pops up to 32 (node, image)
// items of a shared-memory stack per round, tests them in parallel, appends the
// leaves within reach (lane order) and pushes the children of the other nodes within
// reach.  Entry order is fixed by the algorithm, so the counting and the writing
// pass agree.  A walk whose stack would overflow sets *overflow and the caller
// falls back to the one-thread walk above.
constexpr int kWalkWarps = 2;
constexpr int kWalkCap = 2048;  // stack items per warp (16 KB)

struct WalkArgs {
    int nl;
    const int *__restrict__ nlp;                     // device leaf count (replaces nl when set)
    const unsigned long long *__restrict__ skip_ovf;  // fill: skip when a counting walk overflowed
    const int *__restrict__ err;                      // fill: skip when the lists did not fit
    const int *__restrict__ leaf_node;
    const TreeNode *__restrict__ nodes;
    const int *__restrict__ top_node;
    const int *__restrict__ node_leaf;
    const double *__restrict__ leaf_cen;
    const BoxDev *__restrict__ bxs;
    int nb;
    double box;
    const uint32_t *__restrict__ off;  // fill: first entry of every leaf
    float4 *__restrict__ list;         // fill: entries
    float *__restrict__ scale;         // fill: coordinate scale per leaf
    uint32_t *__restrict__ cnt;        // count: entries per leaf
    unsigned long long *overflow;
    unsigned *ticket;  // device-sized builds: leaves beyond the first of each warp, handed out
};

template <bool COUNT>
__device__ void walk_leaf(const WalkArgs &a, int l, int2 *st)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const TreeNode A = a.nodes[a.leaf_node[l]];
    const BoxDev g = a.bxs[a.nb == 1 ? 0 : tbox_of_cell(A.top, a.bxs, a.nb)];
    const int nc = g.nc, loc = A.top - g.cell_off;
    const int ix = loc % nc, iy = (loc / nc) % nc, iz = loc / (nc * nc);
    const float hA = A.hmax * kTreeReach;
    const float slack = 4.8e-7f * g.L32;
    const float sideA = ldexpf(g.L32, -A.level);
    // roots: the non-empty top cells around A's, item = {root node, image index}
    int sp;
    {
        int root = -1;
        if (lane < 27) {
            int jx = ix + lane % 3 - 1, jy = iy + (lane / 3) % 3 - 1, jz = iz + lane / 9 - 1;
            jx = jx < 0 ? jx + nc : (jx >= nc ? jx - nc : jx);
            jy = jy < 0 ? jy + nc : (jy >= nc ? jy - nc : jy);
            jz = jz < 0 ? jz + nc : (jz >= nc ? jz - nc : jz);
            root = a.top_node[g.cell_off + (jz * nc + jy) * nc + jx];
        }
        const unsigned b = __ballot_sync(kFull, root >= 0);
        if (root >= 0) st[__popc(b & lt)] = make_int2(root, lane);
        sp = __popc(b);
    }
    __syncwarp();
    uint32_t cnt = 0;
    const uint32_t base = COUNT ? 0u : a.off[l];
    float sc = sideA;
    double cAx = 0.0, cAy = 0.0, cAz = 0.0;
    if (!COUNT) {
        cAx = a.leaf_cen[3 * l];
        cAy = a.leaf_cen[3 * l + 1];
        cAz = a.leaf_cen[3 * l + 2];
    }
    bool ovf = false;
    while (sp > 0) {
        const int take = min(sp, 32);
        int2 it = make_int2(-1, 0);
        if (lane < take) it = st[sp - 1 - lane];
        sp -= take;
        __syncwarp();
        bool emit = false;
        int nch = 0, child = 0, level = 0;
        const int o = it.y;
        const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
        if (it.x >= 0) {
            const TreeNode N = a.nodes[it.x];
            const float dx = (float)ox * g.L32, dy = (float)oy * g.L32, dz = (float)oz * g.L32;
            const float gx = fmaxf(fmaxf(N.bx0 + dx - A.bx1, A.bx0 - (N.bx1 + dx)), 0.f);
            const float gy = fmaxf(fmaxf(N.by0 + dy - A.by1, A.by0 - (N.by1 + dy)), 0.f);
            const float gz = fmaxf(fmaxf(N.bz0 + dz - A.bz1, A.bz0 - (N.bz1 + dz)), 0.f);
            const float reach = fmaxf(hA, N.hmax * kTreeReach) * (1.f + 1e-5f) + slack;
            if (gx * gx + gy * gy + gz * gz < reach * reach) {
                if (N.child < 0) {
                    emit = true;
                    level = N.level;
                } else {
                    nch = N.nchild;
                    child = N.child;
                }
            }
        }
        const unsigned eb = __ballot_sync(kFull, emit);
        if (!COUNT && emit) {
            const int b = a.node_leaf[it.x];
            const int jx = ix + ox, jy = iy + oy, jz = iz + oz;
            const double kx = jx < 0 ? -1.0 : (jx >= nc ? 1.0 : 0.0), ky = jy < 0 ? -1.0 : (jy >= nc ? 1.0 : 0.0),
                         kz = jz < 0 ? -1.0 : (jz >= nc ? 1.0 : 0.0);
            const double sx = a.leaf_cen[3 * b] + kx * a.box - cAx, sy = a.leaf_cen[3 * b + 1] + ky * a.box - cAy,
                         sz = a.leaf_cen[3 * b + 2] + kz * a.box - cAz;
            const float fx = (float)sx, fy = (float)sy, fz = (float)sz;
            a.list[base + cnt + __popc(eb & lt)] = make_float4(fx, fy, fz, __int_as_float(b));
            // coordinates met in this pair's FP32 arithmetic stay below the two leaf
            // sides plus the offset
            const float m = fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz)));
            sc = fmaxf(sc, 0.5f * (sideA + ldexpf(g.L32, -level) + m) * (1.f + 1e-6f));
        }
        cnt += (uint32_t)__popc(eb);
        // push the children of the nodes within reach (lane order)
        int incl = nch;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += v;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        if (sp + total > kWalkCap) {
            ovf = true;
            break;
        }
        const int start = sp + incl - nch;
        for (int c = 0; c < nch; ++c) st[start + c] = make_int2(child + nch - 1 - c, o);
        sp += total;
        __syncwarp();
    }
    if (ovf) {
        if (lane == 0) atomicAdd(a.overflow, 1ull);
        return;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sc = fmaxf(sc, __shfl_xor_sync(kFull, sc, d));
    if (lane == 0) {
        if (COUNT) a.cnt[l] = cnt;
        else a.scale[l] = sc;
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(32 * kWalkWarps) k_leaf_walk(WalkArgs a)
{
    __shared__ int2 stk[kWalkWarps][kWalkCap];
    if (!COUNT && a.skip_ovf && *a.skip_ovf) return;
    if (!COUNT && a.err && *a.err) return;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nl = a.nlp ? *a.nlp : a.nl;
    const int first = blockIdx.x * kWalkWarps + wib, nw = gridDim.x * kWalkWarps;
    if (!a.ticket) {  // one warp per leaf (host-sized launch)
        for (int l = first; l < nl; l += nw) {
            walk_leaf<COUNT>(a, l, stk[wib]);
            __syncwarp();
        }
        return;
    }
    // persistent warps: the next leaf by ticket, taken one leaf ahead (walks differ
    // widely in length)
    unsigned tk = 0u;
    if (lane == 0) tk = atomicAdd(a.ticket, 1u);
    for (int l = first, nxt = 0; l < nl; l = nxt) {  // warp-uniform
        nxt = nw + (int)__shfl_sync(kFull, tk, 0);
        if (lane == 0 && nxt < nl) tk = atomicAdd(a.ticket, 1u);
        walk_leaf<COUNT>(a, l, stk[wib]);
        __syncwarp();
    }
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

template <typename T>
static int grow(sph_ctx *ctx, T *&p, int64_t &cap, int64_t need)
{
    if (need <= cap) return SPH_OK;
    cudaFree(p);
    p = nullptr;
    const int64_t c = need + need / 4 + 1024;
    SPH_CUDA(ctx, cudaMalloc(&p, sizeof(T) * c));
    cap = c;
    return SPH_OK;
}

// ------------------------------------------------ builds without host reads
// Inside a graph-captured step the sizes of the tree (frontiers, nodes, leaves, list
// entries) stay on the device (TreeCounts): every kernel reads its count there and
// strides over a fixed capacity, so the launch shapes do not depend on the data.
// The capacities are set before the capture: a frontier holds at most
// min(n, 8 floor(n / (leaf_max + 1))) children (only nodes of > leaf_max particles
// split, and they are disjoint on a level), so the nodes of the 14 refined levels
// always fit; the lists get a reserve over the last host build, and lists that
// outgrow it leave the step without pair work and an error for the host.

__global__ void k_tree_begin(const int *__restrict__ cs, int64_t ntop, const uint32_t *__restrict__ off, int n,
                             TreeCounts *__restrict__ tc)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int nroot = (int)off[ntop - 1] + (cs[ntop - 1] < n ? 1 : 0);
    tc->nl = 0;
    tc->err = 0;
    for (int k = 0; k < 18; ++k) tc->level_begin[k] = nroot;
    tc->level_begin[0] = 0;
    tc->list_total = 0ull;
    tc->walk_ovf = 0ull;
    tc->walk_ticket[0] = tc->walk_ticket[1] = 0u;
}

// children of level L: lb[L + 2] = lb[L + 1] + their count (none if they do not fit)
__global__ void k_level_adv(TreeCounts *__restrict__ tc, int level, const uint32_t *__restrict__ nk, int64_t capf,
                            int64_t cap_nodes)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t nnext = nk[capf];  // exclusive prefix past the last frontier entry: the total
    const int64_t b = tc->level_begin[level + 1];
    if (nnext > capf || b + nnext > cap_nodes) {
        tc->err |= kTreeErrNodes;
        nnext = 0;
    }
    tc->level_begin[level + 2] = (int)(b + nnext);
}

__global__ void k_set_nl(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ excl, int n,
                         TreeCounts *__restrict__ tc)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) tc->nl = (int)(excl[n - 1] + flag[n - 1]);
}

// entries [*nlp, cap) of v set to zero
__global__ void k_zero_tail(uint32_t *__restrict__ v, const int *__restrict__ nlp, int64_t cap)
{
    for (int64_t i = *nlp + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = 0u;
}

// the lists must fit their reserve and the 32-bit offsets; if not, no tile is run
__global__ void k_list_check(TreeCounts *__restrict__ tc, int64_t cap_list, int *__restrict__ n_tiles)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const unsigned long long t = tc->list_total;
    if (t > 0xfffffffeull || (int64_t)t > cap_list) {
        tc->err |= kTreeErrList;
        *n_tiles = 0;
    }
}

static int sm_count(sph_ctx *ctx)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    return sms > 0 ? sms : 148;
}

static int build_tree_device(sph_ctx *ctx, sph_particles *parts)
{
    AdaptiveTree &T = ctx->tree;
    const int n = (int)ctx->n;
    const int64_t ntop = ctx->grid.n_cells;
    const int64_t capf = T.dev_capf;
    TreeCounts *dc = T.dc;
    int rc;
    int top_bits = 1;
    while ((1ll << top_bits) < ntop) ++top_bits;
    if (n <= 0) {  // nothing to refine: no leaves, no tiles
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->n_tiles, 0, sizeof(int), ctx->stream));
        ctx->built = true;
        ctx->density_valid = false;
        return SPH_OK;
    }
    if (!dc) return fail(ctx, SPH_ERR_STATE, "device-sized tree build without prepared capacities");
    const int sms = sm_count(ctx);
    const unsigned gp = (unsigned)(8 * sms);  // grid-stride launches
    k_tree_keys<<<nblk(n, 256), 256, 0, ctx->stream>>>(parts->x, parts->y, parts->z, n, ctx->n_boxes, ctx->p.box_size,
                                                       ctx->d_boxes, ctx->keys64);
    SPH_LAUNCH(ctx, "tree keys");
    if ((rc = radix_sort64(ctx, n, top_bits + kMortonShift))) return rc;
    if ((rc = permute_particles(ctx, parts, false))) return rc;
    k_top_start<<<nblk(ntop + 1, 256), 256, 0, ctx->stream>>>(ctx->keys64, n, ntop, ctx->cell_start);
    SPH_LAUNCH(ctx, "top starts");
    k_nonempty<<<nblk(ntop, 256), 256, 0, ctx->stream>>>(ctx->cell_start, ntop, ctx->cell_tiles);
    SPH_LAUNCH(ctx, "top nonempty");
    if ((rc = exclusive_scan_u32(ctx, ctx->cell_tiles, ctx->cell_tiles, ntop))) return rc;
    k_tree_begin<<<1, 32, 0, ctx->stream>>>(ctx->cell_start, ntop, ctx->cell_tiles, n, dc);
    SPH_LAUNCH(ctx, "tree begin");
    k_roots<<<nblk(ntop, 256), 256, 0, ctx->stream>>>(ctx->cell_start, ntop, ctx->cell_tiles, T.nodes, T.top_node,
                                                      T.front);
    SPH_LAUNCH(ctx, "tree roots");
    int *cur = T.front, *nxt = T.front2;
    int *lb = dc->level_begin;
    for (int level = 0; level < kMortonBits; ++level) {
        k_node_split<<<gp, 256, 0, ctx->stream>>>(cur, 0, lb + level, (int)capf + 1, T.nodes, ctx->keys64,
                                                  ctx->leaf_max, T.bounds, T.nkids);
        SPH_LAUNCH(ctx, "node split");
        if ((rc = exclusive_scan_u32(ctx, T.nkids, T.nkids, capf + 1))) return rc;
        k_level_adv<<<1, 32, 0, ctx->stream>>>(dc, level, T.nkids, capf, T.dev_cap_nodes);
        SPH_LAUNCH(ctx, "level advance");
        k_make_children<<<gp, 256, 0, ctx->stream>>>(cur, 0, T.nodes, T.bounds, T.nkids, 0u, 0, lb + level, nxt);
        SPH_LAUNCH(ctx, "make children");
        std::swap(cur, nxt);
    }
    const int *n_nodes = lb + kMortonBits + 1;
    k_leaf_box<<<gp, 256, 0, ctx->stream>>>(T.nodes, 0, n_nodes, parts->x, parts->y, parts->z, parts->h,
                                            ctx->d_boxes, ctx->n_boxes);
    SPH_LAUNCH(ctx, "leaf boxes");
    for (int L = kMortonBits - 1; L >= 0; --L) {  // level kMortonBits holds leaves only
        k_merge_children<<<gp, 256, 0, ctx->stream>>>(T.nodes, 0, 0, lb, L);
        SPH_LAUNCH(ctx, "merge children");
    }
    // leaves in particle order
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->keys, 0, sizeof(uint32_t) * n, ctx->stream));
    k_leaf_marks<<<gp, 256, 0, ctx->stream>>>(T.nodes, 0, n_nodes, ctx->keys, T.node_at);
    SPH_LAUNCH(ctx, "leaf marks");
    if ((rc = exclusive_scan_u32(ctx, ctx->keys, ctx->keys_alt, n))) return rc;
    k_set_nl<<<1, 32, 0, ctx->stream>>>(ctx->keys, ctx->keys_alt, n, dc);
    SPH_LAUNCH(ctx, "leaf count");
    k_leaves<<<nblk(n, 256), 256, 0, ctx->stream>>>(ctx->keys, ctx->keys_alt, n, T.node_at, T.nodes, ctx->d_boxes,
                                                    ctx->n_boxes, T.leaf_of, T.leaf_node, T.node_leaf, T.leaf_rng,
                                                    T.leaf_cen, T.leaf_h, T.leaf_lo, T.leaf_hi);
    SPH_LAUNCH(ctx, "leaves");
    k_leaf_pos<<<nblk(n, 256), 256, 0, ctx->stream>>>(T.leaf_of, T.leaf_cen, parts->x, parts->y, parts->z, parts->h,
                                                      n, ctx->pos4);
    SPH_LAUNCH(ctx, "leaf positions");
    // tiles (the leaf arrays hold n + 1 entries: nl <= n)
    const int *nlp = &dc->nl;
    const int64_t capl = (int64_t)n + 1;
    k_leaf_hsort<<<gp, 32 * kSortWarps, 0, ctx->stream>>>(T.leaf_rng, 0, nlp, parts->h, T.tord, parts->x, parts->y,
                                                          parts->z, ctx->tile_w);
    SPH_LAUNCH(ctx, "leaf h order");
    k_leaf_tiles_n<<<gp, 256, 0, ctx->stream>>>(T.leaf_rng, 0, nlp, (int)capl, ctx->tile_w, T.list_off);
    SPH_LAUNCH(ctx, "leaf tile counts");
    if ((rc = exclusive_scan_u32(ctx, T.list_off, T.list_off, capl))) return rc;
    k_leaf_tiles<<<gp, 256, 0, ctx->stream>>>(T.leaf_rng, T.leaf_node, T.nodes, 0, nlp, ctx->tile_w, T.list_off,
                                              ctx->d_boxes, ctx->n_boxes, ctx->tiles, ctx->n_tiles);
    SPH_LAUNCH(ctx, "leaf tiles");
    // neighbour lists: warp walks, or one-thread walks where a warp's stack overflowed
    const unsigned gw = (unsigned)(7 * sms);  // 7 blocks of 2 walking warps (32 KB stacks) per SM
    WalkArgs wa{0,       nlp,           nullptr,          nullptr,     T.leaf_node,  T.nodes,
                T.top_node, T.node_leaf, T.leaf_cen,    ctx->d_boxes, ctx->n_boxes, ctx->p.box_size,
                T.list_off, T.list,      T.leaf_scale, T.list_off,   &dc->walk_ovf, &dc->walk_ticket[0]};
    k_leaf_walk<true><<<gw, 32 * kWalkWarps, 0, ctx->stream>>>(wa);
    SPH_LAUNCH(ctx, "leaf walk count");
    k_pairs_count<<<gp, 128, 0, ctx->stream>>>(0, nlp, &dc->walk_ovf, T.leaf_node, T.nodes, T.top_node, T.node_leaf,
                                               T.leaf_cen, ctx->d_boxes, ctx->n_boxes, ctx->p.box_size, T.list_off);
    SPH_LAUNCH(ctx, "pair count");
    k_zero_tail<<<gp, 256, 0, ctx->stream>>>(T.list_off, nlp, capl);
    SPH_LAUNCH(ctx, "list tail");
    k_sum_u32<<<gp, 256, 0, ctx->stream>>>(T.list_off, (int)capl, &dc->list_total);
    SPH_LAUNCH(ctx, "list total");
    if ((rc = exclusive_scan_u32(ctx, T.list_off, T.list_off, capl))) return rc;  // list_off[nl] = total
    k_list_check<<<1, 32, 0, ctx->stream>>>(dc, T.dev_cap_list, ctx->n_tiles);
    SPH_LAUNCH(ctx, "list check");
    wa.skip_ovf = &dc->walk_ovf;
    wa.err = &dc->err;
    wa.ticket = &dc->walk_ticket[1];
    k_leaf_walk<false><<<gw, 32 * kWalkWarps, 0, ctx->stream>>>(wa);
    SPH_LAUNCH(ctx, "leaf walk fill");
    k_pairs_fill<<<gp, 128, 0, ctx->stream>>>(0, nlp, &dc->walk_ovf, &dc->err, T.leaf_node, T.nodes, T.top_node,
                                              T.node_leaf, T.leaf_cen, ctx->d_boxes, ctx->n_boxes, ctx->p.box_size,
                                              T.list_off, T.list, T.leaf_scale);
    SPH_LAUNCH(ctx, "pair fill");
    if ((rc = order_tiles(ctx, ctx->tiles, ctx->n_tiles))) return rc;
    ctx->built = true;
    ctx->density_valid = false;
    return SPH_OK;
}

// Capacities for device-sized builds of the current plan (allocations happen here,
// never inside a capture); *sig identifies the arrays a captured build uses.
int tree_prepare_device(sph_ctx *ctx, uint64_t *sig)
{
    AdaptiveTree &T = ctx->tree;
    const int64_t n = std::max<int64_t>(ctx->n, 1);
    const int64_t ntop = ctx->grid.n_cells;
    const int64_t lm = std::max(ctx->leaf_max, 1);
    const int64_t kids = std::min<int64_t>(n, 8 * (n / (lm + 1)) + 8);
    const int64_t capf = std::max<int64_t>(ntop, kids);
    const int64_t cap_nodes = ntop + kMortonBits * kids + 64;
    if (cap_nodes >= (1ll << 31)) return fail(ctx, SPH_ERR_CAPACITY, "tree node capacity beyond 32-bit indices");
    // arrays sized for the host build's needs as well (ntop + 4n + 64 nodes), so that
    // host builds between captured runs do not move them
    const int64_t host_nodes = ntop + 4 * n + 64;
    const int64_t an = std::max(cap_nodes, host_nodes), af = std::max(capf + 1, host_nodes);
    // list reserve: as asked, else twice the last build's entries, at least 2^20
    const int64_t list_need =
        (ctx->p.list_reserve > 0 ? ctx->p.list_reserve : std::max<int64_t>(2 * T.n_entries, 1 << 20)) + 1;
    int rc;
    if ((rc = grow(ctx, ctx->keys64, T.cap_keys, n)) || (rc = grow(ctx, ctx->keys64_alt, T.cap_keys2, n)) ||
        (rc = grow(ctx, T.leaf_of, T.cap_leaf_of, n)) || (rc = grow(ctx, T.node_at, T.cap_node_at, n)) ||
        (rc = grow(ctx, T.tord, T.cap_tord, n)) || (rc = grow(ctx, T.act_ord, T.cap_act_ord, n)) ||
        (rc = grow(ctx, T.top_node, T.cap_top, ntop + 1)) || (rc = grow(ctx, T.nodes, T.cap_nodes, an)) ||
        (rc = grow(ctx, T.node_leaf, T.cap_node_leaf, an)) || (rc = grow(ctx, T.front, T.cap_front, af)) ||
        (rc = grow(ctx, T.front2, T.cap_front2, af)) || (rc = grow(ctx, T.bounds, T.cap_bounds, kBoundsW * af)) ||
        (rc = grow(ctx, T.nkids, T.cap_nkids, std::max(af, n + 2))) ||
        (rc = grow(ctx, T.leaf_node, T.cap_leaf_node, n + 1)) || (rc = grow(ctx, T.leaf_rng, T.cap_leaf_rng, n + 1)) ||
        (rc = grow(ctx, T.leaf_cen, T.cap_leaf_cen, 3 * n + 3)) || (rc = grow(ctx, T.leaf_h, T.cap_leaf_h, n + 1)) ||
        (rc = grow(ctx, T.leaf_lo, T.cap_leaf_lo, n + 1)) || (rc = grow(ctx, T.leaf_hi, T.cap_leaf_hi, n + 1)) ||
        (rc = grow(ctx, T.leaf_scale, T.cap_leaf_scale, n + 1)) ||
        (rc = grow(ctx, T.nact_leaf, T.cap_nact_leaf, n + 1)) || (rc = grow(ctx, T.list_off, T.cap_list_off, n + 2)) ||
        (rc = grow(ctx, T.list, T.cap_list, list_need)))
        return rc;
    if (!T.dc) SPH_CUDA(ctx, cudaMalloc(&T.dc, sizeof(TreeCounts)));
    if (!T.hc) SPH_CUDA(ctx, cudaMallocHost(&T.hc, sizeof(TreeCounts)));
    T.dev_capf = capf;
    T.dev_cap_nodes = cap_nodes;
    T.dev_cap_list = std::min<int64_t>(list_need - 1, T.cap_list);
    // FNV-1a over every array address and capacity the captured kernels see
    // (the sort's ping-pong pair in either order: captures may swap it)
    const void *ptrs[] = {std::min(ctx->keys64, ctx->keys64_alt), std::max(ctx->keys64, ctx->keys64_alt), T.leaf_of, T.node_at, T.tord, T.act_ord, T.top_node,
                          T.nodes, T.node_leaf, T.front, T.front2, T.bounds, T.nkids, T.leaf_node, T.leaf_rng,
                          T.leaf_cen, T.leaf_h, T.leaf_scale, T.nact_leaf, T.list_off, T.list, T.dc,
                          T.leaf_lo, T.leaf_hi};
    const int64_t caps[] = {capf, T.dev_cap_nodes, T.cap_list, T.dev_cap_list, ctx->leaf_max};
    uint64_t hsh = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        for (int b = 0; b < 8; ++b) hsh = (hsh ^ ((v >> (8 * b)) & 0xffu)) * 1099511628211ull;
    };
    for (const void *q : ptrs) mix((uint64_t)(uintptr_t)q);
    for (int64_t c : caps) mix((uint64_t)c);
    *sig = hsh;
    return SPH_OK;
}

// Host copies of the device sizes after captured steps; the list error is fatal
// (the step that met it ran no pair work), an overfull node array is not (its
// leaves stayed larger, the lists exact).
int tree_read_device(sph_ctx *ctx)
{
    AdaptiveTree &T = ctx->tree;
    if (ctx->n <= 0) {
        T.n_nodes = T.n_leaves = 0;
        T.n_entries = 0;
        ctx->st.n_cells = 0;
        return SPH_OK;
    }
    if (!T.dc) return SPH_OK;
    SPH_CUDA(ctx, cudaMemcpyAsync(T.hc, T.dc, sizeof(TreeCounts), cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    T.n_nodes = T.hc->level_begin[kMortonBits + 1];
    T.n_leaves = T.hc->nl;
    T.n_entries = (int64_t)T.hc->list_total;
    ctx->st.n_cells = T.hc->nl;
    if (T.hc->err & kTreeErrList)
        return fail(ctx, SPH_ERR_CAPACITY, "neighbour lists outgrew the reserve of the captured steps (the step "
                                           "that met it did no pair work)");
    return SPH_OK;
}

// Build the adaptive cells for the current plan (top grids): keys, sort, permutation,
// tree, leaves, leaf-relative positions, tiles and neighbour lists.
int build_tree(sph_ctx *ctx, sph_particles *parts)
{
    AdaptiveTree &T = ctx->tree;
    if (T.device_sized) return build_tree_device(ctx, parts);
    const int n = (int)ctx->n;
    const int64_t ntop = ctx->grid.n_cells;
    int rc;
    int64_t np = std::max<int64_t>(ctx->cap, 1);
    if ((rc = grow(ctx, ctx->keys64, T.cap_keys, np)) || (rc = grow(ctx, ctx->keys64_alt, T.cap_keys2, np)) ||
        (rc = grow(ctx, T.leaf_of, T.cap_leaf_of, np)) || (rc = grow(ctx, T.node_at, T.cap_node_at, np)) ||
        (rc = grow(ctx, T.tord, T.cap_tord, np)) ||
        (rc = grow(ctx, T.top_node, T.cap_top, ntop + 1)))
        return rc;
    if (!T.h_u32) SPH_CUDA(ctx, cudaMallocHost(&T.h_u32, 16 * sizeof(uint32_t)));
    if (!T.h_i32) SPH_CUDA(ctx, cudaMallocHost(&T.h_i32, 16 * sizeof(int)));
    int top_bits = 1;
    while ((1ll << top_bits) < ntop) ++top_bits;
    if (top_bits + kMortonShift > 64) return fail(ctx, SPH_ERR_INVALID_ARG, "too many top cells for 64-bit keys");
    if (n <= 0) {  // nothing to refine: no leaves, no tiles
        T.n_nodes = T.n_leaves = 0;
        T.n_entries = 0;
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->n_tiles, 0, sizeof(int), ctx->stream));
        ctx->built = true;
        ctx->density_valid = false;
        ctx->st.n_cells = 0;
        return SPH_OK;
    }
    {
        k_tree_keys<<<nblk(n, 256), 256, 0, ctx->stream>>>(parts->x, parts->y, parts->z, n, ctx->n_boxes,
                                                           ctx->p.box_size, ctx->d_boxes, ctx->keys64);
        SPH_LAUNCH(ctx, "tree keys");
        rc = radix_sort64(ctx, n, top_bits + kMortonShift);
        if (rc) return rc;
        rc = permute_particles(ctx, parts, false);  // caller arrays into sorted order
        if (rc) return rc;
    }
    // top-cell ranges and roots
    k_top_start<<<nblk(ntop + 1, 256), 256, 0, ctx->stream>>>(ctx->keys64, n, ntop, ctx->cell_start);
    SPH_LAUNCH(ctx, "top starts");
    k_nonempty<<<nblk(ntop, 256), 256, 0, ctx->stream>>>(ctx->cell_start, ntop, ctx->cell_tiles);
    SPH_LAUNCH(ctx, "top nonempty");
    rc = exclusive_scan_u32(ctx, ctx->cell_tiles, ctx->cell_tiles, ntop);
    if (rc) return rc;
    // roots = exclusive count before the last top cell + whether the last is non-empty
    SPH_CUDA(ctx, cudaMemcpyAsync(&T.h_u32[0], ctx->cell_tiles + (ntop - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    SPH_CUDA(ctx, cudaMemcpyAsync(&T.h_i32[0], ctx->cell_start + (ntop - 1), sizeof(int), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const uint32_t nroot = T.h_u32[0] + (T.h_i32[0] < n ? 1u : 0u);
    const int64_t node_cap_need = (int64_t)nroot + 4 * (int64_t)n + 64;
    if ((rc = grow(ctx, T.nodes, T.cap_nodes, node_cap_need)) || (rc = grow(ctx, T.front, T.cap_front, node_cap_need)) ||
        (rc = grow(ctx, T.front2, T.cap_front2, node_cap_need)) ||
        (rc = grow(ctx, T.bounds, T.cap_bounds, kBoundsW * node_cap_need)) ||
        (rc = grow(ctx, T.nkids, T.cap_nkids, node_cap_need)) || (rc = grow(ctx, T.node_leaf, T.cap_node_leaf, node_cap_need)))
        return rc;
    k_roots<<<nblk(ntop, 256), 256, 0, ctx->stream>>>(ctx->cell_start, ntop, ctx->cell_tiles, T.nodes, T.top_node,
                                                      T.front);
    SPH_LAUNCH(ctx, "tree roots");
    // refine level by level (host reads the next frontier size)
    int n_nodes = (int)nroot, nfront = (int)nroot;
    int *cur = T.front, *nxt = T.front2;
    std::vector<int> level_begin(1, 0);  // nodes of level L: [level_begin[L], level_begin[L + 1])
    for (int level = 0; level <= kMortonBits && nfront > 0; ++level) {
        k_node_split<<<nblk(nfront, 256), 256, 0, ctx->stream>>>(cur, nfront, nullptr, 0, T.nodes, ctx->keys64,
                                                                 ctx->leaf_max, T.bounds, T.nkids);
        SPH_LAUNCH(ctx, "node split");
        SPH_CUDA(ctx, cudaMemcpyAsync(&T.h_u32[1], T.nkids + (nfront - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        rc = exclusive_scan_u32(ctx, T.nkids, T.nkids, nfront);
        if (rc) return rc;
        SPH_CUDA(ctx, cudaMemcpyAsync(&T.h_u32[2], T.nkids + (nfront - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        const int nnext = (int)(T.h_u32[1] + T.h_u32[2]);
        level_begin.push_back(n_nodes);
        if (nnext == 0) break;
        if ((int64_t)n_nodes + nnext > T.cap_nodes) return fail(ctx, SPH_ERR_INVALID_ARG, "tree node capacity exceeded");
        k_make_children<<<nblk(nfront, 256), 256, 0, ctx->stream>>>(cur, nfront, T.nodes, T.bounds, T.nkids,
                                                                    (uint32_t)nnext, n_nodes, nullptr, nxt);
        SPH_LAUNCH(ctx, "make children");
        n_nodes += nnext;
        nfront = nnext;
        std::swap(cur, nxt);
    }
    T.n_nodes = n_nodes;
    if (level_begin.back() != n_nodes) level_begin.push_back(n_nodes);
    // largest h and bounding box of every node: leaves from their particles, then the
    // levels upwards from their children
    auto node_boxes = [&]() -> int {
        k_leaf_box<<<nblk((int64_t)n_nodes * 32, 256), 256, 0, ctx->stream>>>(
            T.nodes, n_nodes, nullptr, parts->x, parts->y, parts->z, parts->h, ctx->d_boxes, ctx->n_boxes);
        SPH_LAUNCH(ctx, "leaf boxes");
        for (int L = (int)level_begin.size() - 2; L >= 0; --L) {
            const int first = level_begin[L], last = level_begin[L + 1];
            if (last <= first) continue;
            k_merge_children<<<nblk(last - first, 256), 256, 0, ctx->stream>>>(T.nodes, first, last, nullptr, 0);
            SPH_LAUNCH(ctx, "merge children");
        }
        return SPH_OK;
    };
    if (n > 0) {
        rc = node_boxes();
        if (rc) return rc;
    }
    if (ctx->h_guess_pending) {
        // first build with SPH_FLAG_TREE_H_GUESS: h from the tree, node maxima again;
        // if the largest h no longer fits the top grid, plan and build once more
        ctx->h_guess_pending = false;
        k_h_guess<<<nblk(n_nodes, 128), 128, 0, ctx->stream>>>(T.nodes, n_nodes, ctx->d_boxes, ctx->n_boxes,
                                                              (int)(2.f * ctx->p.n_ngb), ctx->p.n_ngb,
                                                              ctx->p.box_size, parts->h);
        SPH_LAUNCH(ctx, "tree h guess");
        rc = node_boxes();
        if (rc) return rc;
        rc = read_box_max_h(ctx, parts);
        if (rc) return rc;
        bool fits = true;
        for (int b = 0; b < ctx->n_boxes; ++b)
            if ((double)ctx->h_box_hmax[b] * ctx->p.cell_factor > ctx->h_boxes[b].L64) fits = false;
        if (!fits) {
            rc = plan_from_hmax(ctx);
            if (rc) return rc;
            return build_tree(ctx, parts);
        }
    }
    // leaves in particle order
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->keys, 0, sizeof(uint32_t) * std::max(n, 1), ctx->stream));
    k_leaf_marks<<<nblk(n_nodes, 256), 256, 0, ctx->stream>>>(T.nodes, n_nodes, nullptr, ctx->keys, T.node_at);
    SPH_LAUNCH(ctx, "leaf marks");
    rc = exclusive_scan_u32(ctx, ctx->keys, ctx->keys_alt, n);
    if (rc) return rc;
    SPH_CUDA(ctx, cudaMemcpyAsync(&T.h_u32[3], ctx->keys_alt + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    SPH_CUDA(ctx, cudaMemcpyAsync(&T.h_u32[4], ctx->keys + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int nl = (int)(T.h_u32[3] + T.h_u32[4]);
    T.n_leaves = nl;
    if ((rc = grow(ctx, T.leaf_node, T.cap_leaf_node, nl + 1)) || (rc = grow(ctx, T.leaf_rng, T.cap_leaf_rng, nl + 1)) ||
        (rc = grow(ctx, T.leaf_cen, T.cap_leaf_cen, 3 * (int64_t)nl + 3)) ||
        (rc = grow(ctx, T.leaf_h, T.cap_leaf_h, nl + 1)) || (rc = grow(ctx, T.leaf_scale, T.cap_leaf_scale, nl + 1)) ||
        (rc = grow(ctx, T.leaf_lo, T.cap_leaf_lo, nl + 1)) || (rc = grow(ctx, T.leaf_hi, T.cap_leaf_hi, nl + 1)) ||
        (rc = grow(ctx, T.list_off, T.cap_list_off, nl + 2)))
        return rc;
    {
        k_leaves<<<nblk(n, 256), 256, 0, ctx->stream>>>(ctx->keys, ctx->keys_alt, n, T.node_at, T.nodes, ctx->d_boxes,
                                                        ctx->n_boxes, T.leaf_of, T.leaf_node, T.node_leaf, T.leaf_rng,
                                                        T.leaf_cen, T.leaf_h, T.leaf_lo, T.leaf_hi);
        SPH_LAUNCH(ctx, "leaves");
        k_leaf_pos<<<nblk(n, 256), 256, 0, ctx->stream>>>(T.leaf_of, T.leaf_cen, parts->x, parts->y, parts->z,
                                                          parts->h, n, ctx->pos4);
        SPH_LAUNCH(ctx, "leaf positions");
    }
    // tiles
    if (nl > 0) {
        k_leaf_hsort<<<nblk(nl, kSortWarps), 32 * kSortWarps, 0, ctx->stream>>>(T.leaf_rng, nl, nullptr, parts->h,
                                                                                 T.tord, parts->x, parts->y, parts->z,
                                                                                 ctx->tile_w);
        SPH_LAUNCH(ctx, "leaf h order");
        k_leaf_tiles_n<<<nblk(nl, 256), 256, 0, ctx->stream>>>(T.leaf_rng, nl, nullptr, 0, ctx->tile_w, T.list_off);
        SPH_LAUNCH(ctx, "leaf tile counts");
        rc = exclusive_scan_u32(ctx, T.list_off, T.list_off, nl);
        if (rc) return rc;
        k_leaf_tiles<<<nblk(nl, 256), 256, 0, ctx->stream>>>(T.leaf_rng, T.leaf_node, T.nodes, nl, nullptr,
                                                            ctx->tile_w, T.list_off, ctx->d_boxes, ctx->n_boxes, ctx->tiles,
                                                            ctx->n_tiles);
        SPH_LAUNCH(ctx, "leaf tiles");
        // neighbour lists: count, scan, fill (warp walks; one-thread walks if a warp's
        // stack overflowed)
        WalkArgs wa{nl, nullptr, nullptr, nullptr, T.leaf_node, T.nodes, T.top_node, T.node_leaf, T.leaf_cen, ctx->d_boxes, ctx->n_boxes,
                    ctx->p.box_size, T.list_off, T.list, T.leaf_scale, T.list_off, ctx->counters + C_WALKOVF, nullptr};
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_WALKOVF, 0, sizeof(unsigned long long), ctx->stream));
        k_leaf_walk<true><<<nblk(nl, kWalkWarps), 32 * kWalkWarps, 0, ctx->stream>>>(wa);
        SPH_LAUNCH(ctx, "leaf walk count");
        SPH_CUDA(ctx, cudaMemcpyAsync(&T.h_u32[8], ctx->counters + C_WALKOVF, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        const bool warp_walk = T.h_u32[8] == 0u;
        if (!warp_walk) {
            k_pairs_count<<<nblk(nl, 128), 128, 0, ctx->stream>>>(nl, nullptr, nullptr, T.leaf_node, T.nodes, T.top_node, T.node_leaf,
                                                                 T.leaf_cen, ctx->d_boxes, ctx->n_boxes,
                                                                 ctx->p.box_size, T.list_off);
            SPH_LAUNCH(ctx, "pair count");
        }
        // the 32-bit offsets must hold the total
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_LISTTOT, 0, sizeof(unsigned long long), ctx->stream));
        k_sum_u32<<<nblk(std::min(nl, 1 << 20), 256), 256, 0, ctx->stream>>>(T.list_off, nl, ctx->counters + C_LISTTOT);
        SPH_LAUNCH(ctx, "list total");
        SPH_CUDA(ctx, cudaMemcpyAsync(&T.h_u32[10], ctx->counters + C_LISTTOT, sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, ctx->stream));
        SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        unsigned long long total = 0;
        memcpy(&total, &T.h_u32[10], sizeof total);
        if (total > 0xfffffffeull)
            return fail(ctx, SPH_ERR_CAPACITY, "neighbour lists exceed 2^32 - 2 entries (h far above the particle "
                                               "spacing in dense regions: see SPH_FLAG_TREE_H_GUESS)");
        SPH_CUDA(ctx, cudaMemcpyAsync(&T.h_u32[5], T.list_off + (nl - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        rc = exclusive_scan_u32(ctx, T.list_off, T.list_off, nl);
        if (rc) return rc;
        SPH_CUDA(ctx, cudaMemcpyAsync(&T.h_u32[6], T.list_off + (nl - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        const int64_t ne = (int64_t)T.h_u32[5] + T.h_u32[6];
        T.n_entries = ne;
        T.h_u32[7] = (uint32_t)ne;  // list_off[nl] = total (pinned source, copied in order)
        SPH_CUDA(ctx, cudaMemcpyAsync(T.list_off + nl, &T.h_u32[7], sizeof(uint32_t), cudaMemcpyHostToDevice,
                                      ctx->stream));
        if ((rc = grow(ctx, T.list, T.cap_list, ne + 1))) return rc;
        if (warp_walk) {
            wa.list = T.list;
            k_leaf_walk<false><<<nblk(nl, kWalkWarps), 32 * kWalkWarps, 0, ctx->stream>>>(wa);
            SPH_LAUNCH(ctx, "leaf walk fill");
        } else {
            k_pairs_fill<<<nblk(nl, 128), 128, 0, ctx->stream>>>(nl, nullptr, nullptr, nullptr, T.leaf_node, T.nodes, T.top_node, T.node_leaf,
                                                                T.leaf_cen, ctx->d_boxes, ctx->n_boxes,
                                                                ctx->p.box_size, T.list_off, T.list, T.leaf_scale);
            SPH_LAUNCH(ctx, "pair fill");
        }
        if ((rc = order_tiles(ctx, ctx->tiles, ctx->n_tiles))) return rc;
    } else {
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->n_tiles, 0, sizeof(int), ctx->stream));
    }
    ctx->built = true;
    ctx->density_valid = false;
    ctx->st.n_cells = nl;
    return SPH_OK;
}

// Largest current h of every leaf into leaf_lo[].w (one warp per leaf; device count
// when nlp is set): the force pass then prunes a leaf's list entry with the largest h
// its sources have, not with kTreeReach x the build-time value.
__global__ void k_leaf_hcur(const int2 *__restrict__ rng, int nl_h, const int *__restrict__ nlp,
                            const float *__restrict__ h, float4 *__restrict__ leaf_lo)
{
    const int lane = threadIdx.x & 31;
    const int nl = nlp ? *nlp : nl_h;
    for (int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; l < nl; l += (gridDim.x * blockDim.x) >> 5) {
        const int2 r = rng[l];  // warp-uniform
        float m = 0.f;
        for (int p = r.x + lane; p < r.y; p += 32) m = fmaxf(m, h[p]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
        if (lane == 0) leaf_lo[l].w = m;
    }
}

int tree_leaf_hcur(sph_ctx *ctx, sph_particles *parts)
{
    AdaptiveTree &T = ctx->tree;
    if (ctx->n <= 0) return SPH_OK;
    if (T.device_sized) {
        if (!T.dc) return SPH_OK;
        k_leaf_hcur<<<8 * sm_count(ctx), 256, 0, ctx->stream>>>(T.leaf_rng, 0, &T.dc->nl, parts->h, T.leaf_lo);
    } else {
        if (T.n_leaves <= 0) return SPH_OK;
        k_leaf_hcur<<<nblk((int64_t)T.n_leaves * 32, 256), 256, 0, ctx->stream>>>(T.leaf_rng, T.n_leaves, nullptr,
                                                                                  parts->h, T.leaf_lo);
    }
    SPH_LAUNCH(ctx, "leaf current h");
    return SPH_OK;
}

// leaves whose largest current h fell below kTreeShrink x their build value
__global__ void k_leaf_shrink(const int2 *__restrict__ rng, int nl, const float *__restrict__ h,
                              const float *__restrict__ hb, unsigned long long *__restrict__ count)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    bool s = false;
    if (l < nl) {
        float m = 0.f;
        for (int p = rng[l].x; p < rng[l].y; ++p) m = fmaxf(m, h[p]);
        s = m < kTreeShrink * hb[l];
    }
    const unsigned b = __ballot_sync(kFull, s);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, (unsigned long long)__popc(b));
}

int tree_shrink_count(sph_ctx *ctx, sph_particles *parts)
{
    const int nl = ctx->tree.n_leaves;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_SHRINK, 0, sizeof(unsigned long long), ctx->stream));
    if (nl <= 0) return SPH_OK;
    k_leaf_shrink<<<nblk(nl, 256), 256, 0, ctx->stream>>>(ctx->tree.leaf_rng, nl, parts->h, ctx->tree.leaf_h,
                                                         ctx->counters + C_SHRINK);
    SPH_LAUNCH(ctx, "leaf shrink");
    return SPH_OK;
}

__global__ void k_top_of_key(const uint64_t *__restrict__ keys, int n, int32_t *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)(keys[i] >> kMortonShift);
}

int tree_cell_keys_out(sph_ctx *ctx, int32_t *dev_keys)
{
    const int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    k_top_of_key<<<nblk(n, 256), 256, 0, ctx->stream>>>(ctx->keys64, n, dev_keys);
    SPH_LAUNCH(ctx, "top cell keys");
    return SPH_OK;
}

// ------------------------------------------------ work order of the pair passes
// A pass hands its tile groups out by a ticket, in array order.  On uneven batched
// boxes the costliest tiles take ~40 % of a warp's share of a pass, and one of them
// taken late leaves its SM working alone at the end (measured: the last SM busy
// ~30 % past the others).  So the groups are put in descending order of cost --
// longest first, as in list scheduling -- estimated as the sources their leaf's list
// streams, by octaves: a counting sort on log2 of the cost.  The order within an
// octave is whatever the atomics give; a tile's sums do not depend on when it runs.
// Groups of 32 / TW tiles move together (TW = 16: two tiles share a warp's batches),
// and a partial last group keeps its place.
constexpr int kOrderOctaves = 32;

__global__ void k_order_key(const int4 *__restrict__ tiles, const int *__restrict__ n_tiles, int tpw,
                            const uint32_t *__restrict__ list_off, const float4 *__restrict__ list,
                            const int2 *__restrict__ rng, uint32_t *__restrict__ key, unsigned *__restrict__ hist)
{
    __shared__ unsigned sh[kOrderOctaves];
    if (threadIdx.x < kOrderOctaves) sh[threadIdx.x] = 0u;
    __syncthreads();
    const int ng = *n_tiles / tpw;  // whole groups
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        unsigned cost = 1u;
        for (int s = 0; s < tpw; ++s) {
            const int lf = tiles[g * tpw + s].x;
            unsigned c = 0u;
            for (uint32_t e = list_off[lf], e1 = list_off[lf + 1]; e < e1; ++e) {
                const int2 r = rng[__float_as_int(list[e].w)];
                c += (unsigned)(r.y - r.x);
            }
            cost = max(cost, c);
        }
        const unsigned b = 31u - __clz(cost);
        key[g] = b;
        atomicAdd(&sh[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kOrderOctaves && sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

// hist[0..31]: groups per octave -> hist[32 + b]: first position of octave b, the
// largest octave first (one warp)
__global__ void k_order_base(unsigned *hist)
{
    const int lane = threadIdx.x & 31, b = 31 - lane;
    const unsigned v = hist[b];
    unsigned incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned u = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += u;
    }
    hist[32 + b] = incl - v;
}

__global__ void k_order_scatter(const int4 *__restrict__ tiles, const int *__restrict__ n_tiles, int tpw,
                                const uint32_t *__restrict__ key, unsigned *__restrict__ cursor,
                                int4 *__restrict__ out)
{
    const int nt = *n_tiles, ng = nt / tpw;
    const int lane = threadIdx.x & 31;
    // warp-uniform trip count; the lanes of one octave take their positions with one
    // atomic (a pass's groups fall into a few octaves: per-lane atomics on one counter
    // would serialise)
    const int stride = gridDim.x * blockDim.x;
    for (int g0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); g0 < ng; g0 += stride) {
        const int g = g0 + lane;
        const bool in = g < ng;
        const unsigned b = in ? key[g] : 0xffffffffu;
        const unsigned peers = __match_any_sync(kFull, b);
        const int leader = __ffs(peers) - 1;
        unsigned base = 0u;
        if (in && lane == leader) base = atomicAdd(&cursor[b], (unsigned)__popc(peers));
        base = __shfl_sync(kFull, base, leader);
        if (in) {
            const unsigned pos = base + (unsigned)__popc(peers & ((1u << lane) - 1u));
            for (int s = 0; s < tpw; ++s) out[pos * tpw + s] = tiles[g * tpw + s];
        }
    }
    const int t = ng * tpw + blockIdx.x * blockDim.x + threadIdx.x;  // the partial group, in place
    if (t < nt) out[t] = tiles[t];
}

__global__ void k_copy_tiles(const int4 *__restrict__ src, const int *__restrict__ n_tiles, int4 *__restrict__ dst)
{
    const int nt = *n_tiles;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) dst[t] = src[t];
}

// Longest-first order of the tile groups of `tiles` (adaptive cells; device count).
// Scratch: the uniform grid's tile flags and positions (unused with adaptive cells)
// and the build's gather scratch (free once the cells are built).
int order_tiles(sph_ctx *ctx, int4 *tiles, const int *n_tiles)
{
    AdaptiveTree &T = ctx->tree;
    if (!ctx->adaptive || ctx->n <= 0 || !T.list_off || !T.list) return SPH_OK;
    if ((int64_t)sizeof(double) * 6 * ctx->cap < (int64_t)sizeof(int4) * ctx->tile_cap) return SPH_OK;  // tiny sets
    const int tpw = 32 / ctx->tile_w;
    unsigned *hist = ctx->tile_pos;
    int4 *out = reinterpret_cast<int4 *>(ctx->s64);
    const unsigned gp = (unsigned)(8 * sm_count(ctx));
    SPH_CUDA(ctx, cudaMemsetAsync(hist, 0, sizeof(unsigned) * 2 * kOrderOctaves, ctx->stream));
    k_order_key<<<gp, 256, 0, ctx->stream>>>(tiles, n_tiles, tpw, T.list_off, T.list, T.leaf_rng, ctx->tile_flag,
                                             hist);
    SPH_LAUNCH(ctx, "tile order keys");
    k_order_base<<<1, 32, 0, ctx->stream>>>(hist);
    SPH_LAUNCH(ctx, "tile order octaves");
    k_order_scatter<<<gp, 256, 0, ctx->stream>>>(tiles, n_tiles, tpw, ctx->tile_flag, hist + kOrderOctaves, out);
    SPH_LAUNCH(ctx, "tile order scatter");
    k_copy_tiles<<<gp, 256, 0, ctx->stream>>>(out, n_tiles, tiles);
    SPH_LAUNCH(ctx, "tile order copy");
    return SPH_OK;
}

int compact_active_leaf_tiles(sph_ctx *ctx)
{
    AdaptiveTree &T = ctx->tree;
    if (T.device_sized) {  // counts on the device, capacities set by tree_prepare_device
        if (ctx->n <= 0 || !T.dc) {
            SPH_CUDA(ctx, cudaMemsetAsync(ctx->n_act_tiles, 0, sizeof(int), ctx->stream));
            return SPH_OK;
        }
        const int64_t capl = std::max<int64_t>(ctx->n, 1) + 1;
        const unsigned gp = (unsigned)(8 * sm_count(ctx));
        k_leaf_active<<<gp, 256, 0, ctx->stream>>>(T.leaf_rng, 0, &T.dc->nl, (int)capl, T.tord, ctx->active,
                                                   ctx->tile_w, ctx->counters + C_UNCONV, T.act_ord, T.nkids,
                                                   T.nact_leaf);
        SPH_LAUNCH(ctx, "leaf active targets");
        int rc = exclusive_scan_u32(ctx, T.nkids, T.nkids, capl);
        if (rc) return rc;
        k_leaf_active_tiles<<<gp, 256, 0, ctx->stream>>>(T.leaf_rng, T.leaf_node, T.nodes, 0, &T.dc->nl, ctx->tile_w,
                                                         T.nkids, T.nact_leaf, ctx->d_boxes, ctx->n_boxes, &T.dc->err,
                                                         ctx->counters + C_UNCONV, ctx->act_tiles, ctx->n_act_tiles);
        SPH_LAUNCH(ctx, "leaf active tiles");
        return order_tiles(ctx, ctx->act_tiles, ctx->n_act_tiles);
    }
    const int nl = T.n_leaves;
    if (nl <= 0) {
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->n_act_tiles, 0, sizeof(int), ctx->stream));
        return SPH_OK;
    }
    int rc;
    if ((rc = grow(ctx, T.act_ord, T.cap_act_ord, std::max<int64_t>(ctx->cap, 1))) ||
        (rc = grow(ctx, T.nact_leaf, T.cap_nact_leaf, nl + 1)))
        return rc;
    // per-leaf tile counts in nkids (free outside the build; it holds >= n_leaves entries)
    k_leaf_active<<<nblk((int64_t)nl * 32, 256), 256, 0, ctx->stream>>>(T.leaf_rng, nl, nullptr, 0, T.tord,
                                                                        ctx->active, ctx->tile_w, nullptr, T.act_ord,
                                                                        T.nkids, T.nact_leaf);
    SPH_LAUNCH(ctx, "leaf active targets");
    rc = exclusive_scan_u32(ctx, T.nkids, T.nkids, nl);
    if (rc) return rc;
    k_leaf_active_tiles<<<nblk(nl, 256), 256, 0, ctx->stream>>>(T.leaf_rng, T.leaf_node, T.nodes, nl, nullptr,
                                                               ctx->tile_w,
                                                               T.nkids, T.nact_leaf, ctx->d_boxes, ctx->n_boxes,
                                                               nullptr, nullptr, ctx->act_tiles, ctx->n_act_tiles);
    SPH_LAUNCH(ctx, "leaf active tiles");
    return order_tiles(ctx, ctx->act_tiles, ctx->n_act_tiles);
}

void free_tree(sph_ctx *ctx)
{
    AdaptiveTree &T = ctx->tree;
    void *ptrs[] = {ctx->keys64, ctx->keys64_alt, T.leaf_of, T.tord, T.act_ord, T.nact_leaf, T.node_at, T.top_node, T.nodes, T.front, T.front2,
                    T.bounds, T.nkids, T.node_leaf, T.leaf_node, T.leaf_rng, T.leaf_cen, T.leaf_h, T.leaf_lo, T.leaf_hi,
                    T.leaf_scale, T.list_off, T.list};
    for (void *p : ptrs) cudaFree(p);
    cudaFree(T.dc);
    cudaFreeHost(T.hc);
    cudaFreeHost(T.h_u32);
    cudaFreeHost(T.h_i32);
    ctx->keys64 = ctx->keys64_alt = nullptr;
    T = AdaptiveTree();
}

}  // namespace sph
