// sph_hpredict.cu -- learned initial smoothing lengths for the h iteration of
// Theuns et al. 2015, Sec. 2 (Newton on N_w(h) = N_ngb).  Not part of the paper:
// a small MLP predicts, from quantities the previous step left behind, the ratio
// between a particle's converged h and its previous h, and the iteration starts
// there instead of at the previous h.  It converges to the same root at the same
// tolerance; the predictor only moves the starting point.
//
//   features (6, per particle, after the cell build of a step, before its density
//   pass; "prev" = the previous hydro pass, dt = this step's time step):
//     f0 = dt * divv_prev                    (compression predicted by the flow)
//     f1 = log(max(n_ngb_prev, 1) / N_ngb)
//     f2 = log(h_cell / h_prev), h_cell = (3 N_ngb / (4 pi n_cell))^(1/3) with
//          n_cell = count / side^3 of the particle's cell (adaptive: its leaf)
//     f3 = log(count / N_ngb)
//     f4 = log(h_prev / side)
//     f5 = dt * vsig_prev / h_prev
//   model: z = (f - mean) / sd;  y = W3 silu(W2 silu(W1 z + b1) + b2) + b3
//          (6 -> 64 -> 64 -> 1, SiLU); log(h0 / h_prev) = y * sd_y + mean_y,
//          clamped to [log 1/2, log g_max]
//   inference: BF16 weights and activations, FP32 accumulation, on the 5th-
//          generation tensor cores: tcgen05.mma with operands in shared memory and
//          the accumulators in tensor memory, 128 particles per MMA tile
//   training: MSE on the normalised target, Adam, FP32 master weights; per block
//          partial gradients reduced in a fixed order (deterministic)
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "sph_internal.cuh"

namespace sph {

constexpr int kF = 6;   // features
constexpr int kHid = 64; // hidden width
// FP32 parameter vector (training state and the source of the BF16 copy)
constexpr int kOffW1 = 0;                    // W1[kHid][kF]
constexpr int kOffB1 = kOffW1 + kHid * kF;   // b1[kHid]
constexpr int kOffW2 = kOffB1 + kHid;        // W2[kHid][kHid]  (out, in)
constexpr int kOffB2 = kOffW2 + kHid * kHid; // b2[kHid]
constexpr int kOffW3 = kOffB2 + kHid;        // W3[kHid]
constexpr int kOffB3 = kOffW3 + kHid;        // b3
constexpr int kNParam = kOffB3 + 1;          // 4673
// normalisation vector: feature means[6], feature sds[6], target mean, target sd
constexpr int kNNorm = 2 * kF + 2;
// BF16 inference copy: W1 rows padded to 8 inputs, W2 rows padded to 72 (bank
// spread of the B-fragment loads), W3
constexpr int kW1Row = 8, kW2Row = 72;
constexpr int kBfW1 = 0, kBfW2 = kHid * kW1Row, kBfW3 = kBfW2 + kHid * kW2Row;
constexpr int kNBf = kBfW3 + kHid;

// training schedule: blocks x sub-tiles x samples per Adam step
constexpr int kTrThreads = 256, kTrS = 64, kTrSub = 4, kTrBlocks = 64;
constexpr int kTrBatch = kTrBlocks * kTrSub * kTrS;  // 16384


__device__ __forceinline__ float silu(float x) { return x / (1.f + __expf(-x)); }
// inference: the quotient by the fast reciprocal (the activations are rounded to
// BF16, 2^-9, far above its couple of FP32 ulps)
__device__ __forceinline__ float silu_fast(float x) { return __fdividef(x, 1.f + __expf(-x)); }
__device__ __forceinline__ float silu_grad(float x)
{
    const float s = 1.f / (1.f + __expf(-x));
    return s * (1.f + x * (1.f - s));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
    return *reinterpret_cast<const uint32_t *>(&v);
}


// ------------------------------------------------------------------ features

struct FeatArgs {
    const float *h, *divv, *vsig;
    const int32_t *n_ngb;
    const double *d_dt;
    // uniform grid
    const uint32_t *keys;
    const int *cell_start;
    // adaptive cells
    const int *leaf_of;
    const int2 *leaf_rng;
    const int *leaf_node;
    const TreeNode *nodes;
    const BoxDev *bxs;
    int nb, n, adaptive;
    float n_ngb_target;
    float *feats;   // n x 6
    float *h_prev;  // n
};

__device__ __forceinline__ int hp_box_of_slot(int p, const BoxDev *__restrict__ bx, int nb)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bx[mid].p_begin <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_hp_features(FeatArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float dt = (float)*a.d_dt;
    const float h = a.h[i];
    const BoxDev g = a.bxs[a.nb == 1 ? 0 : hp_box_of_slot(i, a.bxs, a.nb)];
    int count;
    float side;
    if (a.adaptive) {
        const int l = a.leaf_of[i];
        const int2 r = a.leaf_rng[l];
        count = r.y - r.x;
        side = ldexpf(g.L32, -a.nodes[a.leaf_node[l]].level);
    } else {
        const int c = (int)(a.keys[i] >> 3);
        count = a.cell_start[c + 1] - a.cell_start[c];
        side = g.L32;
    }
    const float N = a.n_ngb_target;
    const float hc = cbrtf(3.f * N / (4.f * 3.14159265f * (float)count)) * side;
    float *f = a.feats + (size_t)6 * i;
    f[0] = dt * a.divv[i];
    f[1] = logf(fmaxf((float)a.n_ngb[i], 1.f) / N);
    f[2] = logf(hc / h);
    f[3] = logf((float)count / N);
    f[4] = logf(h / side);
    f[5] = dt * a.vsig[i] / h;
    a.h_prev[i] = h;
}

// ------------------------------------------------------------------ inference

struct ApplyArgs {
    const float *feats;     // n x 6
    const uint16_t *wbf;    // BF16 weights (kNBf)
    const float *params;    // FP32 biases (b1, b2, b3 at their offsets)
    const float *norm;      // kNNorm
    const float *h_prev;    // n (nullptr: write log-ratios to out)
    float *out;             // n: h0, or the log-ratio
    int n;
    float log_lo, log_hi;   // clamp of log(h0 / h_prev)
    unsigned long long *err;  // set to 1 if a tensor-core wait ran out
};

// One CTA of 4 warps takes tiles of 128 particles, the M of the MMAs.  Tensor memory
// holds the FP32 accumulator, 64 columns: lane r = particle r of the tile, layer 2
// reusing layer 1's columns once its epilogue has read them; warp w reads lanes
// 32w..32w+31, so that in the epilogues every thread owns one particle.  64 columns
// and ~27 KB of shared memory (the features share the buffer of the layer-2
// operand) let 8 CTAs share an SM, whose epilogues hide one another's MMA and
// barrier latencies.  One thread issues the MMAs:
//   layer 1  D1[128 x 64] = Z[128 x 16] W1^T      (one MMA, K = 16: 6 features, zeros)
//   layer 2  D2[128 x 64] = S1[128 x 64] W2^T     (four MMAs, K = 16 each, accumulating)
// with S1 = bf16(silu(D1 + b1)) written back to shared memory by the epilogue of
// layer 1, and y = w3 . silu(D2 + b2) + b3 in the epilogue of layer 2.
constexpr int kTcM = 128, kTcThreads = 128, kTcCols = 64, kTcPerSm = 8;
constexpr int kTcSpin = 1 << 22;  // mbarrier polls before a wait counts as run out

// Operands in shared memory, K-major, no swizzle: 8-row x 16-byte core matrices of
// 128 contiguous bytes, row r at byte 16 (r % 8); element (r, k) of a matrix with kc
// core matrices per 8-row group at ((r / 8) kc + k / 8) 128 + (r % 8) 16 + (k % 8) 2.
// Descriptor strides: next core matrix along K 128 bytes (leading byte offset),
// next 8-row group kc x 128 bytes (stride byte offset).
__device__ __forceinline__ uint32_t canon_off(int r, int k, int kc)
{
    return (uint32_t)((((r >> 3) * kc + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte offset >> 4
// (16-29), stride byte offset >> 4 (32-45), the fixed 0b001 of this descriptor
// version (46-48), base offset 0, swizzle none (61-63 = 0)
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// BF16 (7-9 = 1, 10-12 = 1), both K-major (15, 16 = 0), N >> 3 (17-22), M >> 4 (24-28)
constexpr uint32_t kIdescM128N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(accumulate), "r"(kIdescM128N64));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// bounded wait on an mbarrier phase; false if it ran out
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (int it = 0; it < kTcSpin; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of this warp's 32 lanes (one per thread), waited for
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kTcThreads) k_hp_apply(ApplyArgs a)
{
    // layer-1 activations; its first 4 KB hold the normalised features (K = 16) until
    // the layer-1 MMA has read them
    __shared__ __align__(1024) uint8_t sA2[kTcM * kHid * 2];
    uint8_t *const sA1 = sA2;
    __shared__ __align__(1024) uint8_t sB1[kHid * 16 * 2];   // W1 (out x in), in padded to 16
    __shared__ __align__(1024) uint8_t sB2[kHid * kHid * 2]; // W2 (out x in)
    __shared__ float sW3[kHid], sB1v[kHid], sB2v[kHid], sNorm[kNNorm];
    __shared__ __align__(8) uint64_t sBar;
    __shared__ uint32_t sTmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const __nv_bfloat16 *wb = reinterpret_cast<const __nv_bfloat16 *>(a.wbf);
    // weights into the canonical layouts (zero padding), biases, normalisation
    for (int e = tid; e < kHid * 16; e += kTcThreads) {
        const int o = e >> 4, k = e & 15;
        const __nv_bfloat16 v = k < kW1Row ? wb[kBfW1 + o * kW1Row + k] : __float2bfloat16_rn(0.f);
        *reinterpret_cast<__nv_bfloat16 *>(sB1 + canon_off(o, k, 2)) = v;
    }
    for (int e = tid; e < kHid * kHid; e += kTcThreads) {
        const int o = e >> 6, k = e & 63;
        *reinterpret_cast<__nv_bfloat16 *>(sB2 + canon_off(o, k, 8)) = wb[kBfW2 + o * kW2Row + k];
    }
    for (int k = tid; k < kHid; k += kTcThreads) {
        sW3[k] = __bfloat162float(wb[kBfW3 + k]);
        sB1v[k] = a.params[kOffB1 + k];
        sB2v[k] = a.params[kOffB2 + k];
    }
    if (tid < kNNorm) sNorm[tid] = a.norm[tid];
    const uint32_t bar = smem_u32(&sBar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {  // tensor memory: 64 columns x 128 lanes of FP32
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sTmem)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    async_proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sTmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;  // this warp's TMEM lanes
    const float b3 = a.params[kOffB3];
    const uint32_t a1 = smem_u32(sA1), a2 = smem_u32(sA2), b1 = smem_u32(sB1), b2 = smem_u32(sB2);
    uint32_t parity = 0u;
    bool ok = true;
    const int ntile = (a.n + kTcM - 1) / kTcM;
    for (int tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
        const int p = tile * kTcM + tid;  // this thread's particle (row tid of the tile)
        // layer-1 operand: (f - mean) / sd in BF16, columns 6-15 zero
        {
            __nv_bfloat16 z[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) z[k] = __float2bfloat16_rn(0.f);
            if (p < a.n) {
#pragma unroll
                for (int k = 0; k < kF; ++k)
                    z[k] = __float2bfloat16_rn((a.feats[(size_t)kF * p + k] - sNorm[k]) * (1.f / sNorm[kF + k]));
            }
            *reinterpret_cast<uint4 *>(sA1 + canon_off(tid, 0, 2)) = *reinterpret_cast<const uint4 *>(&z[0]);
            *reinterpret_cast<uint4 *>(sA1 + canon_off(tid, 8, 2)) = *reinterpret_cast<const uint4 *>(&z[8]);
        }
        async_proxy_fence();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            umma_bf16(tmem, umma_sdesc(a1, 128, 256), umma_sdesc(b1, 128, 256), 0u);
            umma_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait(bar, parity)) != 0;
        parity ^= 1u;
        if (!ok) break;
        tc_fence_after();
        // epilogue 1: bias, SiLU, BF16 -> the layer-2 operand
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)(32 * h), v);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                __nv_bfloat16 s8[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int j = 32 * h + 8 * c + e;
                    s8[e] = __float2bfloat16_rn(silu_fast(v[8 * c + e] + sB1v[j]));
                }
                *reinterpret_cast<uint4 *>(sA2 + canon_off(tid, 32 * h + 8 * c, 8)) =
                    *reinterpret_cast<const uint4 *>(s8);
            }
        }
        async_proxy_fence();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)  // K = 16 per MMA: two core matrices along K
                umma_bf16(tmem, umma_sdesc(a2 + 256 * kk, 128, 1024), umma_sdesc(b2 + 256 * kk, 128, 1024),
                          kk > 0 ? 1u : 0u);
            umma_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait(bar, parity)) != 0;
        parity ^= 1u;
        if (!ok) break;
        tc_fence_after();
        // epilogue 2: bias, SiLU, dot with W3 (FP32), de-normalise, clamp
        float s = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)(32 * h), v);
#pragma unroll
            for (int e = 0; e < 32; ++e) s = fmaf(silu_fast(v[e] + sB2v[32 * h + e]), sW3[32 * h + e], s);
        }
        if (p < a.n) {
            const float y = fminf(fmaxf((s + b3) * sNorm[2 * kF + 1] + sNorm[2 * kF], a.log_lo), a.log_hi);
            a.out[p] = a.h_prev ? a.h_prev[p] * __expf(y) : y;
        }
        tc_fence_before();
        __syncthreads();  // every lane read its columns before the next tile's MMAs
    }
    if (!ok) {
        if (tid == 0) atomicOr(a.err, 1ull);
        // an MMA may still be in flight: give it one more bounded wait before the
        // tensor memory is released
        __syncthreads_and(mbar_wait(bar, parity ^ 1u));
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// FP32 parameters -> BF16 inference copy (padding zero)
__global__ void k_hp_to_bf16(const float *__restrict__ P, uint16_t *__restrict__ wbf)
{
    __nv_bfloat16 *w = reinterpret_cast<__nv_bfloat16 *>(wbf);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kNBf; k += gridDim.x * blockDim.x) {
        float v = 0.f;
        if (k < kBfW2) {
            const int o = k / kW1Row, i = k % kW1Row;
            if (i < kF) v = P[kOffW1 + o * kF + i];
        } else if (k < kBfW3) {
            const int o = (k - kBfW2) / kW2Row, i = (k - kBfW2) % kW2Row;
            if (i < kHid) v = P[kOffW2 + o * kHid + i];
        } else {
            v = P[kOffW3 + (k - kBfW3)];
        }
        w[k] = __float2bfloat16_rn(v);
    }
}

// ------------------------------------------------------------------ training

// uniform in [0, 1) from a counter (splitmix64)
__device__ __forceinline__ float hp_uniform(uint64_t seed, uint64_t k)
{
    return (float)(mix64(seed ^ (k * 0x9E3779B97F4A7C15ull)) >> 40) * (1.f / 16777216.f);
}

// Glorot-uniform weights, zero biases
__global__ void k_hp_init(float *P, uint64_t seed)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kNParam; k += gridDim.x * blockDim.x) {
        float lim = 0.f;
        if (k < kOffB1) lim = sqrtf(6.f / (kF + kHid));
        else if (k >= kOffW2 && k < kOffB2) lim = sqrtf(6.f / (kHid + kHid));
        else if (k >= kOffW3 && k < kOffB3) lim = sqrtf(6.f / (kHid + 1));
        P[k] = lim > 0.f ? (2.f * hp_uniform(seed, (uint64_t)k) - 1.f) * lim : 0.f;
    }
}

// FP64 sums of every feature and of the target and of their squares (fixed grid,
// then fixed-order final sum): means and standard deviations for the normalisation
constexpr int kStatBlocks = 152;
__global__ void k_hp_stats_part(const float *__restrict__ X, const float *__restrict__ Y, int64_t n,
                                double *__restrict__ part)
{
    double s[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) s[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int f = 0; f < kF; ++f) {
            const double v = X[6 * i + f];
            s[f] += v;
            s[7 + f] += v * v;
        }
        const double y = Y[i];
        s[6] += y;
        s[13] += y * y;
    }
    __shared__ double sh[14][256];
#pragma unroll
    for (int k = 0; k < 14; ++k) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 14; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 14) part[threadIdx.x * kStatBlocks + blockIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_hp_stats_final(const double *__restrict__ part, int64_t n, float *__restrict__ norm)
{
    const int k = threadIdx.x;  // 0..6: features 0..5, target
    if (k >= 7) return;
    double s = 0.0, q = 0.0;
    for (int b = 0; b < kStatBlocks; ++b) {
        s += part[k * kStatBlocks + b];
        q += part[(7 + k) * kStatBlocks + b];
    }
    const double m = s / (double)n;
    double var = q / (double)n - m * m;
    const double sd = sqrt(fmax(var, 0.0));
    const float sdf = sd > 1e-12 ? (float)sd : 1.f;  // a constant input: unit scale
    if (k < kF) {
        norm[k] = (float)m;
        norm[kF + k] = sdf;
    } else {
        norm[2 * kF] = (float)m;
        norm[2 * kF + 1] = sdf;
    }
}

struct TrainArgs {
    const float *X;   // n x 6 raw features
    const float *Y;   // n raw targets
    int64_t n;
    const float *P;   // parameters
    const float *norm;
    float *gpart;     // [kTrBlocks][kNParam + 1]: partial gradients, then the loss
    int64_t step;     // Adam step index (samples of this step: step * kTrBatch + k)
    uint64_t seed;    // 0: sequential samples, else hashed
};

// one Adam step's gradients: every block takes kTrSub tiles of kTrS samples
__global__ void __launch_bounds__(kTrThreads) k_hp_train_grad(TrainArgs a)
{
    extern __shared__ float sm[];
    float *sP = sm;                    // parameters
    float *sG = sP + kNParam;          // gradient accumulators
    float *X = sG + kNParam;           // [kTrS][kF]
    float *Z1 = X + kTrS * kF;         // [kTrS][kHid]
    float *H1 = Z1 + kTrS * kHid;
    float *Z2 = H1 + kTrS * kHid;
    float *D = Z2 + kTrS * kHid;       // dL/dZ2, then dL/dZ1 (in Z2's place)
    float *dy = D + kTrS * kHid;       // [kTrS]
    float *tg = dy + kTrS;             // [kTrS] normalised targets
    __shared__ float s_loss[kTrThreads];
    const int tid = threadIdx.x;
    for (int k = tid; k < kNParam; k += kTrThreads) {
        sP[k] = a.P[k];
        sG[k] = 0.f;
    }
    float loss = 0.f;
    const float inv_batch = 1.f / (float)kTrBatch;
    __syncthreads();
    for (int sub = 0; sub < kTrSub; ++sub) {
        // samples
        if (tid < kTrS) {
            const uint64_t ctr = (uint64_t)a.step * kTrBatch + ((uint64_t)blockIdx.x * kTrSub + sub) * kTrS + tid;
            const int64_t idx = a.seed == 0 ? (int64_t)(ctr % (uint64_t)a.n)
                                             : (int64_t)(mix64(a.seed ^ (ctr * 0xD1B54A32D192ED03ull)) % (uint64_t)a.n);
            for (int f = 0; f < kF; ++f) X[tid * kF + f] = (a.X[6 * idx + f] - a.norm[f]) / a.norm[kF + f];
            tg[tid] = (a.Y[idx] - a.norm[2 * kF]) / a.norm[2 * kF + 1];
        }
        __syncthreads();
        // layer 1
        for (int e = tid; e < kTrS * kHid; e += kTrThreads) {
            const int s = e / kHid, u = e % kHid;
            float z = sP[kOffB1 + u];
            for (int f = 0; f < kF; ++f) z = fmaf(sP[kOffW1 + u * kF + f], X[s * kF + f], z);
            Z1[e] = z;
            H1[e] = silu(z);
        }
        __syncthreads();
        // layer 2
        for (int e = tid; e < kTrS * kHid; e += kTrThreads) {
            const int s = e / kHid, u = e % kHid;
            float z = sP[kOffB2 + u];
            for (int v = 0; v < kHid; ++v) z = fmaf(sP[kOffW2 + u * kHid + v], H1[s * kHid + v], z);
            Z2[e] = z;
        }
        __syncthreads();
        // output and its error (mean over the whole batch)
        if (tid < kTrS) {
            float y = sP[kOffB3];
            for (int u = 0; u < kHid; ++u) y = fmaf(sP[kOffW3 + u], silu(Z2[tid * kHid + u]), y);
            const float r = y - tg[tid];
            dy[tid] = 2.f * r * inv_batch;
            loss = fmaf(r, r, loss);
        }
        __syncthreads();
        // dW3, db3
        if (tid < kHid) {
            float gsum = 0.f;
            for (int s = 0; s < kTrS; ++s) gsum = fmaf(dy[s], silu(Z2[s * kHid + tid]), gsum);
            sG[kOffW3 + tid] += gsum;
        }
        if (tid == kHid) {
            float gsum = 0.f;
            for (int s = 0; s < kTrS; ++s) gsum += dy[s];
            sG[kOffB3] += gsum;
        }
        // dL/dZ2
        for (int e = tid; e < kTrS * kHid; e += kTrThreads) {
            const int s = e / kHid, u = e % kHid;
            D[e] = dy[s] * sP[kOffW3 + u] * silu_grad(Z2[e]);
        }
        __syncthreads();
        // dW2 (each thread owns 16 entries), db2
        for (int e = tid; e < kHid * kHid; e += kTrThreads) {
            const int u = e / kHid, v = e % kHid;
            float gsum = 0.f;
            for (int s = 0; s < kTrS; ++s) gsum = fmaf(D[s * kHid + u], H1[s * kHid + v], gsum);
            sG[kOffW2 + e] += gsum;
        }
        if (tid < kHid) {
            float gsum = 0.f;
            for (int s = 0; s < kTrS; ++s) gsum += D[s * kHid + tid];
            sG[kOffB2 + tid] += gsum;
        }
        // dL/dZ1 into Z2's place
        for (int e = tid; e < kTrS * kHid; e += kTrThreads) {
            const int s = e / kHid, v = e % kHid;
            float gsum = 0.f;
            for (int u = 0; u < kHid; ++u) gsum = fmaf(D[s * kHid + u], sP[kOffW2 + u * kHid + v], gsum);
            Z2[e] = gsum * silu_grad(Z1[e]);
        }
        __syncthreads();
        // dW1, db1
        for (int e = tid; e < kHid * kF; e += kTrThreads) {
            const int v = e / kF, f = e % kF;
            float gsum = 0.f;
            for (int s = 0; s < kTrS; ++s) gsum = fmaf(Z2[s * kHid + v], X[s * kF + f], gsum);
            sG[kOffW1 + e] += gsum;
        }
        if (tid < kHid) {
            float gsum = 0.f;
            for (int s = 0; s < kTrS; ++s) gsum += Z2[s * kHid + tid];
            sG[kOffB1 + tid] += gsum;
        }
        __syncthreads();
    }
    float *out = a.gpart + (size_t)blockIdx.x * (kNParam + 1);
    for (int k = tid; k < kNParam; k += kTrThreads) out[k] = sG[k];
    s_loss[tid] = loss;
    __syncthreads();
    if (tid == 0) {
        float l = 0.f;
        for (int k = 0; k < kTrS; ++k) l += s_loss[k];
        out[kNParam] = l;
    }
}

// fixed-order sum of the block partials, then Adam (t = step + 1); loss of the step
__global__ void k_hp_adam(const float *__restrict__ gpart, float *__restrict__ P, float *__restrict__ m,
                          float *__restrict__ v, int64_t step, float lr, float *__restrict__ loss_out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > kNParam) return;
    float g = 0.f;
    for (int b = 0; b < kTrBlocks; ++b) g += gpart[(size_t)b * (kNParam + 1) + k];
    if (k == kNParam) {
        *loss_out = g / (float)kTrBatch;
        return;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mk = b1 * m[k] + (1.f - b1) * g;
    const float vk = b2 * v[k] + (1.f - b2) * g * g;
    m[k] = mk;
    v[k] = vk;
    const double t = (double)(step + 1);
    const float c1 = (float)(1.0 - pow((double)b1, t)), c2 = (float)(1.0 - pow((double)b2, t));
    P[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// ------------------------------------------------------------------ host side

static int hp_alloc(sph_ctx *ctx)
{
    HPredictor &H = ctx->hp;
    if (H.params) return SPH_OK;
    SPH_CUDA(ctx, cudaMalloc(&H.params, sizeof(float) * kNParam));
    SPH_CUDA(ctx, cudaMalloc(&H.adam_m, sizeof(float) * kNParam));
    SPH_CUDA(ctx, cudaMalloc(&H.adam_v, sizeof(float) * kNParam));
    SPH_CUDA(ctx, cudaMalloc(&H.norm, sizeof(float) * kNNorm));
    SPH_CUDA(ctx, cudaMalloc(&H.wbf, sizeof(uint16_t) * kNBf));
    SPH_CUDA(ctx, cudaMalloc(&H.gpart, sizeof(float) * kTrBlocks * (kNParam + 1)));
    SPH_CUDA(ctx, cudaMalloc(&H.stat_part, sizeof(double) * 14 * kStatBlocks));
    SPH_CUDA(ctx, cudaMalloc(&H.d_loss, sizeof(float)));
    SPH_CUDA(ctx, cudaMallocHost(&H.h_loss, sizeof(float)));
    SPH_CUDA(ctx, cudaMemsetAsync(H.adam_m, 0, sizeof(float) * kNParam, ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(H.adam_v, 0, sizeof(float) * kNParam, ctx->stream));
    return SPH_OK;
}

static int hp_refresh_bf16(sph_ctx *ctx)
{
    k_hp_to_bf16<<<(kNBf + 255) / 256, 256, 0, ctx->stream>>>(ctx->hp.params, ctx->hp.wbf);
    SPH_LAUNCH(ctx, "predictor bf16 copy");
    return SPH_OK;
}

int hp_init(sph_ctx *ctx, uint64_t seed)
{
    int rc = hp_alloc(ctx);
    if (rc) return rc;
    HPredictor &H = ctx->hp;
    k_hp_init<<<(kNParam + 255) / 256, 256, 0, ctx->stream>>>(H.params, seed);
    SPH_LAUNCH(ctx, "predictor init");
    const float norm[kNNorm] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 0, 1};
    memcpy(H.h_norm.data(), norm, sizeof norm);
    SPH_CUDA(ctx, cudaMemcpyAsync(H.norm, H.h_norm.data(), sizeof norm, cudaMemcpyHostToDevice, ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(H.adam_m, 0, sizeof(float) * kNParam, ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(H.adam_v, 0, sizeof(float) * kNParam, ctx->stream));
    H.adam_t = 0;
    H.norm_set = false;
    H.ready = true;
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // h_norm is read by the copy
    return hp_refresh_bf16(ctx);
}

int hp_load(sph_ctx *ctx, const uint16_t *w_bf16, const float *f32)
{
    int rc = hp_alloc(ctx);
    if (rc) return rc;
    HPredictor &H = ctx->hp;
    // BF16 weights -> FP32 parameters (exact), FP32 biases and normalisation
    float *P = H.h_params.data();
    auto bf = [](uint16_t b) {
        uint32_t u = (uint32_t)b << 16;
        float f;
        memcpy(&f, &u, 4);
        return f;
    };
    for (int k = 0; k < kHid * kF; ++k) P[kOffW1 + k] = bf(w_bf16[k]);
    for (int k = 0; k < kHid * kHid; ++k) P[kOffW2 + k] = bf(w_bf16[kHid * kF + k]);
    for (int k = 0; k < kHid; ++k) P[kOffW3 + k] = bf(w_bf16[kHid * kF + kHid * kHid + k]);
    for (int k = 0; k < kHid; ++k) P[kOffB1 + k] = f32[k];
    for (int k = 0; k < kHid; ++k) P[kOffB2 + k] = f32[kHid + k];
    P[kOffB3] = f32[2 * kHid];
    for (int k = 0; k < kNNorm; ++k) H.h_norm[k] = f32[2 * kHid + 1 + k];
    for (int k = 0; k < kF; ++k)
        if (!(H.h_norm[kF + k] > 0.f)) return fail(ctx, SPH_ERR_INVALID_ARG, "feature scales must be > 0");
    if (!(H.h_norm[2 * kF + 1] > 0.f)) return fail(ctx, SPH_ERR_INVALID_ARG, "target scale must be > 0");
    SPH_CUDA(ctx, cudaMemcpyAsync(H.params, P, sizeof(float) * kNParam, cudaMemcpyHostToDevice, ctx->stream));
    SPH_CUDA(ctx, cudaMemcpyAsync(H.norm, H.h_norm.data(), sizeof(float) * kNNorm, cudaMemcpyHostToDevice,
                                  ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(H.adam_m, 0, sizeof(float) * kNParam, ctx->stream));
    SPH_CUDA(ctx, cudaMemsetAsync(H.adam_v, 0, sizeof(float) * kNParam, ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    H.adam_t = 0;
    H.norm_set = true;
    H.ready = true;
    return hp_refresh_bf16(ctx);
}

int hp_save(sph_ctx *ctx, uint16_t *w_bf16, float *f32)
{
    HPredictor &H = ctx->hp;
    if (!H.ready) return fail(ctx, SPH_ERR_STATE, "no predictor weights (init, load or train first)");
    uint16_t *wb = H.h_wbf.data();
    SPH_CUDA(ctx, cudaMemcpyAsync(wb, H.wbf, sizeof(uint16_t) * kNBf, cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaMemcpyAsync(H.h_params.data(), H.params, sizeof(float) * kNParam, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    SPH_CUDA(ctx, cudaMemcpyAsync(H.h_norm.data(), H.norm, sizeof(float) * kNNorm, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int o = 0; o < kHid; ++o)
        for (int i = 0; i < kF; ++i) w_bf16[o * kF + i] = wb[kBfW1 + o * kW1Row + i];
    for (int o = 0; o < kHid; ++o)
        for (int i = 0; i < kHid; ++i) w_bf16[kHid * kF + o * kHid + i] = wb[kBfW2 + o * kW2Row + i];
    for (int k = 0; k < kHid; ++k) w_bf16[kHid * kF + kHid * kHid + k] = wb[kBfW3 + k];
    for (int k = 0; k < kHid; ++k) f32[k] = H.h_params[kOffB1 + k];
    for (int k = 0; k < kHid; ++k) f32[kHid + k] = H.h_params[kOffB2 + k];
    f32[2 * kHid] = H.h_params[kOffB3];
    for (int k = 0; k < kNNorm; ++k) f32[2 * kHid + 1 + k] = H.h_norm[k];
    return SPH_OK;
}

int hp_params(sph_ctx *ctx, float *out)
{
    HPredictor &H = ctx->hp;
    if (!H.ready) return fail(ctx, SPH_ERR_STATE, "no predictor weights (init, load or train first)");
    SPH_CUDA(ctx, cudaMemcpyAsync(H.h_params.data(), H.params, sizeof(float) * kNParam, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    memcpy(out, H.h_params.data(), sizeof(float) * kNParam);
    return SPH_OK;
}

int hp_ensure(sph_ctx *ctx, int64_t n)
{
    HPredictor &H = ctx->hp;
    if (n <= H.cap) return SPH_OK;
    cudaFree(H.feats);
    cudaFree(H.h_prev);
    H.feats = H.h_prev = nullptr;
    H.cap = 0;
    SPH_CUDA(ctx, cudaMalloc(&H.feats, sizeof(float) * 6 * n));
    SPH_CUDA(ctx, cudaMalloc(&H.h_prev, sizeof(float) * n));
    H.cap = n;
    return SPH_OK;
}

// features of the current (built) state into ctx->hp.feats, h into ctx->hp.h_prev
int hp_features(sph_ctx *ctx, sph_particles *parts)
{
    const int n = (int)ctx->n;
    int rc = hp_ensure(ctx, std::max(n, 1));
    if (rc) return rc;
    if (!ctx->built) return fail(ctx, SPH_ERR_STATE, "predictor features need a cell build");
    if (n <= 0) return SPH_OK;
    FeatArgs a;
    memset(&a, 0, sizeof a);
    a.h = parts->h;
    a.divv = parts->divv;
    a.vsig = parts->vsig;
    a.n_ngb = parts->n_ngb;
    a.d_dt = ctx->d_dt;
    a.keys = ctx->keys;
    a.cell_start = ctx->cell_start;
    a.leaf_of = ctx->tree.leaf_of;
    a.leaf_rng = ctx->tree.leaf_rng;
    a.leaf_node = ctx->tree.leaf_node;
    a.nodes = ctx->tree.nodes;
    a.bxs = ctx->d_boxes;
    a.nb = ctx->n_boxes;
    a.n = n;
    a.adaptive = ctx->adaptive ? 1 : 0;
    a.n_ngb_target = ctx->p.n_ngb;
    a.feats = ctx->hp.feats;
    a.h_prev = ctx->hp.h_prev;
    k_hp_features<<<(n + 255) / 256, 256, 0, ctx->stream>>>(a);
    SPH_LAUNCH(ctx, "predictor features");
    return SPH_OK;
}

// persistent grid: at most 8 CTAs per SM (8 x 64 of the 512 tensor-memory columns)
static int hp_grid(sph_ctx *ctx, int64_t n)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (sms <= 0) sms = 148;
    const int64_t want = (n + kTcM - 1) / kTcM;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * kTcPerSm));
}

// MLP on arbitrary features: out = log-ratio (h_prev null) or h_prev * exp(log-ratio)
int hp_run(sph_ctx *ctx, const float *feats, const float *h_prev, float *out, int64_t n, float log_lo, float log_hi)
{
    if (!ctx->hp.ready) return fail(ctx, SPH_ERR_STATE, "no predictor weights (init, load or train first)");
    if (n <= 0) return SPH_OK;
    ApplyArgs a{feats, ctx->hp.wbf, ctx->hp.params, ctx->hp.norm, h_prev, out, (int)n, log_lo, log_hi,
                ctx->counters + C_TCERR};
    k_hp_apply<<<hp_grid(ctx, n), kTcThreads, 0, ctx->stream>>>(a);
    SPH_LAUNCH(ctx, "predictor mlp");
    // outside a capture the run-out flag is read here; captured steps fold it into
    // the step flags
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SPH_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
        SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_counters + C_TCERR, ctx->counters + C_TCERR, sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, ctx->stream));
        SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->h_counters[C_TCERR]) return fail(ctx, SPH_ERR_TIMEOUT, "predictor: a tensor-core wait ran out");
    }
    return SPH_OK;
}

// inside a step, after the build: features, then h <- h_prev * exp(prediction)
int hp_apply_step(sph_ctx *ctx, sph_particles *parts)
{
    int rc = hp_features(ctx, parts);
    if (rc) return rc;
    // growth is capped so that h stays within what the cells (lists) were built for
    const float g_max = ctx->adaptive ? std::min(std::min(1.2f, ctx->p.cell_factor), kTreeReach) : 1.2f;
    return hp_run(ctx, ctx->hp.feats, ctx->hp.h_prev, parts->h, ctx->n, logf(0.5f), logf(g_max));
}

__global__ void k_hp_target(const float *__restrict__ h, const float *__restrict__ h_prev, int n, float *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = logf(h[i] / h_prev[i]);
}

int hp_targets(sph_ctx *ctx, sph_particles *parts, float *dev_target)
{
    const int n = (int)ctx->n;
    if (n <= 0) return SPH_OK;
    if (ctx->hp.cap < n) return fail(ctx, SPH_ERR_STATE, "no predictor features for this state");
    k_hp_target<<<(n + 255) / 256, 256, 0, ctx->stream>>>(parts->h, ctx->hp.h_prev, n, dev_target);
    SPH_LAUNCH(ctx, "predictor targets");
    return SPH_OK;
}

// append this step's (features, target) pairs to the caller's collection buffers
int hp_collect(sph_ctx *ctx, sph_particles *parts)
{
    HPredictor &H = ctx->hp;
    const int64_t n = ctx->n;
    if (!H.col_feats || n <= 0 || H.col_n + n > H.col_cap) return SPH_OK;
    SPH_CUDA(ctx, cudaMemcpyAsync(H.col_feats + 6 * H.col_n, H.feats, sizeof(float) * 6 * n,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
    int rc = hp_targets(ctx, parts, H.col_target + H.col_n);
    if (rc) return rc;
    H.col_n += n;
    return SPH_OK;
}

static int hp_smem_optin(sph_ctx *ctx, size_t bytes)
{
    static bool done = false;
    if (done) return SPH_OK;
    SPH_CUDA(ctx, cudaFuncSetAttribute(k_hp_train_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done = true;
    return SPH_OK;
}

int hp_train(sph_ctx *ctx, const float *X, const float *Y, int64_t n, int epochs, float lr, uint64_t seed,
             float *loss_out)
{
    if (!ctx->hp.ready) {
        int rc = hp_init(ctx, seed ? seed : 1);
        if (rc) return rc;
    }
    HPredictor &H = ctx->hp;
    if (!H.norm_set) {  // normalisation from this training set
        k_hp_stats_part<<<kStatBlocks, 256, 0, ctx->stream>>>(X, Y, n, H.stat_part);
        SPH_LAUNCH(ctx, "predictor stats");
        k_hp_stats_final<<<1, 32, 0, ctx->stream>>>(H.stat_part, n, H.norm);
        SPH_LAUNCH(ctx, "predictor stats final");
        H.norm_set = true;
    }
    const size_t smem = sizeof(float) * (2 * kNParam + kTrS * kF + 4 * kTrS * kHid + 2 * kTrS);
    int rc = hp_smem_optin(ctx, smem);
    if (rc) return rc;
    const int64_t steps_per_epoch = (n + kTrBatch - 1) / kTrBatch;
    for (int e = 0; e < epochs; ++e)
        for (int64_t s = 0; s < steps_per_epoch; ++s) {
            TrainArgs a{X, Y, n, H.params, H.norm, H.gpart, H.adam_t, seed};
            k_hp_train_grad<<<kTrBlocks, kTrThreads, smem, ctx->stream>>>(a);
            SPH_LAUNCH(ctx, "predictor gradients");
            k_hp_adam<<<(kNParam + 1 + 255) / 256, 256, 0, ctx->stream>>>(H.gpart, H.params, H.adam_m, H.adam_v,
                                                                         H.adam_t, lr, H.d_loss);
            SPH_LAUNCH(ctx, "predictor adam");
            ++H.adam_t;
        }
    rc = hp_refresh_bf16(ctx);
    if (rc) return rc;
    SPH_CUDA(ctx, cudaMemcpyAsync(H.h_loss, H.d_loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (loss_out) *loss_out = *H.h_loss;
    return SPH_OK;
}

void hp_free(sph_ctx *ctx)
{
    HPredictor &H = ctx->hp;
    void *d[] = {H.params, H.adam_m, H.adam_v, H.norm, H.wbf, H.gpart, H.stat_part, H.d_loss, H.feats, H.h_prev};
    for (void *p : d) cudaFree(p);
    cudaFreeHost(H.h_loss);
    H = HPredictor();
}

static_assert(kNParam == 4673 && kNNorm == 14 && kNBf == 5184, "host copies in HPredictor are sized for these");

}  // namespace sph
