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
// comes from.

__device__ __forceinline__ int64_t bin_len(int L, int b) { return (int64_t)1 << (L - b); }

// act[i] = the particle's step ends at integer time s; counts them
__global__ void k_bin_active(const int8_t *__restrict__ bins, int n, int64_t s, int L, uint8_t *__restrict__ act,
                             unsigned long long *count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool a = false;
    if (i < n) {
        a = (s & (bin_len(L, bins[i]) - 1)) == 0;
        act[i] = a ? 1 : 0;
    }
    unsigned m = __ballot_sync(kFull, a);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(count, (unsigned long long)__popc(m));
}

// half kick of the active particles (all of them if act is null) over their own
// step: v += a dt_b/2 (FP64); u <- max(u + dudt dt_b/2, 0), counting floors.  The
// arithmetic is k_kick's with dt = 2^(L-b) unit.
__global__ void k_bin_kick(sph_particles P, int n, const int8_t *__restrict__ bins, const uint8_t *__restrict__ act,
                           int L, double unit, unsigned long long *floors)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool fl = false;
    if (i < n && (act == nullptr || act[i])) {
        const double half_dt = 0.5 * ((double)bin_len(L, bins[i]) * unit);
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

// deepest bin over all particles
__global__ void k_bin_max(const int8_t *__restrict__ bins, int n, unsigned long long *out)
{
    unsigned m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = max(m, (unsigned)bins[i]);
    m = __reduce_max_sync(kFull, m);
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)m);
}

// The cell build permutes the particle arrays it knows; the density outputs that
// inactive particles keep (rho, P, c, f, |curl v|), their bins and active flags
// follow the same permutation here (slot p takes what slot perm[p] held).
__global__ void k_bin_gather(const uint32_t *__restrict__ perm, int n, sph_particles P,
                             const int8_t *__restrict__ bins, const uint8_t *__restrict__ act, float *__restrict__ s32,
                             int64_t cap, int8_t *__restrict__ bins_out, uint8_t *__restrict__ act_out)
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
}

// Copy the gathered outputs back; then, per particle, the velocity and internal
// energy predicted to the current time s (v_half + a (t - t_mid), t_mid the middle of
// the particle's own step: +dt_b/2 at the end of a step, as in the global step) and
// the packed force inputs of the density pass (rho, f P / rho^2, c, Balsara B), for
// the particles that keep their last density.
__global__ void k_bin_predict(sph_particles P, int n, const float *__restrict__ s32, int64_t cap,
                              const int8_t *__restrict__ bins, int64_t s, int L, double unit, int use_balsara,
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
    const int64_t D = bin_len(L, bins[p]);
    const int64_t r = s & (D - 1);
    const int64_t s0 = r == 0 ? s - D : s - r;  // start of the step that contains s
    const double tau = 0.5 * ((double)(2 * (s - s0) - D) * unit);
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
                                                           ctx->bin_s32, ctx->bin_cap, ctx->bins_tmp,
                                                           ctx->bin_active_tmp);
    SPH_LAUNCH(ctx, "bin gather");
    std::swap(ctx->bins, ctx->bins_tmp);
    std::swap(ctx->bin_active, ctx->bin_active_tmp);
    k_bin_predict<<<(n + 255) / 256, 256, 0, ctx->stream>>>(*parts, n, ctx->bin_s32, ctx->bin_cap, ctx->bins,
                                                            ctx->bin_now, ctx->bin_levels, ctx->bin_unit,
                                                            ctx->p.use_balsara, ctx->vel4, ctx->upred, ctx->thermo4);
    SPH_LAUNCH(ctx, "bin predict");
    return SPH_OK;
}

int bin_active(sph_ctx *ctx, unsigned long long *n_active)
{
    const int n = (int)ctx->n;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_BINACT, 0, sizeof(unsigned long long), ctx->stream));
    if (n > 0) {
        k_bin_active<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->bins, n, ctx->bin_now, ctx->bin_levels,
                                                               ctx->bin_active, ctx->counters + C_BINACT);
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
    k_bin_kick<<<(n + 255) / 256, 256, 0, ctx->stream>>>(*parts, n, ctx->bins, all ? nullptr : ctx->bin_active,
                                                         ctx->bin_levels, ctx->bin_unit, ctx->counters + C_FLOORS);
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

int bin_max_read(sph_ctx *ctx, int *max_bin, unsigned long long *over)
{
    const int n = (int)ctx->n;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->counters + C_BINMAX, 0, sizeof(unsigned long long), ctx->stream));
    if (n > 0) {
        k_bin_max<<<kRedBlocks, kRedThreads, 0, ctx->stream>>>(ctx->bins, n, ctx->counters + C_BINMAX);
        SPH_LAUNCH(ctx, "bin max");
    }
    SPH_CUDA(ctx, cudaMemcpyAsync(ctx->h_counters + C_BINMAX, ctx->counters + C_BINMAX,
                                  2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
    SPH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *max_bin = (int)ctx->h_counters[C_BINMAX];
    *over = ctx->h_counters[C_BINOVER];
    return SPH_OK;
}

}  // namespace sph
