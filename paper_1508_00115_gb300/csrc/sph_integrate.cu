// sph_integrate.cu -- marching particles forward in time (Theuns et al. 2015,
// Sec. 2: "positions by velocities, velocities by accelerations") and the O(N)
// reductions around the pair passes: CFL time step and the conserved quantities.
// Positions, velocities, kicks, drifts and the global sums are FP64; the sums use a
// fixed grid and tree order, so they are deterministic.  The step's dt lives on the
// device (ctx->d_dt), so a whole step can be replayed from a CUDA graph.
#include <math.h>

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
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
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

}  // namespace sph
