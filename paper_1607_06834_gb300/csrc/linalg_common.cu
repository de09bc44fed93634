// Rounding-independent helper kernels of the ROK step: step begin, flag set,
// and the CFL time-step bound (a max reduction, independent of order).
#include <math.h>

#include "linalg.cuh"

namespace rok {

namespace {

__device__ __forceinline__ size_t gtid() { return (size_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t gstride() { return (size_t)gridDim.x * blockDim.x; }

__global__ void begin_kernel(StepState *st, double h, double gamma, int M)
{
    st->h = h;
    st->hg = h * gamma;
    st->meff = M;
    st->active = M > 0 ? 1 : 0;
    st->beta = 0.0;
    st->wnorm0 = 0.0;
}

__global__ void begin_batch_kernel(StepState *st, const double *h, double gamma, int M, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    StepState *s = st + k;
    const double hk = h[k];
    s->h = hk;
    s->hg = hk * gamma;
    s->meff = M;
    s->active = M > 0 ? 1 : 0;
    s->beta = 0.0;
    s->wnorm0 = 0.0;
}

__global__ void clear_status_kernel(StepState *st, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) st[k].status = 0;
}

__global__ void set_int_kernel(int *p, int v) { *p = v; }

__global__ void f2d_kernel(const float *src, double *dst, size_t n)
{
    for (size_t e = gtid(); e < n; e += gstride()) dst[e] = (double)src[e];
}

__global__ void cfl_kernel(const double *y, const StencilConsts C, const double *six, const double *siy,
                           const double *sjx, const double *sjy, const double *vol, double *pmax)
{
    __shared__ double sh[32];
    const size_t nc = (size_t)C.nx * C.ny;
    const double g = C.gm1 + 1.0;
    double best = 0.0;
    for (size_t c = gtid(); c < nc; c += gstride()) {
        double rho = y[c], u = y[nc + c] / rho, v = y[2 * nc + c] / rho;
        double p = C.gm1 * (y[3 * nc + c] - 0.5 * rho * (u * u + v * v));
        double a = sqrt(g * p / rho);
        double ax, ay, bx, by, vo;
        if (six) { ax = six[c]; ay = siy[c]; bx = sjx[c]; by = sjy[c]; vo = vol[c]; }
        else { ax = 1.0 / C.rdy; ay = 0.0; bx = 0.0; by = 1.0 / C.rdx; vo = (1.0 / C.rdx) * (1.0 / C.rdy); }
        double si2 = ax * ax + ay * ay, sj2 = bx * bx + by * by;
        double lam = (fabs(u * ax + v * ay) + a * sqrt(si2)) / vo + (fabs(u * bx + v * by) + a * sqrt(sj2)) / vo;
        if (C.viscous && C.mu > 0.0) {
            double mu = C.mu;
            if (C.sutherland) {
                double t = (p / rho) * C.inv_tref;
                mu = C.mu * (t * sqrt(t)) * ((1.0 + C.suth_s) / (t + C.suth_s));
            }
            double nu = fmax(4.0 / 3.0, C.g_over_pr) * mu / rho;
            lam += 2.0 * nu * (si2 + sj2) / (vo * vo);
        }
        best = fmax(best, lam);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) sh[wid] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, sh[w]);
        pmax[blockIdx.x] = b;
    }
}

}  // namespace

cudaError_t launch_set_int(int *p, int v, cudaStream_t s)
{
    set_int_kernel<<<1, 1, 0, s>>>(p, v);
    return cudaGetLastError();
}

cudaError_t launch_f2d(const float *src, double *dst, size_t n, cudaStream_t s)
{
    f2d_kernel<<<1024, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_begin(StepState *st, double h, double gamma, int M, cudaStream_t s)
{
    begin_kernel<<<1, 1, 0, s>>>(st, h, gamma, M);
    return cudaGetLastError();
}

cudaError_t launch_begin_batch(StepState *st, const double *h, double gamma, int M, int n, cudaStream_t s)
{
    begin_batch_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, h, gamma, M, n);
    return cudaGetLastError();
}

cudaError_t launch_clear_status(StepState *st, int n, cudaStream_t s)
{
    clear_status_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, n);
    return cudaGetLastError();
}

cudaError_t launch_cfl(const double *y, const StencilConsts &c, const double *six, const double *siy,
                       const double *sjx, const double *sjy, const double *vol, double *pmax, int P,
                       cudaStream_t s)
{
    cfl_kernel<<<P, 256, 0, s>>>(y, c, six, siy, sjx, sjy, vol, pmax);
    return cudaGetLastError();
}

}  // namespace rok
