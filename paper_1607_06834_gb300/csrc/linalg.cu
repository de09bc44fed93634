// Vector kernels of the ROK step: deterministic reductions (fixed grid, fixed
// per-thread order, xor-butterfly warp trees), modified-Gram-Schmidt passes of
// the Arnoldi process (Sec. 2.3.3), the projected Rosenbrock stage solves of
// Eq. ROK, stage vectors, combines, the FD increment and the CFL bound.
//
// On GB300 the FP64 pipe is the scarce unit (about two FP64 FMA per clock per
// SM), so an FP64 dot or AXPY sits close to the HBM/FP64 balance point; the
// passes below read each vector once and fuse the MGS update of one basis
// vector with the dot product against the next.
#include <math.h>

#include "linalg.cuh"

namespace rok {

namespace {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the block; result valid in every thread; sh >= 33 doubles
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double r = lane < nw ? sh[lane] : 0.0;
        r = warp_sum(r);
        if (lane == 0) sh[32] = r;
    }
    __syncthreads();
    return sh[32];
}

// sum of P partials in a fixed order (identical in every block)
__device__ __forceinline__ double reduce_partials(const double *p, int P, double *sh)
{
    double v = 0.0;
    for (int k = threadIdx.x; k < P; k += blockDim.x) v += p[k];
    return block_sum(v, sh);
}

__device__ __forceinline__ size_t gtid() { return (size_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t gstride() { return (size_t)gridDim.x * blockDim.x; }

__global__ void dot2_kernel(const double *a0, const double *b0, const double *a1, const double *b1, size_t n,
                            double *partials, int P, const int *active)
{
    if (active && *active == 0) return;
    __shared__ double sh[34];
    double s0 = 0.0, s1 = 0.0;
    if (a1) {
        for (size_t e = gtid(); e < n; e += gstride()) {
            s0 += a0[e] * b0[e];
            s1 += a1[e] * b1[e];
        }
    } else {
        for (size_t e = gtid(); e < n; e += gstride()) s0 += a0[e] * b0[e];
    }
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s0;
        partials[P + blockIdx.x] = s1;
    }
}

__global__ void mgs_kernel(double *w, const double *vprev, const double *vnext, size_t n, const double *pin, int P,
                           double *hout, double *pout, int first, StepState *st)
{
    if (st->active == 0) return;
    __shared__ double sh[34];
    const double h = reduce_partials(pin, P, sh);
    if (first) {
        double wn2 = reduce_partials(pin + P, P, sh);
        if (blockIdx.x == 0 && threadIdx.x == 0) st->wnorm0 = sqrt(wn2);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *hout = h;
    double s = 0.0;
    if (vnext) {
        for (size_t e = gtid(); e < n; e += gstride()) {
            double we = w[e] - h * vprev[e];
            w[e] = we;
            s += vnext[e] * we;
        }
    } else {
        for (size_t e = gtid(); e < n; e += gstride()) {
            double we = w[e] - h * vprev[e];
            w[e] = we;
            s += we * we;
        }
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) pout[blockIdx.x] = s;
}

__global__ void normalize_kernel(const double *w, double *v, size_t n, const double *pin, int P, double *hsub,
                                 int column, StepState *st)
{
    // block 0 may clear st->active below while other blocks start: read it once
    // per block so that every thread of a block takes the same branch
    __shared__ int act;
    if (threadIdx.x == 0) act = st->active;
    __syncthreads();
    if (act == 0) return;
    __shared__ double sh[34];
    const double hn = sqrt(reduce_partials(pin, P, sh));
    // column 0: v_1 = f(y_n)/beta, beta = 0 leaves an empty basis; later columns
    // stop when h_{j+1,j} <= 1e-12 ||J v_j|| (also catches NaN)
    const bool brk = column == 0 ? !(hn > 0.0) : !(hn > 1e-12 * st->wnorm0);
    if (brk) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->active = 0;
            st->meff = column;
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (hsub) *hsub = hn;
        if (column == 0) st->beta = hn;
    }
    const double r = 1.0 / hn;
    for (size_t e = gtid(); e < n; e += gstride()) v[e] = w[e] * r;
}

constexpr int kDotChunk = 8;

__global__ void multidot_kernel(const double *F, const double *V, size_t ldv, size_t n, double *pout, int P,
                                const StepState *st)
{
    const int m = st->meff;
    __shared__ double sh[34];
    for (int m0 = 0; m0 < m; m0 += kDotChunk) {
        const int cnt = min(kDotChunk, m - m0);
        double acc[kDotChunk];
#pragma unroll
        for (int c = 0; c < kDotChunk; ++c) acc[c] = 0.0;
        for (size_t e = gtid(); e < n; e += gstride()) {
            const double f = F[e];
#pragma unroll
            for (int c = 0; c < kDotChunk; ++c)
                if (c < cnt) acc[c] += V[(size_t)(m0 + c) * ldv + e] * f;
        }
#pragma unroll
        for (int c = 0; c < kDotChunk; ++c) {
            if (c < cnt) {
                double t = block_sum(acc[c], sh);
                if (threadIdx.x == 0) pout[(size_t)(m0 + c) * P + blockIdx.x] = t;
            }
        }
    }
}

// One warp: LU with partial pivoting of L = I - h g H, row-major stride kMaxKrylov.
__global__ void lu_kernel(StepState *st)
{
    const int m = st->meff;
    const double hg = st->hg;
    const int lane = threadIdx.x;
    double *A = st->LU;
    for (int idx = lane; idx < m * m; idx += 32) {
        int i = idx / m, j = idx % m;
        A[i * kMaxKrylov + j] = (i == j ? 1.0 : 0.0) - hg * st->H[i * kMaxKrylov + j];
    }
    __syncwarp();
    for (int k = 0; k < m; ++k) {
        // pivot: largest |A[i][k]|, i >= k (ties: smallest index)
        double best = -1.0;
        int bi = k;
        for (int i = k + lane; i < m; i += 32) {
            double a = fabs(A[i * kMaxKrylov + k]);
            if (a > best) { best = a; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (bi != k)
            for (int j = lane; j < m; j += 32) {
                double t = A[k * kMaxKrylov + j];
                A[k * kMaxKrylov + j] = A[bi * kMaxKrylov + j];
                A[bi * kMaxKrylov + j] = t;
            }
        if (lane == 0) st->piv[k] = bi;
        __syncwarp();
        const double d = A[k * kMaxKrylov + k];
        if (!(fabs(d) > 0.0) || !isfinite(d)) {
            if (lane == 0) st->status |= kStatusSingular;
            return;
        }
        for (int i = k + 1 + lane; i < m; i += 32) {
            double l = A[i * kMaxKrylov + k] / d;
            A[i * kMaxKrylov + k] = l;
            for (int j = k + 1; j < m; ++j) A[i * kMaxKrylov + j] -= l * A[k * kMaxKrylov + j];
        }
        __syncwarp();
    }
}

struct GamRow {
    double g[4];
};

__global__ void stage_solve_kernel(int stage, GamRow gr, const double *pin, int P, StepState *st)
{
    const int m = st->meff;
    const double h = st->h;
    __shared__ double phi[kMaxKrylov], acc[kMaxKrylov], x[kMaxKrylov];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < P; ++b) s += pin[(size_t)i * P + b];
        phi[i] = s;
        double a = 0.0;
        for (int j = 0; j < stage; ++j) a = a + gr.g[j] * st->lam[j][i];
        acc[i] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // rhs = h phi + h H acc
        for (int i = 0; i < m; ++i) {
            double t = 0.0;
            for (int j = 0; j < m; ++j) t += st->H[i * kMaxKrylov + j] * acc[j];
            x[i] = h * phi[i] + h * t;
        }
        // P L U x = rhs: apply the row interchanges, then the two triangular solves
        for (int k = 0; k < m; ++k) {
            int p = st->piv[k];
            if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
        }
        const double *A = st->LU;
        for (int i = 0; i < m; ++i) {
            double t = x[i];
            for (int j = 0; j < i; ++j) t -= A[i * kMaxKrylov + j] * x[j];
            x[i] = t;
        }
        for (int i = m - 1; i >= 0; --i) {
            double t = x[i];
            for (int j = i + 1; j < m; ++j) t -= A[i * kMaxKrylov + j] * x[j];
            x[i] = t / A[i * kMaxKrylov + i];
        }
        bool ok = true;
        for (int i = 0; i < m; ++i) {
            st->lam[stage][i] = x[i];
            st->cvec[stage][i] = x[i] - h * phi[i];
            st->phi[i] = phi[i];
            ok = ok && isfinite(x[i]);
        }
        if (!ok) st->status |= kStatusNonfinite;
    }
}

__global__ void stage_vec_kernel(double *k, const double *F, const double *V, size_t ldv, size_t n, int stage,
                                 const StepState *st)
{
    __shared__ double c[kMaxKrylov];
    const int m = st->meff;
    const double h = st->h;
    for (int i = threadIdx.x; i < m; i += blockDim.x) c[i] = st->cvec[stage][i];
    __syncthreads();
    for (size_t e = gtid(); e < n; e += gstride()) {
        double a = 0.0;
        for (int i = 0; i < m; ++i) a += c[i] * V[(size_t)i * ldv + e];
        k[e] = a + h * F[e];
    }
}

struct AxpyArgs {
    const double *v[8];
    double c[8];
};

__global__ void axpy_n_kernel(double *out, const double *base, AxpyArgs a, int count, size_t n,
                              const StepState *guard)
{
    if (guard && guard->status != 0) return;
    for (size_t e = gtid(); e < n; e += gstride()) {
        double t = base[e];
        for (int q = 0; q < count; ++q) t = t + a.c[q] * a.v[q][e];
        out[e] = t;
    }
}

__global__ void basis_combine_kernel(double *out, const double *base, const double *V, size_t ldv, size_t n,
                                     int count, const double *gcoef)
{
    __shared__ double c[kMaxKrylov + 1];
    for (int i = threadIdx.x; i < count; i += blockDim.x) c[i] = gcoef[i];
    __syncthreads();
    for (size_t e = gtid(); e < n; e += gstride()) {
        double a = 0.0;
        for (int i = 0; i < count; ++i) a += c[i] * V[(size_t)i * ldv + e];
        out[e] = base[e] + a;
    }
}

__global__ void eps_kernel(const double *pin, int P, int v_unit, double eps_given, StepState *st)
{
    __shared__ double sh[34];
    const double yn = sqrt(reduce_partials(pin, P, sh));
    const double vn = v_unit ? 1.0 : sqrt(reduce_partials(pin + P, P, sh));
    if (threadIdx.x == 0) {
        double eps = eps_given;
        if (!(eps > 0.0)) {
            // sqrt(u (1 + ||y||)) / ||v||, u = 2^-52, rounded to the nearest power of two
            double x = sqrt(2.220446049250313e-16 * (1.0 + yn)) / vn;
            int e2;
            double mant = frexp(x, &e2);
            if (mant < sqrt(0.5)) e2 -= 1;
            eps = ldexp(1.0, e2);
        }
        st->eps = eps;
        st->inv_eps = 1.0 / eps;
        st->ynorm = yn;
    }
}

__global__ void begin_kernel(StepState *st, double h, double gamma, int M)
{
    st->h = h;
    st->hg = h * gamma;
    st->meff = M;
    st->active = M > 0 ? 1 : 0;
    st->beta = 0.0;
    st->wnorm0 = 0.0;
}

__global__ void sum_sqrt_kernel(const double *pin, int P, double *dst)
{
    __shared__ double sh[34];
    double s = reduce_partials(pin, P, sh);
    if (threadIdx.x == 0) *dst = sqrt(s);
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

__global__ void set_int_kernel(int *p, int v) { *p = v; }

// Lorenz-96 (appendix): f_i = (u_{i+1} - u_{i-2}) u_{i-1} - u_i + F, periodic,
// with the stencil launch's state formation and epilogue.
__global__ void lorenz_kernel(const StencilConsts C, const StencilIO io, int n)
{
    if (io.active && *io.active == 0) return;
    double cf[kMaxAdd];
#pragma unroll
    for (int t = 0; t < kMaxAdd; ++t) cf[t] = io.coef_dev[t] ? io.coef[t] * *io.coef_dev[t] : io.coef[t];
    const double s1 = io.s1_dev ? io.s1 * *io.s1_dev : io.s1;
    const double s2 = io.s2_dev ? io.s2 * *io.s2_dev : io.s2;
    auto q = [&](int i) {
        i = (i % n + n) % n;
        double v = io.base[i];
        for (int t = 0; t < io.nadd; ++t) v = v + cf[t] * io.add[t][i];
        return v;
    };
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double r = ((q(i + 1) - q(i - 2)) * q(i - 1) - q(i)) + C.lorenz_f;
        double t = io.sub ? (r - io.sub[i]) : r;
        t = t * s1;
        double o = io.add_out ? io.add_out[i] + s2 * t : t;
        io.out[i] = o;
        if (!isfinite(o)) atomicOr(io.status, kStatusNonfinite);
    }
}

}  // namespace

#define ROK_LAUNCH_CHECK() return cudaGetLastError()

static int s_elem_blocks = 1216;   // grid of the element-wise kernels (set from the SM count)

void set_elem_blocks(int b) { s_elem_blocks = b > 0 ? b : 1216; }

cudaError_t launch_set_int(int *p, int v, cudaStream_t s)
{
    set_int_kernel<<<1, 1, 0, s>>>(p, v);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_lorenz(const StencilConsts &c, const StencilIO &io, int n, cudaStream_t s)
{
    lorenz_kernel<<<(n + 255) / 256, 256, 0, s>>>(c, io, n);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_dot2(const double *a0, const double *b0, const double *a1, const double *b1, size_t n,
                        double *partials, int P, const int *active, cudaStream_t s)
{
    dot2_kernel<<<P, kRedThreads, 0, s>>>(a0, b0, a1, b1, n, partials, P, active);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_mgs(double *w, const double *vprev, const double *vnext, size_t n, const double *pin, int P,
                       double *hout, double *pout, bool first, StepState *st, cudaStream_t s)
{
    mgs_kernel<<<P, kRedThreads, 0, s>>>(w, vprev, vnext, n, pin, P, hout, pout, first ? 1 : 0, st);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_normalize(const double *w, double *v, size_t n, const double *pin, int P, double *hsub,
                             int column, StepState *st, cudaStream_t s)
{
    normalize_kernel<<<P, kRedThreads, 0, s>>>(w, v, n, pin, P, hsub, column, st);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_multidot(const double *F, const double *V, size_t ldv, size_t n, double *pout, int P,
                            const StepState *st, cudaStream_t s)
{
    multidot_kernel<<<P, kRedThreads, 0, s>>>(F, V, ldv, n, pout, P, st);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_stage_solve(int stage, const double *gam_row, const double *pin, int P, StepState *st,
                               cudaStream_t s)
{
    GamRow gr;
    for (int j = 0; j < 4; ++j) gr.g[j] = gam_row[j];
    stage_solve_kernel<<<1, 64, 0, s>>>(stage, gr, pin, P, st);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_lu(StepState *st, cudaStream_t s)
{
    lu_kernel<<<1, 32, 0, s>>>(st);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_stage_vec(double *k, const double *F, const double *V, size_t ldv, size_t n, int stage,
                             const StepState *st, cudaStream_t s)
{
    stage_vec_kernel<<<s_elem_blocks, kRedThreads, 0, s>>>(k, F, V, ldv, n, stage, st);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_axpy_n(double *out, const double *base, const double *const *v, const double *c, int count,
                          size_t n, const StepState *guard, cudaStream_t s)
{
    if (count > 8) return cudaErrorInvalidValue;
    AxpyArgs a;
    for (int q = 0; q < 8; ++q) {
        a.v[q] = q < count ? v[q] : nullptr;
        a.c[q] = q < count ? c[q] : 0.0;
    }
    axpy_n_kernel<<<s_elem_blocks, kRedThreads, 0, s>>>(out, base, a, count, n, guard);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_basis_combine(double *out, const double *base, const double *V, size_t ldv, size_t n,
                                 int count, const double *gcoef, cudaStream_t s)
{
    basis_combine_kernel<<<s_elem_blocks, kRedThreads, 0, s>>>(out, base, V, ldv, n, count, gcoef);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_eps(const double *pin, int P, bool v_unit, double eps_given, StepState *st, cudaStream_t s)
{
    eps_kernel<<<1, kRedThreads, 0, s>>>(pin, P, v_unit ? 1 : 0, eps_given, st);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_begin(StepState *st, double h, double gamma, int M, cudaStream_t s)
{
    begin_kernel<<<1, 1, 0, s>>>(st, h, gamma, M);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_sum_sqrt(const double *pin, int P, double *dst, cudaStream_t s)
{
    sum_sqrt_kernel<<<1, kRedThreads, 0, s>>>(pin, P, dst);
    ROK_LAUNCH_CHECK();
}

cudaError_t launch_cfl(const double *y, const StencilConsts &c, const double *six, const double *siy,
                       const double *sjx, const double *sjy, const double *vol, double *pmax, int P,
                       cudaStream_t s)
{
    cfl_kernel<<<P, kRedThreads, 0, s>>>(y, c, six, siy, sjx, sjy, vol, pmax);
    ROK_LAUNCH_CHECK();
}

}  // namespace rok
