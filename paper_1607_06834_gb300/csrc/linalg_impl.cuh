// Vector kernels of the ROK step (Sec. 2.3.3): inner products, the
// modified-Gram-Schmidt passes of the Arnoldi process, the projected stage
// solves of Eq. ROK, stage vectors and combines.
//
// Compiled twice like the stencil (linalg_fast.cu, linalg_strict.cu with
// --fmad=false), each time inside namespace ROK_NS.
//
// Every inner product is the pairwise sum of the rounded entrywise products: a
// balanced binary tree over the natural index order, zero-padded to a power of
// two.  The GPU evaluates exactly that tree:
//   - a warp owns 256 consecutive entries; lane l loads entries 32k + l
//     (k = 0..7, coalesced); an xor butterfly over the lanes (distances 1, 2,
//     4, 8, 16) forms the sums of the eight aligned 32-entry groups, which are
//     then added as a 3-level tree in registers;
//   - a CTA of 8 warps owns 2048 consecutive entries; the warp sums are added
//     as a 3-level tree;
//   - the consumer of the CTA partials adds them as a tree again (every CTA of
//     the consuming kernel computes the same value in the same order).
// Addition is commutative in IEEE arithmetic, so both partners of a butterfly
// hold the same sum.  The result is deterministic and independent of the
// launch configuration (extra zero leaves change nothing).
//
// On GB300 the FP64 pipe is the scarce unit (about two FP64 FMA per clock per
// SM), so FP64 vector passes sit near the HBM/FP64 balance point; each pass
// reads its vectors once, keeps eight independent loads per thread in flight,
// and the MGS update of one vector is fused with the inner product against
// the next.
#pragma once
#include <math.h>

#include "linalg.cuh"

namespace rok {
namespace ROK_NS {

constexpr int RT = 256;            // threads per CTA
constexpr int EPL = 8;             // entries per lane
constexpr int RB = RT * EPL;       // entries per CTA (2048)

__device__ __forceinline__ double lane_tree(double v)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum of the eight 32-entry groups of a warp: p[k] holds entry 32k + lane
__device__ __forceinline__ double warp_tree8(const double (&p)[EPL])
{
    double s[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) s[k] = lane_tree(p[k]);
    return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

// tree over the 8 warp sums of a CTA; sh >= 9 doubles; result in every thread
__device__ __forceinline__ double cta_tree(double wsum, double *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = wsum;
    __syncthreads();
    if (wid == 0) {
        double v = lane < 8 ? sh[lane] : 0.0;
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        if (lane == 0) sh[8] = v;
    }
    __syncthreads();
    return sh[8];
}

// Tree sum of p[0..P) (zero-padded to a power of two), identical in every CTA.
// Thread t owns the C = P2/256 consecutive leaves [tC, tC + C) (C >= 1) and
// adds them as an aligned tree with a carry stack, then lane and warp trees.
__device__ __forceinline__ double tree_partials(const double *p, int P, double *sh)
{
    int P2 = 1;
    while (P2 < P) P2 <<= 1;
    const int C = P2 > RT ? P2 / RT : 1;
    const int t = threadIdx.x;
    double v = 0.0;
    if (C == 1) {
        v = t < P ? p[t] : 0.0;
    } else {
        double stack[16];
        int lo = t * C;
        for (int k = 0; k < C; ++k) {
            double s = lo + k < P ? p[lo + k] : 0.0;
            int lvl = 0;
            for (int m = k; m & 1; m >>= 1, ++lvl) s = stack[lvl] + s;
            stack[lvl] = s;
        }
        int top = 0;
        while ((1 << top) < C) ++top;
        v = stack[top];
    }
    v = lane_tree(v);
    return cta_tree(v, sh);
}

__device__ __forceinline__ size_t warp_base()
{
    return ((size_t)blockIdx.x * RT + (threadIdx.x & ~31)) * EPL;
}

// partials[b] = <a0, b0> and partials[P + b] = <a1, b1> (if a1) over CTA b's range
__global__ void __launch_bounds__(RT) dot2_kernel(const double *a0, const double *b0, const double *a1,
                                                  const double *b1, size_t n, double *partials, int P,
                                                  const int *active)
{
    if (active && *active == 0) return;
    __shared__ double sh[10];
    const size_t base = warp_base() + (threadIdx.x & 31);
    double p[EPL], q[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
        size_t e = base + 32 * k;
        p[k] = e < n ? a0[e] * b0[e] : 0.0;
        q[k] = (a1 && e < n) ? a1[e] * b1[e] : 0.0;
    }
    double s0 = cta_tree(warp_tree8(p), sh);
    double s1 = cta_tree(warp_tree8(q), sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s0;
        partials[P + blockIdx.x] = s1;
    }
}

// h = tree(pin); H entry <- h; w <- w - h vprev; pout[b] = <vnext, w> (or <w, w>)
__global__ void __launch_bounds__(RT) mgs_kernel(double *w, const double *vprev, const double *vnext, size_t n,
                                                 const double *pin, int P, double *hout, double *pout, int first,
                                                 StepState *st)
{
    if (st->active == 0) return;
    __shared__ double sh[10];
    const double h = tree_partials(pin, P, sh);
    if (first) {
        double wn2 = tree_partials(pin + P, P, sh);
        if (blockIdx.x == 0 && threadIdx.x == 0) st->wnorm0 = sqrt(wn2);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *hout = h;
    const size_t base = warp_base() + (threadIdx.x & 31);
    double p[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
        size_t e = base + 32 * k;
        double pr = 0.0;
        if (e < n) {
            double we = w[e] - h * vprev[e];
            w[e] = we;
            pr = vnext ? vnext[e] * we : we * we;
        }
        p[k] = pr;
    }
    double s = cta_tree(warp_tree8(p), sh);
    if (threadIdx.x == 0) pout[blockIdx.x] = s;
}

// hn = sqrt(tree(pin)); breakdown test; v = w * (1/hn)
__global__ void __launch_bounds__(RT) normalize_kernel(const double *w, double *v, size_t n, const double *pin,
                                                       int P, double *hsub, int column, StepState *st)
{
    // block 0 may clear st->active below while other CTAs start: read it once
    // per CTA so that every thread of a CTA takes the same branch
    __shared__ int act;
    __shared__ double sh[10];
    if (threadIdx.x == 0) act = st->active;
    __syncthreads();
    if (act == 0) return;
    const double hn = sqrt(tree_partials(pin, P, sh));
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
    for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < n; e += (size_t)gridDim.x * RT) v[e] = w[e] * r;
}

// pout[m * P + b] = <V_m, F> over CTA b's range, m < meff
__global__ void __launch_bounds__(RT) multidot_kernel(const double *F, const double *V, size_t ldv, size_t n,
                                                      double *pout, int P, const StepState *st)
{
    const int m = st->meff;
    __shared__ double sh[10];
    const size_t base = warp_base() + (threadIdx.x & 31);
    double f[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
        size_t e = base + 32 * k;
        f[k] = e < n ? F[e] : 0.0;
    }
    for (int i = 0; i < m; ++i) {
        const double *Vi = V + (size_t)i * ldv;
        double p[EPL];
#pragma unroll
        for (int k = 0; k < EPL; ++k) {
            size_t e = base + 32 * k;
            p[k] = e < n ? Vi[e] * f[k] : 0.0;
        }
        double s = cta_tree(warp_tree8(p), sh);
        if (threadIdx.x == 0) pout[(size_t)i * P + blockIdx.x] = s;
    }
}

// One warp: LU with partial pivoting of L = I - h g H (first largest |pivot|),
// row-major stride kMaxKrylov.  Each entry sees the same operation sequence as
// a sequential elimination.
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
            for (int j = k + 1; j < m; ++j) A[i * kMaxKrylov + j] = A[i * kMaxKrylov + j] - l * A[k * kMaxKrylov + j];
        }
        __syncwarp();
    }
}

struct GamRow {
    double g[4];
};

// stage i: phi = V^T F_i (tree of the CTA partials), rhs = h phi + h H acc with
// acc = sum_{j<i} gamma_ij lambda_j, lambda_i = LU solve, cvec_i = lambda_i - h phi
__global__ void stage_solve_kernel(int stage, GamRow gr, const double *pin, int P, StepState *st)
{
    const int m = st->meff;
    const double h = st->h;
    __shared__ double phi[kMaxKrylov], acc[kMaxKrylov], x[kMaxKrylov];
    __shared__ double sh[10];
    for (int i = 0; i < m; ++i) {
        double s = tree_partials(pin + (size_t)i * P, P, sh);
        if (threadIdx.x == 0) phi[i] = s;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double a = 0.0;
        for (int j = 0; j < stage; ++j) a = a + gr.g[j] * st->lam[j][i];
        acc[i] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < m; ++i) {
            double t = 0.0;
            for (int j = 0; j < m; ++j) t = t + st->H[i * kMaxKrylov + j] * acc[j];
            x[i] = h * phi[i] + h * t;
        }
        for (int k = 0; k < m; ++k) {
            int p = st->piv[k];
            if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
        }
        const double *A = st->LU;
        for (int i = 0; i < m; ++i) {
            double t = x[i];
            for (int j = 0; j < i; ++j) t = t - A[i * kMaxKrylov + j] * x[j];
            x[i] = t;
        }
        for (int i = m - 1; i >= 0; --i) {
            double t = x[i];
            for (int j = i + 1; j < m; ++j) t = t - A[i * kMaxKrylov + j] * x[j];
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

// k = sum_{i<meff} cvec[stage][i] V_i + h F (basis order)
__global__ void __launch_bounds__(RT) stage_vec_kernel(double *k, const double *F, const double *V, size_t ldv,
                                                       size_t n, int stage, const StepState *st)
{
    __shared__ double c[kMaxKrylov];
    const int m = st->meff;
    const double h = st->h;
    for (int i = threadIdx.x; i < m; i += blockDim.x) c[i] = st->cvec[stage][i];
    __syncthreads();
    for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < n; e += (size_t)gridDim.x * RT) {
        double a = 0.0;
        for (int i = 0; i < m; ++i) a = a + c[i] * V[(size_t)i * ldv + e];
        k[e] = a + h * F[e];
    }
}

struct AxpyArgs {
    const double *v[8];
    double c[8];
};

// out = base + sum_q c_q v_q in order; skipped when a guard status is latched
__global__ void __launch_bounds__(RT) axpy_n_kernel(double *out, const double *base, AxpyArgs a, int count,
                                                    size_t n, const StepState *guard)
{
    if (guard && guard->status != 0) return;
    for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < n; e += (size_t)gridDim.x * RT) {
        double t = base[e];
        for (int q = 0; q < count; ++q) t = t + a.c[q] * a.v[q][e];
        out[e] = t;
    }
}

__global__ void __launch_bounds__(RT) basis_combine_kernel(double *out, const double *base, const double *V,
                                                           size_t ldv, size_t n, int count, const double *gcoef)
{
    __shared__ double c[kMaxKrylov + 1];
    for (int i = threadIdx.x; i < count; i += blockDim.x) c[i] = gcoef[i];
    __syncthreads();
    for (size_t e = (size_t)blockIdx.x * RT + threadIdx.x; e < n; e += (size_t)gridDim.x * RT) {
        double a = 0.0;
        for (int i = 0; i < count; ++i) a = a + c[i] * V[(size_t)i * ldv + e];
        out[e] = base[e] + a;
    }
}

// eps = sqrt(u (1 + ||y||)) / ||v|| rounded to the nearest power of two (or as given)
__global__ void eps_kernel(const double *pin, int P, int v_unit, double eps_given, StepState *st)
{
    __shared__ double sh[10];
    const double yn = sqrt(tree_partials(pin, P, sh));
    const double vn = v_unit ? 1.0 : sqrt(tree_partials(pin + P, P, sh));
    if (threadIdx.x == 0) {
        double eps = eps_given;
        if (!(eps > 0.0)) {
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

__global__ void sum_sqrt_kernel(const double *pin, int P, double *dst)
{
    __shared__ double sh[10];
    double s = tree_partials(pin, P, sh);
    if (threadIdx.x == 0) *dst = sqrt(s);
}

// ---- launchers ----------------------------------------------------------------

inline int blocks_for(size_t n) { return (int)((n + RB - 1) / RB); }

static cudaError_t dot2(const double *a0, const double *b0, const double *a1, const double *b1, size_t n,
                        double *partials, int P, const int *active, cudaStream_t s)
{
    dot2_kernel<<<P, RT, 0, s>>>(a0, b0, a1, b1, n, partials, P, active);
    return cudaGetLastError();
}

static cudaError_t mgs(double *w, const double *vprev, const double *vnext, size_t n, const double *pin, int P,
                       double *hout, double *pout, bool first, StepState *st, cudaStream_t s)
{
    mgs_kernel<<<P, RT, 0, s>>>(w, vprev, vnext, n, pin, P, hout, pout, first ? 1 : 0, st);
    return cudaGetLastError();
}

static cudaError_t normalize(const double *w, double *v, size_t n, const double *pin, int P, double *hsub,
                             int column, StepState *st, cudaStream_t s)
{
    normalize_kernel<<<P, RT, 0, s>>>(w, v, n, pin, P, hsub, column, st);
    return cudaGetLastError();
}

static cudaError_t multidot(const double *F, const double *V, size_t ldv, size_t n, double *pout, int P,
                            const StepState *st, cudaStream_t s)
{
    multidot_kernel<<<P, RT, 0, s>>>(F, V, ldv, n, pout, P, st);
    return cudaGetLastError();
}

static cudaError_t stage_solve(int stage, const double *gam_row, const double *pin, int P, StepState *st,
                               cudaStream_t s)
{
    GamRow gr;
    for (int j = 0; j < 4; ++j) gr.g[j] = gam_row[j];
    stage_solve_kernel<<<1, RT, 0, s>>>(stage, gr, pin, P, st);
    return cudaGetLastError();
}

static cudaError_t lu(StepState *st, cudaStream_t s)
{
    lu_kernel<<<1, 32, 0, s>>>(st);
    return cudaGetLastError();
}

static cudaError_t stage_vec(double *k, const double *F, const double *V, size_t ldv, size_t n, int stage,
                             const StepState *st, int grid, cudaStream_t s)
{
    stage_vec_kernel<<<grid, RT, 0, s>>>(k, F, V, ldv, n, stage, st);
    return cudaGetLastError();
}

static cudaError_t axpy_n(double *out, const double *base, const double *const *v, const double *c, int count,
                          size_t n, const StepState *guard, int grid, cudaStream_t s)
{
    if (count > 8) return cudaErrorInvalidValue;
    AxpyArgs a;
    for (int q = 0; q < 8; ++q) {
        a.v[q] = q < count ? v[q] : nullptr;
        a.c[q] = q < count ? c[q] : 0.0;
    }
    axpy_n_kernel<<<grid, RT, 0, s>>>(out, base, a, count, n, guard);
    return cudaGetLastError();
}

static cudaError_t basis_combine(double *out, const double *base, const double *V, size_t ldv, size_t n, int count,
                                 const double *gcoef, int grid, cudaStream_t s)
{
    basis_combine_kernel<<<grid, RT, 0, s>>>(out, base, V, ldv, n, count, gcoef);
    return cudaGetLastError();
}

static cudaError_t eps(const double *pin, int P, bool v_unit, double eps_given, StepState *st, cudaStream_t s)
{
    eps_kernel<<<1, RT, 0, s>>>(pin, P, v_unit ? 1 : 0, eps_given, st);
    return cudaGetLastError();
}

static cudaError_t sum_sqrt(const double *pin, int P, double *dst, cudaStream_t s)
{
    sum_sqrt_kernel<<<1, RT, 0, s>>>(pin, P, dst);
    return cudaGetLastError();
}

const LinalgOps ops = {dot2, mgs, normalize, multidot, stage_solve, lu, stage_vec, axpy_n, basis_combine, eps,
                       sum_sqrt};

}  // namespace ROK_NS
}  // namespace rok
