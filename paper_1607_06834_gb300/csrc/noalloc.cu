// rok_jvp_noalloc: the finite-difference Jacobian-vector product without any
// device allocation, for callers that cannot call cudaMalloc.
//
// The scratch that rok_jvp takes from its context (the CTA partial sums of
// ||y||^2 and ||v||^2, the increment eps and 1/eps, the latched status word)
// lives here in one file-scope __device__ array.  Every GPU that loads the
// library holds it until the process exits.  Host code cannot use the array's
// name as a device address; the address is resolved once per device with
// cudaGetSymbolAddress and cached.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "linalg.cuh"
#include "rok_internal.h"

using namespace rok;

namespace {

constexpr int kNoAllocMaxPartials = ROK_NOALLOC_MAX_N / 2048;

struct NoAllocScratch {
    StepState st;                                  // eps, 1/eps, ||y||, status word
    double partials[2 * kNoAllocMaxPartials];      // CTA partials of ||y||^2, ||v||^2
};

__device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
NoAllocScratch *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (resolved on first use).
rok_status scratch_address(NoAllocScratch **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ROK_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return ROK_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ROK_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_scratch_addr[dev];
    return ROK_OK;
}

__global__ void clear_status_kernel(int *status) { *status = 0; }

__global__ void copy_status_kernel(const int *src, int *dst) { *dst = *src; }

// Constants of the uniform-grid residual, computed by the same expressions as
// for a context (so that the result equals rok_jvp's bit for bit).
void uniform_consts(const rok_problem_desc &d, StencilConsts &C)
{
    memset(&C, 0, sizeof(C));
    C.nx = d.nx;
    C.ny = d.kind == ROK_LORENZ96 ? 1 : d.ny;
    for (int k = 0; k < 4; ++k) C.bc[k] = d.bc[k];
    C.viscous = d.kind == ROK_NS2D;
    C.sutherland = d.kind == ROK_NS2D && d.sutherland_s > 0.0;
    C.gm1 = d.gamma - 1.0;
    C.inv_gm1 = 1.0 / C.gm1;
    C.c_lo = 0.25 * (1.0 - d.muscl_kappa);
    C.c_hi = 0.25 * (1.0 + d.muscl_kappa);
    C.efix = d.entropy_fix;
    C.kfac = d.kind == ROK_NS2D ? d.gamma / (C.gm1 * d.prandtl) : 0.0;
    C.c23 = 2.0 / 3.0;
    C.g_over_pr = d.kind == ROK_NS2D ? d.gamma / d.prandtl : 0.0;
    C.mu = d.kind == ROK_NS2D ? d.mu : 0.0;
    C.inv_tref = C.sutherland ? 1.0 / d.t_ref : 0.0;
    C.suth_s = d.sutherland_s;
    if (d.kind != ROK_LORENZ96) {
        double dx = d.lx / d.nx, dy = d.ly / d.ny;
        C.rdx = 1.0 / dx;
        C.rdy = 1.0 / dy;
        C.q_rdx = 0.25 * C.rdx;
        C.q_rdy = 0.25 * C.rdy;
        double rinv = 1.0 / d.q_inf[0];
        double u = d.q_inf[1] * rinv, v = d.q_inf[2] * rinv;
        double p = C.gm1 * (d.q_inf[3] - 0.5 * (d.q_inf[1] * u + d.q_inf[2] * v));
        double T = p * rinv;
        double mu = d.mu;
        if (C.sutherland) {
            double t = T * C.inv_tref;
            mu = d.mu * (t * sqrt(t)) * ((1.0 + d.sutherland_s) / (t + d.sutherland_s));
        }
        C.prim_inf[0] = d.q_inf[0];
        C.prim_inf[1] = u;
        C.prim_inf[2] = v;
        C.prim_inf[3] = p;
        C.prim_inf[4] = T;
        C.prim_inf[5] = d.kind == ROK_NS2D ? mu : 0.0;
        set_fast_consts(C);
    }
    C.lorenz_f = d.lorenz_f;
}

}  // namespace

extern "C" rok_status rok_jvp_noalloc(const rok_problem_desc *d, const double *y, const double *fy, const double *v,
                                      double *jv, double eps, int *status, void *cuda_stream)
{
    if (!d || !y || !fy || !v || !jv) return ROK_ERR_INVALID_ARG;
    if (jv == y || jv == v || jv == fy) return ROK_ERR_INVALID_ARG;
    if (d->rounding != ROK_ROUND_FAST && d->rounding != ROK_ROUND_STRICT) return ROK_ERR_INVALID_ARG;
    if (d->jvp != ROK_JVP_FD) return ROK_ERR_UNSUPPORTED;   // the dual-number product is not offered here
    size_t N;
    if (d->kind == ROK_LORENZ96) {
        if (d->nx < 4) return ROK_ERR_INVALID_ARG;
        N = (size_t)d->nx;
    } else if (d->kind == ROK_EULER2D || d->kind == ROK_NS2D) {
        if (d->nx < 2 || d->ny < 2 || !(d->gamma > 1.0)) return ROK_ERR_INVALID_ARG;
        if (d->xv || d->yv) return ROK_ERR_UNSUPPORTED;   // curvilinear metrics would need device memory
        if (!(d->lx > 0.0) || !(d->ly > 0.0)) return ROK_ERR_INVALID_ARG;
        for (int k = 0; k < 4; ++k)
            if (d->bc[k] != ROK_BC_PERIODIC) return ROK_ERR_UNSUPPORTED;
        if (d->kind == ROK_NS2D && (!(d->prandtl > 0.0) || d->mu < 0.0)) return ROK_ERR_INVALID_ARG;
        if (d->kind == ROK_NS2D && d->sutherland_s > 0.0 && !(d->t_ref > 0.0)) return ROK_ERR_INVALID_ARG;
        N = 4 * (size_t)d->nx * (size_t)d->ny;
    } else {
        return ROK_ERR_INVALID_ARG;
    }
    if (N > (size_t)ROK_NOALLOC_MAX_N) return ROK_ERR_INVALID_ARG;   // beyond the static scratch

    NoAllocScratch *scr = nullptr;
    rok_status r = scratch_address(&scr);
    if (r != ROK_OK) return r;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool strict = d->rounding == ROK_ROUND_STRICT;
    const LinalgOps &ops = strict ? strict::ops : fast::ops;
    StencilConsts C;
    uniform_consts(*d, C);
    const int P = reduction_blocks(N);
    StepState *st = &scr->st;

    clear_status_kernel<<<1, 1, 0, s>>>(&st->status);
    if (cudaGetLastError() != cudaSuccess) return ROK_ERR_CUDA;
    // ||y||^2, ||v||^2 partials, then eps = sqrt(u (1 + ||y||)) / ||v|| rounded to a power of two
    if (ops.dot2(y, y, v, v, N, scr->partials, P, nullptr, s) != cudaSuccess) return ROK_ERR_CUDA;
    if (ops.eps(scr->partials, P, false, eps, st, s) != cudaSuccess) return ROK_ERR_CUDA;
    StencilIO io;
    memset(&io, 0, sizeof(io));
    io.base = y;
    io.add[0] = v;
    io.coef[0] = 1.0;
    io.coef_dev[0] = &st->eps;
    io.nadd = 1;
    io.sub = fy;
    io.s1 = 1.0;
    io.s1_dev = &st->inv_eps;
    io.s2 = 1.0;
    io.out = jv;
    io.status = &st->status;
    cudaError_t e;
    if (d->kind == ROK_LORENZ96) e = strict ? strict::launch_lorenz(C, io, C.nx, s) : fast::launch_lorenz(C, io, C.nx, s);
    else e = strict ? strict::launch_cart(C, io, s) : fast::launch_cart(C, io, s);
    if (e != cudaSuccess) return ROK_ERR_CUDA;
    if (status) {
        copy_status_kernel<<<1, 1, 0, s>>>(&st->status, status);
        if (cudaGetLastError() != cudaSuccess) return ROK_ERR_CUDA;
    }
    return ROK_OK;
}
