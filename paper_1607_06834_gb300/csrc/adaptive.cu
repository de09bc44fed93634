// Adaptive time stepping with embedded error estimates: ROK4 with its embedded
// order-2 weights and the DOPRI5 comparator (the paper compares methods with
// adaptive steps, Sec. 4.2; Table of Sec. 3.1 lists DOPRI5).
//
// Controller (Hairer, Norsett & Wanner I, Sec. II.4): err = weighted RMS norm
// of the estimate, sqrt(sum_i (e_i / sc_i)^2 / N), sc_i = atol + rtol
// max(|y_i|, |ynew_i|); accept when err <= 1; the next step is
// h min(facmax, max(facmin, safety err^(-1/(q+1)))), q the embedded order,
// never larger than h right after a rejection; a non-finite err rejects with
// facmin; the last step ends at T.  The sum of the norm is the pairwise tree
// of the per-chunk partials, finished on the host; the controller is plain
// host arithmetic.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "coefficients.h"
#include "context.h"
#include "linalg.cuh"

using namespace rok;

namespace rok_host {
rok_status launch_stencil(rok_ctx *c, const StencilIO &io);
StencilIO plain_io(rok_ctx *c, const double *y, double *out);
}  // namespace rok_host

namespace {

#define CU(x)                                      \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) return ROK_ERR_CUDA; \
    } while (0)

// pairwise (aligned binary tree) sum of p[0..n), zero-padded to a power of two
double tree_sum(const double *p, int n)
{
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    std::vector<double> b(n2, 0.0);
    for (int i = 0; i < n; ++i) b[i] = p[i];
    for (int len = n2; len > 1; len >>= 1)
        for (int i = 0; i < len / 2; ++i) b[i] = b[2 * i] + b[2 * i + 1];
    return b[0];
}

// weighted RMS norm of e = sum_q d_q k_q between y and ynew
rok_status wrms(rok_ctx *c, const double *y, const double *ynew, const double *const *kv, const double *d, int count,
                double atol, double rtol, double *err)
{
    CU(c->ops->err_sum(y, ynew, kv, d, count, atol, rtol, c->N, c->pA, c->P, c->stream));
    c->launches++;
    CU(cudaMemcpyAsync(c->h_part, c->pA, c->P * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    *err = sqrt(tree_sum(c->h_part, c->P) / (double)c->N);
    return ROK_OK;
}

struct Controller {
    rok_adapt_opts o;
    int q;
    double t = 0.0, h = 0.0;
    int acc = 0, rej = 0;
    bool after_reject = false;

    bool done(double T) const { return !(T - t > 1e-12 * T) || acc + rej >= o.max_steps; }
    // returns true when the step of size h is accepted
    bool update(double err)
    {
        double fac;
        if (!isfinite(err)) fac = o.facmin;
        else if (err == 0.0) fac = o.facmax;
        else fac = std::min(o.facmax, std::max(o.facmin, o.safety * pow(err, -1.0 / (q + 1))));
        const bool ok = isfinite(err) && err <= 1.0;
        if (ok) {
            t = t + h;
            acc++;
            if (after_reject) fac = std::min(fac, 1.0);
            after_reject = false;
        } else {
            rej++;
            after_reject = true;
            fac = std::min(fac, 1.0);
        }
        h = h * fac;
        return ok;
    }
};

rok_status check_opts(const rok_adapt_opts *o, double T)
{
    if (!o || !(T > 0.0) || !isfinite(T)) return ROK_ERR_INVALID_ARG;
    if (!(o->h0 > 0.0) || !(o->atol >= 0.0) || !(o->rtol >= 0.0) || !(o->atol + o->rtol > 0.0)) return ROK_ERR_INVALID_ARG;
    if (!(o->safety > 0.0) || !(o->facmin > 0.0) || !(o->facmax >= 1.0) || o->max_steps < 1) return ROK_ERR_INVALID_ARG;
    return ROK_OK;
}

void fill_info(rok_adapt_info *info, const Controller &k, long long evals)
{
    if (!info) return;
    memset(info, 0, sizeof(*info));
    info->accepted = k.acc;
    info->rejected = k.rej;
    info->t = k.t;
    info->h_next = k.h;
    info->residual_evals = evals;
}

}  // namespace

extern "C" {

rok_status rok_integrate(rok_ctx *c, double *y, double T, int M, const rok_adapt_opts *o, rok_adapt_info *info)
{
    if (!c || !y || M < 0 || M > c->mmax) return ROK_ERR_INVALID_ARG;
    rok_status r = check_opts(o, T);
    if (r != ROK_OK) return r;
    const size_t N = c->N;
    double *ytry = c->t1;   // the attempted step (t1 is not used by rok_step)
    Controller k;
    k.o = *o;
    k.q = 2;
    k.h = o->h0;
    double d[4];
    for (int i = 0; i < 4; ++i) d[i] = kRokB[i] - kRokBhat[i];
    const double *kv[4] = {c->K[0], c->K[1], c->K[2], c->K[3]};
    long long evals = 0;
    while (!k.done(T)) {
        if (k.t + k.h > T) k.h = T - k.t;
        CU(cudaMemcpyAsync(ytry, y, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        rok_step_info si;
        r = rok_step(c, ytry, k.h, M, &si);
        evals += 1 + M + 3;
        double err = INFINITY;
        if (r == ROK_OK) {
            if ((r = wrms(c, y, ytry, kv, d, 4, o->atol, o->rtol, &err)) != ROK_OK) return r;
        } else if (r != ROK_ERR_NONFINITE) {
            return r;
        }
        if (k.update(err)) CU(cudaMemcpyAsync(y, ytry, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
    CU(cudaStreamSynchronize(c->stream));
    fill_info(info, k, evals);
    return k.t < T && T - k.t > 1e-12 * T ? ROK_ERR_NOT_CONVERGED : ROK_OK;
}

rok_status dopri5_integrate(rok_ctx *c, double *y, double T, const rok_adapt_opts *o, rok_adapt_info *info)
{
    if (!c || !y) return ROK_ERR_INVALID_ARG;
    rok_status r = check_opts(o, T);
    if (r != ROK_OK) return r;
    const size_t N = c->N;
    double *pool[8] = {c->F[0], c->F[1], c->F[2], c->F[3], c->K[0], c->K[1], c->K[2], c->K[3]};
    int kb[7] = {0, 1, 2, 3, 4, 5, 6};   // buffer of stage k_{i+1}
    int spare = 7;
    double *ynew = c->t1, *Y = c->t0;
    Controller k;
    k.o = *o;
    k.q = 4;
    k.h = o->h0;
    long long evals = 0;
    CU(launch_set_int(&c->st->status, 0, c->stream));
    // k_1 = f(y)
    r = rok_host::launch_stencil(c, rok_host::plain_io(c, y, pool[kb[0]]));
    if (r != ROK_OK) return r;
    evals++;
    while (!k.done(T)) {
        if (k.t + k.h > T) k.h = T - k.t;
        const double h = k.h;
        for (int i = 1; i < 7; ++i) {
            const double *vv[8];
            double cc[8];
            int cnt = 0;
            for (int j = 0; j < i; ++j)
                if (kDp5A[i][j] != 0.0) {
                    vv[cnt] = pool[kb[j]];
                    cc[cnt] = h * kDp5A[i][j];
                    cnt++;
                }
            double *dst = i == 6 ? ynew : Y;   // the 7th stage state is y_{n+1}
            CU(c->ops->axpy_n(dst, y, vv, cc, cnt, N, nullptr, c->egrid, c->stream));
            c->launches++;
            r = rok_host::launch_stencil(c, rok_host::plain_io(c, dst, pool[kb[i]]));
            if (r != ROK_OK) return r;
            evals++;
        }
        const double *ev[8];
        double dd[8];
        int cnt = 0;
        for (int j = 0; j < 7; ++j) {
            const double dj = kDp5B[j] - kDp5Bhat[j];
            if (dj != 0.0) {
                ev[cnt] = pool[kb[j]];
                dd[cnt] = h * dj;
                cnt++;
            }
        }
        double err = INFINITY;
        if ((r = wrms(c, y, ynew, ev, dd, cnt, o->atol, o->rtol, &err)) != ROK_OK) return r;
        if (k.update(err)) {
            CU(cudaMemcpyAsync(y, ynew, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            // first same as last: k_7 = f(y_{n+1}) becomes k_1
            const int old1 = kb[0];
            kb[0] = kb[6];
            kb[6] = spare;
            spare = old1;
        }
    }
    // non-finite stages latch the status word; rejected steps have handled them
    CU(launch_set_int(&c->st->status, 0, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    fill_info(info, k, evals);
    return k.t < T && T - k.t > 1e-12 * T ? ROK_ERR_NOT_CONVERGED : ROK_OK;
}

}  // extern "C"
