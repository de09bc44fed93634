// C ABI of librok (include/rok.h): context, workspace, and the host drivers of
// the ROK4 step (Sec. 2.2.2, Eq. ROK), classical RK4 (Sec. 2.1, Eq. RK) and
// ESDIRK3 with matrix-free Newton-GMRES (Sec. 2.1, Eqs. Newton, SDIRK_Newton,
// Newton_Jac_Matrix).  Every arithmetic step runs in the CUDA kernels of
// stencil_*.cu and linalg.cu; the host only enqueues launches (and, for the
// Newton-GMRES comparator, reads small Hessenberg columns back).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <utility>
#include <vector>

#include "coefficients.h"
#include "context.h"
#include "linalg.cuh"
#include "rok_internal.h"

using namespace rok;

namespace {

#define CU(x)                                      \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) return ROK_ERR_CUDA; \
    } while (0)

rok_status stencil(rok_ctx *c, const StencilIO &io)
{
    c->launches++;
    c->stencil_launches++;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (c->time_stencil && !c->capturing) {
        if (c->ev_free.empty()) {
            cudaEvent_t a, b;
            CU(cudaEventCreate(&a));
            CU(cudaEventCreate(&b));
            c->ev_free.push_back({a, b});
        }
        ev = c->ev_free.back();
        c->ev_free.pop_back();
        CU(cudaEventRecord(ev.first, c->stream));
    }
    cudaError_t e;
    if (c->kind == ROK_LORENZ96) e = c->strict ? strict::launch_lorenz(c->C, io, c->C.nx, c->stream) : fast::launch_lorenz(c->C, io, c->C.nx, c->stream);
    else if (c->curv) e = c->strict ? strict::launch_curv(c->C, c->G, io, c->stream) : fast::launch_curv(c->C, c->G, io, c->stream);
    else e = c->strict ? strict::launch_cart(c->C, io, c->stream) : fast::launch_cart(c->C, io, c->stream);
    if (e != cudaSuccess) return ROK_ERR_CUDA;
    if (ev.first) {
        CU(cudaEventRecord(ev.second, c->stream));
        c->ev_used.push_back(ev);
    }
    return ROK_OK;
}

StencilIO io_plain(rok_ctx *c, const double *y, double *out)
{
    StencilIO io;
    memset(&io, 0, sizeof(io));
    io.base = y;
    io.s1 = 1.0;
    io.s2 = 1.0;
    io.out = out;
    io.status = &c->st->status;
    return io;
}

// jv = (f(y + eps v) - f0) * inv_eps with eps, inv_eps from the step state
StencilIO io_jvp(rok_ctx *c, const double *y, const double *v, const double *f0, double *out)
{
    StencilIO io = io_plain(c, y, out);
    io.add[0] = v;
    io.coef[0] = 1.0;
    io.coef_dev[0] = &c->st->eps;
    io.nadd = 1;
    io.sub = f0;
    io.s1_dev = &c->st->inv_eps;
    return io;
}

void free_ctx(rok_ctx *c)
{
    if (!c) return;
    rok_free_adjoint(c);
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->gev[0]) cudaEventDestroy(c->gev[0]);
    if (c->gev[1]) cudaEventDestroy(c->gev[1]);
    for (auto &e : c->ev_used) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    for (auto &e : c->ev_free) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    cudaFree(c->V);
    cudaFree(c->Vf);
    for (int i = 0; i < 4; ++i) { cudaFree(c->F[i]); cudaFree(c->K[i]); }
    cudaFree(c->w); cudaFree(c->t0); cudaFree(c->t1); cudaFree(c->t2);
    cudaFree(c->pA); cudaFree(c->pB); cudaFree(c->pM);
    cudaFree(c->st);
    cudaFree(c->colcnt);
    cudaFreeHost(c->h_st);
    cudaFreeHost(c->h_part);
    for (double *p : c->geo_bufs) cudaFree(p);
    cudaFree(c->cfl_six); cudaFree(c->cfl_siy); cudaFree(c->cfl_sjx); cudaFree(c->cfl_sjy); cudaFree(c->cfl_vol);
    delete c;
}

// ---- curvilinear metrics (host, no FMA contraction) -----------------------------
struct Pt { double x, y; };

struct Verts {
    const rok_problem_desc *d;
    double X(int i, int j) const { return d->xv[(size_t)j * (d->nx + 1) + i]; }
    double Y(int i, int j) const { return d->yv[(size_t)j * (d->nx + 1) + i]; }
    // vertex (i, j) with i in [-1, nx+1], j in [-1, ny+1]: a periodic side wraps
    // with the period offset, other sides extrapolate linearly along the grid line
    Pt at(int i, int j) const
    {
        const int nx = d->nx, ny = d->ny;
        double ox = 0.0, oy = 0.0;
        if (i < 0 || i > nx) {
            if (d->bc[0] == ROK_BC_PERIODIC) {
                int jj = j < 0 ? 0 : (j > ny ? ny : j);
                double px = X(nx, jj) - X(0, jj), py = Y(nx, jj) - Y(0, jj);
                if (i < 0) { i += nx; ox -= px; oy -= py; }
                else { i -= nx; ox += px; oy += py; }
            } else {
                Pt a = at(i < 0 ? 0 : nx, j), b = at(i < 0 ? 1 : nx - 1, j);
                return {2.0 * a.x - b.x, 2.0 * a.y - b.y};
            }
        }
        if (j < 0 || j > ny) {
            if (d->bc[2] == ROK_BC_PERIODIC) {
                double px = X(i, ny) - X(i, 0), py = Y(i, ny) - Y(i, 0);
                if (j < 0) { j += ny; ox -= px; oy -= py; }
                else { j -= ny; ox += px; oy += py; }
            } else {
                int j0 = j < 0 ? 0 : ny, j1 = j < 0 ? 1 : ny - 1;
                return {(2.0 * X(i, j0) - X(i, j1)) + ox, (2.0 * Y(i, j0) - Y(i, j1)) + oy};
            }
        }
        return {X(i, j) + ox, Y(i, j) + oy};
    }
};

// Green-Gauss on the quadrilateral P0 (cell), P1 (vertex), P2 (cell), P3 (vertex)
void diamond(Pt p0, Pt p1, Pt p2, Pt p3, double *c)
{
    double d1x = p2.x - p0.x, d1y = p2.y - p0.y, d2x = p3.x - p1.x, d2y = p3.y - p1.y;
    double inv2a = 1.0 / (d1x * d2y - d1y * d2x);
    c[0] = d2y * inv2a;
    c[1] = -d1y * inv2a;
    c[2] = -d2x * inv2a;
    c[3] = d1x * inv2a;
}

rok_status build_geometry(rok_ctx *c)
{
    const rok_problem_desc &d = c->d;
    const int nx = d.nx, ny = d.ny;
    Verts V{&d};
    const size_t nfi = (size_t)(nx + 1) * ny, nfj = (size_t)nx * (ny + 1), nce = (size_t)(nx + 2) * (ny + 2);
    std::vector<double> cx(nce), cy(nce);
    auto CI = [&](int i, int j) { return (size_t)(j + 1) * (nx + 2) + (i + 1); };
    std::vector<double> inv_vol((size_t)nx * ny), vol((size_t)nx * ny);
    for (int j = -1; j <= ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            Pt a = V.at(i, j), b = V.at(i + 1, j), e = V.at(i + 1, j + 1), f = V.at(i, j + 1);
            cx[CI(i, j)] = 0.25 * (((a.x + b.x) + e.x) + f.x);
            cy[CI(i, j)] = 0.25 * (((a.y + b.y) + e.y) + f.y);
            if (i >= 0 && i < nx && j >= 0 && j < ny) {
                double area = 0.5 * ((e.x - a.x) * (f.y - b.y) - (e.y - a.y) * (f.x - b.x));
                if (!(area > 0.0)) return ROK_ERR_INVALID_ARG;
                inv_vol[(size_t)j * nx + i] = 1.0 / area;
                vol[(size_t)j * nx + i] = area;
            }
        }
    std::vector<double> in_x(nfi), in_y(nfi), il(nfi), ic[4], jn_x(nfj), jn_y(nfj), jl(nfj), jc[4];
    for (int k = 0; k < 4; ++k) { ic[k].resize(nfi); jc[k].resize(nfj); }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            size_t f = (size_t)j * (nx + 1) + i;
            double ex = V.X(i, j + 1) - V.X(i, j), ey = V.Y(i, j + 1) - V.Y(i, j);
            double len = sqrt(ex * ex + ey * ey);
            il[f] = len; in_x[f] = ey / len; in_y[f] = -ex / len;
            double cc[4];
            diamond({cx[CI(i - 1, j)], cy[CI(i - 1, j)]}, {V.X(i, j), V.Y(i, j)}, {cx[CI(i, j)], cy[CI(i, j)]},
                    {V.X(i, j + 1), V.Y(i, j + 1)}, cc);
            for (int k = 0; k < 4; ++k) ic[k][f] = cc[k];
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t f = (size_t)j * nx + i;
            double ex = V.X(i + 1, j) - V.X(i, j), ey = V.Y(i + 1, j) - V.Y(i, j);
            double len = sqrt(ex * ex + ey * ey);
            jl[f] = len; jn_x[f] = -ey / len; jn_y[f] = ex / len;
            double cc[4];
            diamond({cx[CI(i, j - 1)], cy[CI(i, j - 1)]}, {V.X(i + 1, j), V.Y(i + 1, j)}, {cx[CI(i, j)], cy[CI(i, j)]},
                    {V.X(i, j), V.Y(i, j)}, cc);
            for (int k = 0; k < 4; ++k) jc[k][f] = cc[k];
        }
    // mean face-area vectors of each cell (time-step bound)
    std::vector<double> six((size_t)nx * ny), siy((size_t)nx * ny), sjx((size_t)nx * ny), sjy((size_t)nx * ny);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t cc = (size_t)j * nx + i;
            double exa = V.X(i, j + 1) - V.X(i, j), eya = V.Y(i, j + 1) - V.Y(i, j);
            double exb = V.X(i + 1, j + 1) - V.X(i + 1, j), eyb = V.Y(i + 1, j + 1) - V.Y(i + 1, j);
            six[cc] = 0.5 * (eya + eyb);
            siy[cc] = 0.5 * (-exa - exb);
            double exc = V.X(i + 1, j) - V.X(i, j), eyc = V.Y(i + 1, j) - V.Y(i, j);
            double exd = V.X(i + 1, j + 1) - V.X(i, j + 1), eyd = V.Y(i + 1, j + 1) - V.Y(i, j + 1);
            sjx[cc] = 0.5 * (-eyc - eyd);
            sjy[cc] = 0.5 * (exc + exd);
        }
    auto up = [&](const std::vector<double> &h, const double **dst) -> rok_status {
        double *p = nullptr;
        if (cudaMalloc(&p, h.size() * sizeof(double)) != cudaSuccess) return ROK_ERR_NOMEM;
        c->geo_bufs.push_back(p);
        if (cudaMemcpy(p, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return ROK_ERR_CUDA;
        *dst = p;
        return ROK_OK;
    };
    rok_status s;
    const std::vector<double> *src[] = {&in_x, &in_y, &il, &ic[0], &ic[1], &ic[2], &ic[3],
                                        &jn_x, &jn_y, &jl, &jc[0], &jc[1], &jc[2], &jc[3], &inv_vol};
    const double **dst[] = {&c->G.in_x, &c->G.in_y, &c->G.il, &c->G.ic0, &c->G.ic1, &c->G.ic2, &c->G.ic3,
                            &c->G.jn_x, &c->G.jn_y, &c->G.jl, &c->G.jc0, &c->G.jc1, &c->G.jc2, &c->G.jc3,
                            &c->G.inv_vol};
    for (int k = 0; k < 15; ++k)
        if ((s = up(*src[k], dst[k])) != ROK_OK) return s;
    const double *tmp;
    if ((s = up(six, &tmp)) != ROK_OK) return s; c->cfl_six = const_cast<double *>(tmp); c->geo_bufs.pop_back();
    if ((s = up(siy, &tmp)) != ROK_OK) return s; c->cfl_siy = const_cast<double *>(tmp); c->geo_bufs.pop_back();
    if ((s = up(sjx, &tmp)) != ROK_OK) return s; c->cfl_sjx = const_cast<double *>(tmp); c->geo_bufs.pop_back();
    if ((s = up(sjy, &tmp)) != ROK_OK) return s; c->cfl_sjy = const_cast<double *>(tmp); c->geo_bufs.pop_back();
    if ((s = up(vol, &tmp)) != ROK_OK) return s; c->cfl_vol = const_cast<double *>(tmp); c->geo_bufs.pop_back();
    return ROK_OK;
}

void to_prim_host(const rok_problem_desc &d, const StencilConsts &C, const double *q, double *w)
{
    double rinv = 1.0 / q[0];
    double u = q[1] * rinv, v = q[2] * rinv;
    double p = C.gm1 * (q[3] - 0.5 * (q[1] * u + q[2] * v));
    double T = p * rinv;
    w[0] = q[0]; w[1] = u; w[2] = v; w[3] = p; w[4] = T;
    double mu = d.mu;
    if (d.kind == ROK_NS2D && d.sutherland_s > 0.0) {
        double t = T * C.inv_tref;
        mu = d.mu * (t * sqrt(t)) * ((1.0 + d.sutherland_s) / (t + d.sutherland_s));
    }
    w[5] = d.kind == ROK_NS2D ? mu : 0.0;
}

rok_status fail_latched(rok_ctx *c)
{
    int s = c->h_st->status;
    if (s & kStatusNonfinite) return ROK_ERR_NONFINITE;
    if (s & kStatusSingular) return ROK_ERR_NONFINITE;
    if (s & kStatusTimeout) return ROK_ERR_TIMEOUT;
    return ROK_OK;
}

// Synchronise, read the step state, fill info, clear the latched status.
rok_status sync_read(rok_ctx *c, rok_step_info *info)
{
    CU(cudaMemcpyAsync(c->h_st, c->st, offsetof(StepState, H), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    rok_status s = fail_latched(c);
    if (c->h_st->status) CU(launch_set_int(&c->st->status, 0, c->stream));
    c->last.status = s;
    c->last.m_eff = c->h_st->meff;
    c->last.eps = c->h_st->eps;
    if (info) *info = c->last;
    return s;
}

// Columns 0..M-1 of the Arnoldi process of Sec. 2.2.2 (v_1 already in V[0]):
// JVP of v_j, then the modified-Gram-Schmidt column, either in one persistent
// cooperative launch or as dot2 + (j+1) mgs passes + normalize.  Both forms
// perform the same arithmetic.
rok_status arnoldi_columns(rok_ctx *c, const double *y, int M)
{
    const size_t N = c->N;
    const int P = c->P;
    StepState *st = c->st;
    cudaStream_t s = c->stream;
    rok_status r;
    void *Vb = c->fp32 ? (void *)c->Vf : (void *)c->V;
    if (c->col_ctas > 0 && c->persistent && M > 0)
        CU(cudaMemsetAsync(c->colcnt, 0, column_counter_offset(M) * sizeof(unsigned), s));
    for (int j = 0; j < M; ++j) {
        StencilIO io;
        if (c->exact_jvp) {
            io = io_plain(c, y, c->w);   // J(y) v_j by dual numbers
            if (c->fp32) io.dirf = c->Vf + (size_t)j * N;
            else io.dir = c->V + (size_t)j * N;
        } else if (c->fp32) {
            io = io_plain(c, y, c->w);
            io.addf = c->Vf + (size_t)j * N;
            io.coef_f = 1.0;
            io.coef_f_dev = &st->eps;
            io.sub = c->F[0];
            io.s1_dev = &st->inv_eps;
        } else {
            io = io_jvp(c, y, c->V + (size_t)j * N, c->F[0], c->w);
        }
        io.active = &st->active;
        if ((r = stencil(c, io)) != ROK_OK) return r;
        cudaError_t e = cudaErrorNotSupported;
        if (c->col_ctas > 0 && c->persistent)
            e = c->ops->arnoldi_column(c->w, Vb, c->fp32 ? 1 : 0, N, N, j, j + 1 < M ? 1 : 0, P,
                                       c->fp32 ? c->pM : c->pA, c->pB,
                                       c->colcnt + column_counter_offset(j), st, c->col_ctas, s);
        if (e == cudaSuccess) {
            c->launches++;
            continue;
        }
        if (e != cudaErrorNotSupported || c->fp32) return ROK_ERR_CUDA;
        (void)cudaGetLastError();
        // <v_1, w> and ||w||^2
        CU(c->ops->dot2(c->V, c->w, c->w, c->w, N, c->pA, P, &st->active, s));
        c->launches++;
        double *pin = c->pA, *pout = c->pB;
        for (int i = 1; i <= j + 1; ++i) {
            const double *vnext = i <= j ? c->V + (size_t)i * N : nullptr;
            CU(c->ops->mgs(c->w, c->V + (size_t)(i - 1) * N, vnext, N, pin, P,
                           &st->H[(i - 1) * kMaxKrylov + j], pout, i == 1, st, s));
            c->launches++;
            double *t = pin; pin = pout; pout = t;
        }
        if (j + 1 < M) {
            CU(c->ops->normalize(c->w, c->V + (size_t)(j + 1) * N, N, pin, P, &st->H[(j + 1) * kMaxKrylov + j],
                                 j + 1, st, s));
            c->launches++;
        }
    }
    return ROK_OK;
}

// ---- ROK4 step, enqueue only ------------------------------------------------------
// The step size h, h gamma, M_eff and the Arnoldi flag live in the device step
// state (written by launch_begin before this body), so the body can be captured
// once in a CUDA graph and replayed for any h.
rok_status enqueue_rok_body(rok_ctx *c, double *y, int M)
{
    const size_t N = c->N;
    const int P = c->P;
    StepState *st = c->st;
    cudaStream_t s = c->stream;
    c->launches += 2;
    // F1 = f(y_n)
    rok_status r = stencil(c, io_plain(c, y, c->F[0]));
    if (r != ROK_OK) return r;
    // eps from ||y_n|| (unit basis vectors)
    CU(c->ops->dot2(y, y, nullptr, nullptr, N, c->pA, P, nullptr, s));
    CU(c->ops->eps(c->pA, P, true, 0.0, st, s));
    c->launches += 2;
    void *Vb = c->fp32 ? (void *)c->Vf : (void *)c->V;
    if (M > 0) {
        // v_1 = F1 / ||F1|| (in the basis precision)
        CU(c->ops->first_vector(c->F[0], Vb, c->fp32 ? 1 : 0, N, c->pA, P, st, s));
        c->launches += 2;
        rok_status ra = arnoldi_columns(c, y, M);
        if (ra != ROK_OK) return ra;
        CU(c->ops->lu(st, s));
        c->launches++;
    }
    for (int i = 0; i < 4; ++i) {
        if (i > 0) {
            StencilIO io = io_plain(c, y, c->F[i]);
            for (int j = 0; j < i; ++j)
                if (kRokAlpha[i][j] != 0.0) {
                    io.add[io.nadd] = c->K[j];
                    io.coef[io.nadd] = kRokAlpha[i][j];
                    io.nadd++;
                }
            if ((r = stencil(c, io)) != ROK_OK) return r;
        }
        if (M > 0) {
            CU(c->ops->multidot(c->F[i], Vb, c->fp32 ? 1 : 0, N, N, c->pM, P, st, s));
            CU(c->ops->stage_solve(i, kRokGammaOff[i], c->pM, P, st, s));
            c->launches += 2;
        }
        CU(c->ops->stage_vec(c->K[i], c->F[i], Vb, c->fp32 ? 1 : 0, N, N, i, st, c->egrid, s));
        c->launches++;
    }
    const double *kv[4] = {c->K[0], c->K[1], c->K[2], c->K[3]};
    CU(c->ops->axpy_n(y, y, kv, kRokB, 4, N, st, c->egrid, s));
    c->launches++;
    return ROK_OK;
}

// pairwise (aligned binary tree) sum of p[0..n), zero-padded to a power of two
double host_tree(const double *p, int n)
{
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    std::vector<double> b(n2, 0.0);
    for (int i = 0; i < n; ++i) b[i] = p[i];
    for (int len = n2; len > 1; len >>= 1)
        for (int i = 0; i < len / 2; ++i) b[i] = b[2 * i] + b[2 * i + 1];
    return b[0];
}

double host_norm(rok_ctx *c, const double *a, rok_status *err)
{
    cudaError_t e1 = c->ops->dot2(a, a, nullptr, nullptr, c->N, c->pA, c->P, nullptr, c->stream);
    cudaError_t e2 = cudaMemcpyAsync(c->h_part, c->pA, sizeof(double) * c->P, cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e3 = cudaStreamSynchronize(c->stream);
    c->launches++;
    if (e1 || e2 || e3) { *err = ROK_ERR_CUDA; return 0.0; }
    return sqrt(host_tree(c->h_part, c->P));
}

}  // namespace

// entry points of the forward machinery for the reverse step (adjoint.cu)
namespace rok_host {
rok_status enqueue_step_body(rok_ctx *c, double *y, int M) { return enqueue_rok_body(c, y, M); }
rok_status launch_stencil(rok_ctx *c, const StencilIO &io) { return stencil(c, io); }
StencilIO plain_io(rok_ctx *c, const double *y, double *out) { return io_plain(c, y, out); }
}  // namespace rok_host

// ============================== public entry points ==============================
extern "C" {

const char *rok_status_string(rok_status s)
{
    switch (s) {
    case ROK_OK: return "ok";
    case ROK_ERR_INVALID_ARG: return "invalid argument";
    case ROK_ERR_CUDA: return "CUDA runtime error";
    case ROK_ERR_NONFINITE: return "non-finite value in a residual or stage solve";
    case ROK_ERR_NOT_CONVERGED: return "Newton iteration did not converge";
    case ROK_ERR_TIMEOUT: return "bounded device wait expired";
    case ROK_ERR_UNSUPPORTED: return "unsupported in this build";
    case ROK_ERR_NOMEM: return "out of device memory";
    }
    return "unknown status";
}

rok_status rok_init(rok_ctx **out, const rok_problem_desc *d, void *stream)
{
    if (!out || !d) return ROK_ERR_INVALID_ARG;
    *out = nullptr;
    if (d->kind < ROK_EULER2D || d->kind > ROK_LORENZ96) return ROK_ERR_INVALID_ARG;
    if (d->krylov_max < 0 || d->krylov_max > kMaxKrylov) return ROK_ERR_INVALID_ARG;
    if (d->rounding != ROK_ROUND_FAST && d->rounding != ROK_ROUND_STRICT) return ROK_ERR_INVALID_ARG;
    if (d->basis != ROK_BASIS_FP64 && d->basis != ROK_BASIS_FP32) return ROK_ERR_INVALID_ARG;
    if (d->jvp != ROK_JVP_FD && d->jvp != ROK_JVP_EXACT) return ROK_ERR_INVALID_ARG;
    if (d->kind == ROK_LORENZ96) {
        if (d->nx < 4) return ROK_ERR_INVALID_ARG;
    } else {
        if (d->nx < 2 || d->ny < 2) return ROK_ERR_INVALID_ARG;
        if ((long long)d->nx * d->ny > (1LL << 28)) return ROK_ERR_INVALID_ARG;
        for (int k = 0; k < 4; ++k)
            if (d->bc[k] < ROK_BC_PERIODIC || d->bc[k] > ROK_BC_FARFIELD) return ROK_ERR_INVALID_ARG;
        if ((d->bc[0] == ROK_BC_PERIODIC) != (d->bc[1] == ROK_BC_PERIODIC)) return ROK_ERR_INVALID_ARG;
        if ((d->bc[2] == ROK_BC_PERIODIC) != (d->bc[3] == ROK_BC_PERIODIC)) return ROK_ERR_INVALID_ARG;
        if ((d->xv == nullptr) != (d->yv == nullptr)) return ROK_ERR_INVALID_ARG;
        if (!(d->gamma > 1.0)) return ROK_ERR_INVALID_ARG;
        if (d->xv == nullptr) {
            if (!(d->lx > 0.0) || !(d->ly > 0.0)) return ROK_ERR_INVALID_ARG;
            for (int k = 0; k < 4; ++k)   // the uniform-grid stencil is periodic only
                if (d->bc[k] != ROK_BC_PERIODIC) return ROK_ERR_UNSUPPORTED;
        }
        if (d->kind == ROK_NS2D && (!(d->prandtl > 0.0) || d->mu < 0.0)) return ROK_ERR_INVALID_ARG;
        if (d->kind == ROK_NS2D && d->sutherland_s > 0.0 && !(d->t_ref > 0.0)) return ROK_ERR_INVALID_ARG;
    }
    rok_ctx *c = new rok_ctx();
    c->d = *d;
    c->d.xv = c->d.yv = nullptr;
    c->kind = d->kind;
    c->strict = d->rounding == ROK_ROUND_STRICT;
    c->curv = d->kind != ROK_LORENZ96 && d->xv != nullptr;
    c->fp32 = d->basis == ROK_BASIS_FP32;
    c->exact_jvp = d->jvp == ROK_JVP_EXACT;
    c->stream = (cudaStream_t)stream;
    c->mmax = d->krylov_max;
    c->nc = d->kind == ROK_LORENZ96 ? (size_t)d->nx : (size_t)d->nx * d->ny;
    c->N = d->kind == ROK_LORENZ96 ? (size_t)d->nx : 4 * c->nc;

    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->P = reduction_blocks(c->N);
    c->egrid = 8 * sms;
    c->ops = c->strict ? &strict::ops : &fast::ops;

    StencilConsts &C = c->C;
    memset(&C, 0, sizeof(C));
    C.nx = d->nx;
    C.ny = d->kind == ROK_LORENZ96 ? 1 : d->ny;
    for (int k = 0; k < 4; ++k) C.bc[k] = d->bc[k];
    C.viscous = d->kind == ROK_NS2D;
    C.sutherland = d->kind == ROK_NS2D && d->sutherland_s > 0.0;
    C.gm1 = d->gamma - 1.0;
    C.inv_gm1 = 1.0 / C.gm1;
    C.c_lo = 0.25 * (1.0 - d->muscl_kappa);
    C.c_hi = 0.25 * (1.0 + d->muscl_kappa);
    C.efix = d->entropy_fix;
    C.kfac = d->kind == ROK_NS2D ? d->gamma / (C.gm1 * d->prandtl) : 0.0;
    C.c23 = 2.0 / 3.0;
    C.g_over_pr = d->kind == ROK_NS2D ? d->gamma / d->prandtl : 0.0;
    C.mu = d->kind == ROK_NS2D ? d->mu : 0.0;
    C.inv_tref = C.sutherland ? 1.0 / d->t_ref : 0.0;
    C.suth_s = d->sutherland_s;
    if (d->kind != ROK_LORENZ96) {
        double dx = d->lx / d->nx, dy = d->ly / d->ny;
        C.rdx = d->xv ? 0.0 : 1.0 / dx;
        C.rdy = d->xv ? 0.0 : 1.0 / dy;
        C.q_rdx = 0.25 * C.rdx;
        C.q_rdy = 0.25 * C.rdy;
        to_prim_host(*d, C, d->q_inf, C.prim_inf);
        set_fast_consts(C);
    }
    C.lorenz_f = d->lorenz_f;

    const size_t N = c->N;
    auto al = [&](double **p, size_t n) { return cudaMalloc(p, n * sizeof(double)) == cudaSuccess; };
    bool ok = al(&c->V, (size_t)(c->mmax + 1) * N) && al(&c->w, N) && al(&c->t0, N) && al(&c->t1, N) &&
              al(&c->t2, N) && al(&c->pA, 4 * (size_t)c->P) && al(&c->pB, 2 * (size_t)c->P) &&
              al(&c->pM, (size_t)(kMaxKrylov + 2) * c->P);
    for (int i = 0; i < 4 && ok; ++i) ok = al(&c->F[i], N) && al(&c->K[i], N);
    if (ok && c->fp32) ok = cudaMalloc(&c->Vf, (size_t)(c->mmax + 1) * N * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&c->st, sizeof(StepState)) == cudaSuccess;
    ok = ok && cudaMalloc(&c->colcnt, column_counter_offset(kMaxKrylov) * sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMallocHost(&c->h_st, sizeof(StepState)) == cudaSuccess;
    ok = ok && cudaMallocHost(&c->h_part, sizeof(double) * 2 * (kMaxKrylov + 2) * (size_t)c->P) == cudaSuccess;
    if (!ok) { free_ctx(c); return ROK_ERR_NOMEM; }
    if (cudaMemset(c->st, 0, sizeof(StepState)) != cudaSuccess) { free_ctx(c); return ROK_ERR_CUDA; }
    c->col_ctas = c->ops->arnoldi_column_ctas(sms);
    if (c->fp32 && (c->col_ctas <= 0 || (c->P + c->col_ctas - 1) / c->col_ctas > 2)) {
        // the binary32 basis runs on the persistent column kernel only
        free_ctx(c);
        return ROK_ERR_UNSUPPORTED;
    }
    memset(c->h_st, 0, sizeof(StepState));
    if (c->curv) {
        c->d.xv = d->xv; c->d.yv = d->yv;   // used only while building the metrics
        rok_status s = build_geometry(c);
        c->d.xv = c->d.yv = nullptr;
        if (s != ROK_OK) { free_ctx(c); return s; }
    }
    *out = c;
    return ROK_OK;
}

rok_status rok_destroy(rok_ctx *c)
{
    if (!c) return ROK_OK;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
    return ROK_OK;
}

rok_status rok_set_persistent(rok_ctx *c, int enable)
{
    if (!c) return ROK_ERR_INVALID_ARG;
    if (c->fp32 && !enable) return ROK_ERR_UNSUPPORTED;   // the binary32 basis needs the column kernel
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return ROK_ERR_CUDA;
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    c->graph_launches.clear();
    c->persistent = enable != 0;
    return ROK_OK;
}

rok_status rok_set_stream(rok_ctx *c, void *stream)
{
    if (!c) return ROK_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->stream);
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    c->graph_launches.clear();
    c->stream = (cudaStream_t)stream;
    return ROK_OK;
}

rok_status rok_residual(rok_ctx *c, const double *y, double *f)
{
    if (!c || !y || !f || y == f) return ROK_ERR_INVALID_ARG;
    return stencil(c, io_plain(c, y, f));
}

rok_status rok_jvp(rok_ctx *c, const double *y, const double *fy, const double *v, double *jv, double eps, int mode)
{
    if (!c || !y || !v || !jv || jv == y || jv == v) return ROK_ERR_INVALID_ARG;
    if (mode == ROK_JVP_EXACT) {
        StencilIO io = io_plain(c, y, jv);
        io.dir = v;
        return stencil(c, io);
    }
    if (mode != ROK_JVP_FD) return ROK_ERR_INVALID_ARG;
    rok_status r;
    if (!fy) {
        if ((r = stencil(c, io_plain(c, y, c->t0))) != ROK_OK) return r;
        fy = c->t0;
    }
    // ||y||^2 and ||v||^2 for the automatic increment
    CU(c->ops->dot2(y, y, v, v, c->N, c->pA, c->P, nullptr, c->stream));
    CU(c->ops->eps(c->pA, c->P, false, eps, c->st, c->stream));
    c->launches += 2;
    return stencil(c, io_jvp(c, y, v, fy, jv));
}

rok_status rok_arnoldi(rok_ctx *c, const double *y, int M, double *Vout, double *Hout, int *m_eff)
{
    if (!c || !y || !Vout || !Hout || !m_eff || M < 1 || M > c->mmax) return ROK_ERR_INVALID_ARG;
    const size_t N = c->N;
    const int P = c->P;
    StepState *st = c->st;
    cudaStream_t s = c->stream;
    CU(launch_begin(st, 0.0, kRokGamma, M, s));
    rok_status r = stencil(c, io_plain(c, y, c->F[0]));
    if (r != ROK_OK) return r;
    CU(c->ops->dot2(y, y, nullptr, nullptr, N, c->pA, P, nullptr, s));
    CU(c->ops->eps(c->pA, P, true, 0.0, st, s));
    CU(c->ops->first_vector(c->F[0], c->fp32 ? (void *)c->Vf : (void *)c->V, c->fp32 ? 1 : 0, N, c->pA, P, st, s));
    CU(cudaMemsetAsync(st->H, 0, sizeof(st->H), s));
    c->launches += 5;
    if ((r = arnoldi_columns(c, y, M)) != ROK_OK) return r;
    r = sync_read(c, nullptr);
    int me = c->h_st->meff;
    *m_eff = me;
    if (c->fp32) CU(launch_f2d(c->Vf, Vout, (size_t)me * N, s));   // exact widening
    else CU(cudaMemcpyAsync(Vout, c->V, (size_t)me * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpy2DAsync(Hout, M * sizeof(double), st->H, kMaxKrylov * sizeof(double), M * sizeof(double), M,
                         cudaMemcpyDeviceToDevice, s));
    CU(cudaStreamSynchronize(s));
    // entries beyond the built basis are zero
    if (me < M) {
        std::vector<double> hh((size_t)M * M);
        CU(cudaMemcpy(hh.data(), Hout, hh.size() * sizeof(double), cudaMemcpyDeviceToHost));
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j)
                if (i >= me || j >= me) hh[(size_t)i * M + j] = 0.0;
        CU(cudaMemcpy(Hout, hh.data(), hh.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    return r;
}

rok_status rok_step(rok_ctx *c, double *y, double h, int M, rok_step_info *info)
{
    if (!c || !y || M < 0 || M > c->mmax || !(h > 0.0) || !isfinite(h)) return ROK_ERR_INVALID_ARG;
    if (c->kind == ROK_LORENZ96 && (size_t)M > c->N) return ROK_ERR_INVALID_ARG;
    c->last = rok_step_info{};
    c->last.residual_evals = 1 + M + 3;
    c->last.jvps = M;
    CU(launch_begin(c->st, h, kRokGamma, M, c->stream));
    c->launches++;
    if (c->use_graph && !c->time_stencil) {
        // graphs are captured and replayed on a private non-blocking stream fenced
        // by events to the caller's stream (capture is not allowed on the legacy
        // default stream)
        cudaStream_t user = c->stream;
        if (!c->gstream) {
            CU(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
            CU(cudaEventCreateWithFlags(&c->gev[0], cudaEventDisableTiming));
            CU(cudaEventCreateWithFlags(&c->gev[1], cudaEventDisableTiming));
        }
        CU(cudaEventRecord(c->gev[0], user));
        CU(cudaStreamWaitEvent(c->gstream, c->gev[0], 0));
        auto key = std::make_pair(y, M);
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            cudaGraph_t g;
            long long l0 = c->launches;
            c->capturing = true;
            c->stream = c->gstream;
            cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
            rok_status r = e == cudaSuccess ? enqueue_rok_body(c, y, M) : ROK_ERR_CUDA;
            cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(c->gstream, &g) : e;
            c->stream = user;
            c->capturing = false;
            if (r != ROK_OK) return r;
            if (e2 != cudaSuccess) return ROK_ERR_CUDA;
            cudaGraphExec_t ge;
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return ROK_ERR_CUDA;
            it = c->graphs.emplace(key, ge).first;
            c->graph_launches[key] = c->launches - l0;
            c->launches = l0;
        }
        CU(cudaGraphLaunch(it->second, c->gstream));
        CU(cudaEventRecord(c->gev[1], c->gstream));
        CU(cudaStreamWaitEvent(user, c->gev[1], 0));
        c->launches += c->graph_launches[key];
        if (info) return sync_read(c, info);
        return ROK_OK;
    }
    rok_status r = enqueue_rok_body(c, y, M);
    if (r != ROK_OK) return r;
    if (info) return sync_read(c, info);
    return ROK_OK;
}

rok_status rk_step(rok_ctx *c, double *y, double h, rok_step_info *info)
{
    if (!c || !y || !(h > 0.0) || !isfinite(h)) return ROK_ERR_INVALID_ARG;
    rok_status r;
    for (int i = 0; i < 4; ++i) {
        StencilIO io = io_plain(c, y, c->K[i]);
        for (int j = 0; j < i; ++j)
            if (kRk4A[i][j] != 0.0) {
                io.add[io.nadd] = c->K[j];
                io.coef[io.nadd] = h * kRk4A[i][j];
                io.nadd++;
            }
        if ((r = stencil(c, io)) != ROK_OK) return r;
    }
    const double *kv[4] = {c->K[0], c->K[1], c->K[2], c->K[3]};
    double cb[4];
    for (int j = 0; j < 4; ++j) cb[j] = h * kRk4B[j];
    CU(c->ops->axpy_n(y, y, kv, cb, 4, c->N, c->st, c->egrid, c->stream));
    c->launches++;
    c->last = rok_step_info{};
    c->last.residual_evals = 4;
    if (info) return sync_read(c, info);
    return ROK_OK;
}

// x = (I - hg J_n)^{-1} rhs by restarted GMRES(m) from x0 = 0, on the device:
// the Arnoldi columns of (I - hg J_n) by modified Gram-Schmidt (the persistent
// column kernel where it fits, else one launch per pass), the Givens rotations
// of the Hessenberg columns, the residual estimate and the stop decision in the
// step state.  The host enqueues one whole restart cycle (m columns; the
// columns after a stop are skipped on the device: the JVP and the column kernel
// check the Arnoldi flag) and reads the GMRES state once per cycle.  Stops at
// ||rhs - op(x)|| <= tol ||rhs|| (the least-squares estimate).  J_n at y is
// applied by the FD product with base F0 = f(y) (or exactly).  Uses c->V, the
// step state's H, c->w and c->F[1] as workspace; rhs and x must be other buffers.
static rok_status gmres_solve(rok_ctx *c, const double *y, const double *F0, double hg, const double *rhs,
                              double *x, const esdirk_opts &op, int *its_out, bool *conv_out, int *jvps,
                              int *res_evals)
{
    const size_t N = c->N;
    const int P = c->P;
    const int m = op.gmres_m;
    StepState *st = c->st;
    cudaStream_t s = c->stream;
    double *wv = c->w;
    rok_status r;
    // op(v) = v - h g J_n v into out; skipped on the device when *active == 0
    auto apply_op = [&](const double *v, double *out, const int *active) -> rok_status {
        StencilIO io;
        if (c->exact_jvp) {
            io = io_plain(c, y, out);
            io.dir = v;
        } else {
            io = io_jvp(c, y, v, F0, out);
        }
        io.add_out = v;
        io.s2 = -hg;
        io.active = active;
        return stencil(c, io);
    };
    const bool persistent = c->col_ctas > 0 && c->persistent;
    CU(cudaMemsetAsync(x, 0, N * sizeof(double), s));
    CU(c->ops->dot2(rhs, rhs, nullptr, nullptr, N, c->pA, P, nullptr, s));
    CU(c->ops->gmres_start(c->pA, P, op.gmres_tol, m, st, s));
    c->launches += 2;
    int restarts_applied = 0;
    bool conv = false;
    const GmresState &hgm = c->h_st->gm;
    for (int cycle = 0; cycle <= op.gmres_restarts; ++cycle) {
        const double *r0 = rhs;
        if (cycle > 0) {
            // r0 = rhs - op(x)
            if ((r = apply_op(x, wv, nullptr)) != ROK_OK) return r;
            restarts_applied++;
            const double *vv[1] = {wv};
            double cc[1] = {-1.0};
            CU(c->ops->axpy_n(c->F[1], rhs, vv, cc, 1, N, nullptr, c->egrid, s));
            c->launches++;
            r0 = c->F[1];
        }
        // beta = ||r0||, stop test, g = beta e_1; v_0 = r0 / beta
        CU(c->ops->dot2(r0, r0, nullptr, nullptr, N, c->pA, P, nullptr, s));
        CU(c->ops->gmres_cycle(c->pA, P, st, s));
        CU(c->ops->first_vector(r0, c->V, 0, N, c->pB, P, st, s));
        c->launches += 4;
        if (persistent) CU(cudaMemsetAsync(c->colcnt, 0, column_counter_offset(m) * sizeof(unsigned), s));
        for (int j = 0; j < m; ++j) {
            if ((r = apply_op(c->V + (size_t)j * N, wv, &st->active)) != ROK_OK) return r;
            cudaError_t e = cudaErrorNotSupported;
            if (persistent)
                e = c->ops->arnoldi_column(wv, c->V, 0, N, N, j, 1, P, c->pA, c->pB,
                                           c->colcnt + column_counter_offset(j), st, c->col_ctas, s);
            if (e == cudaSuccess) {
                c->launches++;
            } else {
                if (e != cudaErrorNotSupported) return ROK_ERR_CUDA;
                (void)cudaGetLastError();
                CU(c->ops->dot2(c->V, wv, wv, wv, N, c->pA, P, &st->active, s));
                double *pin = c->pA, *pout = c->pB;
                for (int q = 1; q <= j + 1; ++q) {
                    const double *vnext = q <= j ? c->V + (size_t)q * N : nullptr;
                    CU(c->ops->mgs(wv, c->V + (size_t)(q - 1) * N, vnext, N, pin, P,
                                   &st->H[(q - 1) * kMaxKrylov + j], pout, q == 1, st, s));
                    double *t = pin;
                    pin = pout;
                    pout = t;
                }
                CU(c->ops->normalize(wv, c->V + (size_t)(j + 1) * N, N, pin, P,
                                     &st->H[(j + 1) * kMaxKrylov + j], j + 1, st, s));
                c->launches += 3 + j;
            }
            CU(c->ops->gmres_givens(j, st, s));
            c->launches++;
        }
        // x += V y with R y = g (no-op when the cycle started converged)
        CU(c->ops->gmres_lsq(st, s));
        CU(c->ops->basis_combine(x, x, c->V, N, N, m, st->gcoef, &st->gm.k, c->egrid, s));
        CU(cudaMemcpyAsync(&c->h_st->gm, &st->gm, sizeof(GmresState), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        c->launches += 2;
        if (hgm.conv) {
            conv = true;
            break;
        }
    }
    *its_out = hgm.its;
    *conv_out = conv;
    *jvps += hgm.its + restarts_applied;
    *res_evals += hgm.its + restarts_applied;
    return ROK_OK;
}

static rok_status check_gmres_opts(const rok_ctx *c, const esdirk_opts &op)
{
    if (op.gmres_m < 1 || op.gmres_m > c->mmax || op.gmres_m > kMaxKrylov || op.gmres_restarts < 0 ||
        op.newton_max < 1 || !(op.gmres_tol > 0.0) || !(op.newton_tol > 0.0))
        return ROK_ERR_INVALID_ARG;
    return ROK_OK;
}

rok_status esdirk_step(rok_ctx *c, double *y, double h, const esdirk_opts *o, rok_step_info *info)
{
    if (!c || !y || !(h > 0.0) || !isfinite(h)) return ROK_ERR_INVALID_ARG;
    esdirk_opts op = {30, 1e-6, 5, 1e-10, 10};
    if (o) op = *o;
    if (check_gmres_opts(c, op) != ROK_OK) return ROK_ERR_INVALID_ARG;
    const size_t N = c->N;
    const int P = c->P;
    StepState *st = c->st;
    cudaStream_t s = c->stream;
    const double hg = h * kEsdGamma;
    rok_status r, err = ROK_OK;
    int newton_total = 0, gmres_total = 0, res_evals = 0, jvps = 0;
    bool converged = true;
    // k_1 = f(y_n); J_n products use eps from ||y_n||
    if ((r = stencil(c, io_plain(c, y, c->K[0]))) != ROK_OK) return r;
    CU(c->ops->dot2(y, y, nullptr, nullptr, N, c->pA, P, nullptr, s));
    CU(c->ops->eps(c->pA, P, true, 0.0, st, s));
    c->launches += 2;
    res_evals++;
    double *xi = c->t0, *rhs = c->t1, *dk = c->t2;
    for (int i = 1; i < 4; ++i) {
        // xi_i = y_n + h sum_{j<i} a_ij k_j
        const double *kv[4];
        double cf[4];
        int cnt = 0;
        for (int j = 0; j < i; ++j)
            if (kEsdA[i][j] != 0.0) { kv[cnt] = c->K[j]; cf[cnt] = h * kEsdA[i][j]; cnt++; }
        CU(c->ops->axpy_n(xi, y, kv, cf, cnt, N, nullptr, c->egrid, s));
        CU(cudaMemcpyAsync(c->K[i], c->K[i - 1], N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        c->launches++;
        bool conv = false;
        for (int it = 0; it < op.newton_max; ++it) {
            // rhs = -G(k) = f(xi + h g k) - k
            StencilIO io = io_plain(c, xi, rhs);
            io.add[0] = c->K[i];
            io.coef[0] = hg;
            io.nadd = 1;
            io.sub = c->K[i];
            if ((r = stencil(c, io)) != ROK_OK) return r;
            res_evals++;
            // GMRES(m) for (I - h g J_n) dk = rhs, x0 = 0
            int its = 0;
            bool gconv = false;
            if ((r = gmres_solve(c, y, c->K[0], hg, rhs, dk, op, &its, &gconv, &jvps, &res_evals)) != ROK_OK)
                return r;
            gmres_total += its;
            newton_total++;
            // k += dk; test h g ||dk|| <= tol ||xi + h g k||
            const double *dv[1] = {dk};
            double one[1] = {1.0};
            CU(c->ops->axpy_n(c->K[i], c->K[i], dv, one, 1, N, nullptr, c->egrid, s));
            const double *kv2[1] = {c->K[i]};
            double hgc[1] = {hg};
            CU(c->ops->axpy_n(c->F[2], xi, kv2, hgc, 1, N, nullptr, c->egrid, s));
            c->launches += 2;
            double dn = host_norm(c, dk, &err);
            if (err) return err;
            double yn = host_norm(c, c->F[2], &err);
            if (err) return err;
            if (hg * dn <= op.newton_tol * yn) { conv = true; break; }
        }
        converged = converged && conv;
    }
    const double *kv[4] = {c->K[0], c->K[1], c->K[2], c->K[3]};
    double cb[4];
    for (int j = 0; j < 4; ++j) cb[j] = h * kEsdB[j];
    CU(c->ops->axpy_n(converged ? y : c->t0, y, kv, cb, 4, N, st, c->egrid, s));
    c->launches++;
    c->last = rok_step_info{};
    c->last.residual_evals = res_evals;
    c->last.jvps = jvps;
    c->last.newton_iters = newton_total;
    c->last.gmres_iters = gmres_total;
    rok_status rs = sync_read(c, nullptr);
    c->last.newton_iters = newton_total;
    c->last.gmres_iters = gmres_total;
    c->last.residual_evals = res_evals;
    c->last.jvps = jvps;
    if (rs == ROK_OK && !converged) rs = ROK_ERR_NOT_CONVERGED;
    c->last.status = rs;
    if (info) *info = c->last;
    return rs;
}

// Coefficients of Eq. ROS for a Rosenbrock method: ROS4 is published for the
// transformed stages u_i = h sum_j gamma_ij k_j, so Gamma = (diag(1/g) - C)^{-1}
// (lower triangular, by substitution), alpha = A Gamma, b = m Gamma; ROW is
// published in the form of Eq. ROS.
static void ros_tableau(int method, double al[4][4], double ga[4][4], double b[4], double *g)
{
    if (method == ROK_ROS_ROW) {
        *g = kRowGamma;
        for (int i = 0; i < 4; ++i) {
            b[i] = kRowB[i];
            for (int j = 0; j < 4; ++j) {
                al[i][j] = kRowAlpha[i][j];
                ga[i][j] = kRowGammaOff[i][j];
            }
        }
        return;
    }
    const double gg = kRos4Gamma;
    double Gam[4][4] = {};
    // columns of the inverse of L = diag(1/g) - C (lower triangular)
    for (int col = 0; col < 4; ++col)
        for (int i = col; i < 4; ++i) {
            double t = i == col ? 1.0 : 0.0;
            for (int k = col; k < i; ++k) t += kRos4C[i][k] * Gam[k][col];
            Gam[i][col] = t * gg;
        }
    *g = gg;
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) {
            double t = 0.0;
            for (int k = 0; k < 4; ++k) t += kRos4A[i][k] * Gam[k][j];
            al[i][j] = t;
            ga[i][j] = j < i ? Gam[i][j] : 0.0;
        }
        double t = 0.0;
        for (int k = 0; k < 4; ++k) t += kRos4M[k] * Gam[k][i];
        b[i] = t;
    }
}

rok_status ros_step(rok_ctx *c, double *y, double h, int method, const esdirk_opts *o, rok_step_info *info)
{
    if (!c || !y || !(h > 0.0) || !isfinite(h)) return ROK_ERR_INVALID_ARG;
    if (method != ROK_ROS_ROS4 && method != ROK_ROS_ROW) return ROK_ERR_INVALID_ARG;
    esdirk_opts op = {30, 1e-6, 5, 1e-10, 10};
    if (o) op = *o;
    if (check_gmres_opts(c, op) != ROK_OK) return ROK_ERR_INVALID_ARG;
    const size_t N = c->N;
    const int P = c->P;
    StepState *st = c->st;
    cudaStream_t s = c->stream;
    double al[4][4], ga[4][4], bw[4], g;
    ros_tableau(method, al, ga, bw, &g);
    const double hg = h * g;
    rok_status r;
    int gmres_total = 0, res_evals = 0, jvps = 0;
    bool converged = true;
    // F0 = f(y_n) (first right-hand side and base of the FD products); eps from ||y_n||
    double *F0 = c->F[0], *xi = c->t0, *rhs = c->t1, *u = c->F[2];
    if ((r = stencil(c, io_plain(c, y, F0))) != ROK_OK) return r;
    CU(c->ops->dot2(y, y, nullptr, nullptr, N, c->pA, P, nullptr, s));
    CU(c->ops->eps(c->pA, P, true, 0.0, st, s));
    c->launches += 2;
    res_evals++;
    for (int i = 0; i < 4; ++i) {
        const double *frhs = F0;
        if (i > 0) {
            // Y_i = y_n + h sum_{j<i} alpha_ij k_j; rhs = f(Y_i)
            const double *kv[4];
            double cf[4];
            int cnt = 0;
            for (int j = 0; j < i; ++j)
                if (al[i][j] != 0.0) { kv[cnt] = c->K[j]; cf[cnt] = h * al[i][j]; cnt++; }
            CU(c->ops->axpy_n(xi, y, kv, cf, cnt, N, nullptr, c->egrid, s));
            c->launches++;
            if ((r = stencil(c, io_plain(c, xi, rhs))) != ROK_OK) return r;
            res_evals++;
            // rhs += h J_n sum_{j<i} gamma_ij k_j
            cnt = 0;
            for (int j = 0; j < i; ++j)
                if (ga[i][j] != 0.0) { kv[cnt] = c->K[j]; cf[cnt] = ga[i][j]; cnt++; }
            if (cnt > 0) {
                CU(c->ops->axpy_n(u, nullptr, kv, cf, cnt, N, nullptr, c->egrid, s));
                c->launches++;
                StencilIO io;
                if (c->exact_jvp) {
                    io = io_plain(c, y, rhs);
                    io.dir = u;
                } else {
                    io = io_jvp(c, y, u, F0, rhs);
                }
                io.add_out = rhs;
                io.s2 = h;
                if ((r = stencil(c, io)) != ROK_OK) return r;
                jvps++;
                res_evals++;
            }
            frhs = rhs;
        }
        // (I - h g J_n) k_i = rhs by GMRES(m) from 0
        int its = 0;
        bool gconv = false;
        if ((r = gmres_solve(c, y, F0, hg, frhs, c->K[i], op, &its, &gconv, &jvps, &res_evals)) != ROK_OK) return r;
        gmres_total += its;
        converged = converged && gconv;
    }
    const double *kv[4] = {c->K[0], c->K[1], c->K[2], c->K[3]};
    double cb[4];
    for (int j = 0; j < 4; ++j) cb[j] = h * bw[j];
    CU(c->ops->axpy_n(converged ? y : c->t0, y, kv, cb, 4, N, st, c->egrid, s));
    c->launches++;
    c->last = rok_step_info{};
    rok_status rs = sync_read(c, nullptr);
    c->last.gmres_iters = gmres_total;
    c->last.residual_evals = res_evals;
    c->last.jvps = jvps;
    if (rs == ROK_OK && !converged) rs = ROK_ERR_NOT_CONVERGED;
    c->last.status = rs;
    if (info) *info = c->last;
    return rs;
}

rok_status rok_dt_from_cfl(rok_ctx *c, const double *y, double cfl, double *dt)
{
    if (!c || !y || !dt || !(cfl > 0.0)) return ROK_ERR_INVALID_ARG;
    if (c->kind == ROK_LORENZ96) return ROK_ERR_UNSUPPORTED;
    CU(launch_cfl(y, c->C, c->cfl_six, c->cfl_siy, c->cfl_sjx, c->cfl_sjy, c->cfl_vol, c->pA, c->P, c->stream));
    CU(cudaMemcpyAsync(c->h_part, c->pA, sizeof(double) * c->P, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->launches++;
    double m = 0.0;
    for (int b = 0; b < c->P; ++b) m = fmax(m, c->h_part[b]);
    if (!(m > 0.0) || !isfinite(m)) return ROK_ERR_NONFINITE;
    *dt = cfl / m;
    return ROK_OK;
}

rok_status rok_sync(rok_ctx *c, rok_step_info *info)
{
    if (!c) return ROK_ERR_INVALID_ARG;
    return sync_read(c, info);
}

rok_status rok_set_graph(rok_ctx *c, int enable)
{
    if (!c) return ROK_ERR_INVALID_ARG;
    c->use_graph = enable != 0;
    return ROK_OK;
}

rok_status rok_get_counters(rok_ctx *c, rok_counters *out, int reset)
{
    if (!c || !out) return ROK_ERR_INVALID_ARG;
    if (!c->ev_used.empty()) {
        CU(cudaStreamSynchronize(c->stream));
        for (auto &e : c->ev_used) {
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, e.first, e.second));
            c->stencil_ms += ms;
            c->stencil_timed++;
            c->ev_free.push_back(e);
        }
        c->ev_used.clear();
    }
    out->launches = c->launches;
    out->stencil_launches = c->stencil_launches;
    out->stencil_ms = c->stencil_ms;
    out->stencil_timed = c->stencil_timed;
    if (reset) {
        c->launches = c->stencil_launches = c->stencil_timed = 0;
        c->stencil_ms = 0.0;
    }
    return ROK_OK;
}

rok_status rok_set_stencil_timing(rok_ctx *c, int enable)
{
    if (!c) return ROK_ERR_INVALID_ARG;
    c->time_stencil = enable != 0;
    return ROK_OK;
}

}  // extern "C"
