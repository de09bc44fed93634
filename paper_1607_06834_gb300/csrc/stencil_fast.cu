// Residual stencil, FMA contraction allowed (default rounding mode): the
// uniform-grid faces use the restructured doubled-flux formulas, the Roe
// averages and the speed of sound come from reciprocal square roots.
#define ROK_NS fast
#define ROK_STENCIL_FAST
#include "stencil_impl.cuh"

// Self-test of the reciprocal the FMA-build stencil uses (no counterpart in the
// paper): r[k] = rcp(x[k]) for n inputs, one thread per entry.
namespace {
__global__ void rcp_selftest_kernel(const double *__restrict__ x, double *__restrict__ r, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        r[k] = rok::fast::rcp(x[k]);
}
}  // namespace

extern "C" rok_status rok_selftest_rcp(const double *x, double *r, long long n, void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!x || !r))) return ROK_ERR_INVALID_ARG;
    if (n == 0) return ROK_OK;
    const long long blocks = (n + 255) / 256;
    rcp_selftest_kernel<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, (cudaStream_t)cuda_stream>>>(x, r, n);
    return cudaGetLastError() == cudaSuccess ? ROK_OK : ROK_ERR_CUDA;
}
