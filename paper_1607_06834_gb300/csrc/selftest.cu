// Self-test of the bounded device waits of the persistent Gram-Schmidt column
// kernels: one CTA waits on an arrival counter that nothing advances, through
// the same wait routine, with a short poll limit.  The wait must give up,
// latch kStatusTimeout in the step state and return; the host reads it and
// restores the status the context had, so the context stays usable.  No GPU fault is involved.
#include <cuda_runtime.h>

#include "context.h"
#define ROK_NS selftest
#define ROK_LINALG_DEVICE_ONLY
#include "linalg_impl.cuh"

using namespace rok;
using namespace rok::selftest;

namespace {

__global__ void __launch_bounds__(RT) wait_selftest_kernel(const unsigned *cnt, int *status, long long polls,
                                                           int *returned)
{
    // two arrivals expected, none made: the wait can only end by its limit
    const bool ok = gen_wait(cnt, 2u, status, polls);
    if (threadIdx.x == 0) *returned = ok ? 1 : 2;
}

}  // namespace

extern "C" rok_status rok_selftest_wait(rok_ctx *c, long long polls, int *expired, double *ms)
{
    if (!c || !expired || polls < 1 || polls > kBarrierSpins) return ROK_ERR_INVALID_ARG;
    cudaStream_t s = c->stream;
    int *flag = nullptr;
    if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) return ROK_ERR_NOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rok_status r = ROK_OK;
    int h_status = 0, h_flag = 0, h_prev = 0;
    float t = 0.0f;
    // a status latched by an earlier step is kept and put back afterwards
    if (cudaMemcpyAsync(&h_prev, &c->st->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemsetAsync(c->colcnt, 0, sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess || cudaMemsetAsync(&c->st->status, 0, sizeof(int), s) != cudaSuccess ||
        cudaEventRecord(e0, s) != cudaSuccess) {
        r = ROK_ERR_CUDA;
    } else {
        wait_selftest_kernel<<<1, RT, 0, s>>>(c->colcnt, &c->st->status, polls, flag);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaMemcpyAsync(&h_status, &c->st->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
            cudaMemcpyAsync(&c->st->status, &h_prev, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            r = ROK_ERR_CUDA;
    }
    if (r == ROK_OK) {
        *expired = (h_flag == 2 && (h_status & kStatusTimeout)) ? 1 : 0;
        if (ms) *ms = t;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(flag);
    return r;
}
