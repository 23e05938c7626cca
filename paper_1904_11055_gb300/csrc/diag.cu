// Diagnostic: the bounded wait of the tensor-core pipelines, made to run out.
// A producer that never arrives is simulated by an mbarrier nobody arrives on;
// the waiting warp must give up after the clock budget, set the error word and
// return, leaving the context usable.
#include <cuda_runtime.h>

#include "../../include/polyspec.h"
#include "../../include/polyspec_diag.h"
#include "tc.cuh"

namespace ps {

__global__ void stalled_wait_kernel(int* __restrict__ err) {
    __shared__ uint64_t bar;
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);  // one arrival expected; none comes
        tc::mbar_fence_init();
        s_abort = 0;
    }
    __syncthreads();
    volatile int* abort = &s_abort;
    const bool done = tc::mbar_wait_warp(&bar, 0, abort);
    if (threadIdx.x == 0) *err = done ? 0 : tc::kErrTimeout;
}

}  // namespace ps

extern "C" int poly_diag_stalled_wait(double* ms_out) {
    int* d_err = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&d_err, sizeof(int)) || cudaMemset(d_err, 0xff, sizeof(int)) || cudaEventCreate(&e0) ||
        cudaEventCreate(&e1)) {
        cudaGetLastError();
        if (d_err) cudaFree(d_err);
        return POLY_ERR_CUDA;
    }
    cudaEventRecord(e0);
    ps::stalled_wait_kernel<<<1, 32>>>(d_err);
    cudaEventRecord(e1);
    int err = -1;
    cudaError_t ce = cudaGetLastError();
    if (!ce) ce = cudaMemcpy(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    float ms = 0.f;
    if (!ce) cudaEventElapsedTime(&ms, e0, e1);
    if (ms_out) *ms_out = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_err);
    if (ce) return POLY_ERR_CUDA;
    return err == ps::tc::kErrTimeout ? POLY_ERR_TIMEOUT : (err == 0 ? POLY_OK : POLY_ERR_CUDA);
}
