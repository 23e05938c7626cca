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

// Eight independent FMA chains per thread; the sum is stored so nothing folds away.
template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T* __restrict__ out) {
    const T b = (T)1.0000001, c = (T)1e-7;
    T a[8];
    for (int i = 0; i < 8; i++) a[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) a[i] = fma(a[i], b, c);
    }
    T s = 0;
    for (int i = 0; i < 8; i++) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace ps

extern "C" int poly_diag_fma_peak(int is_double, int iters, double* tflops_out, double* ms_out) {
    if (iters < 1 || iters > (1 << 24) || !tflops_out) return POLY_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) {
        cudaGetLastError();
        return POLY_ERR_CUDA;
    }
    const int blocks = sms * 16, threads = 256;
    void* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * 8) || cudaEventCreate(&e0) || cudaEventCreate(&e1)) {
        cudaGetLastError();
        if (out) cudaFree(out);
        if (e0) cudaEventDestroy(e0);
        return POLY_ERR_CUDA;
    }
    float ms = 0.f;
    for (int rep = 0; rep < 2; rep++) {
        cudaEventRecord(e0);
        if (is_double)
            ps::fma_peak_kernel<double><<<blocks, threads>>>(iters, (double*)out);
        else
            ps::fma_peak_kernel<float><<<blocks, threads>>>(iters, (float*)out);
        cudaEventRecord(e1);
    }
    cudaError_t ce = cudaGetLastError();
    if (!ce) ce = cudaEventSynchronize(e1);
    if (!ce) ce = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (ce) return POLY_ERR_CUDA;
    if (ms_out) *ms_out = ms;
    *tflops_out = 2.0 * blocks * threads * 8.0 * iters / (ms * 1e-3) / 1e12;
    return POLY_OK;
}

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
