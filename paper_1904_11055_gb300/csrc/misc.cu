// Small helper kernels.
#include "common.cuh"
#include "kernels.h"

namespace ps {

template <typename T>
__global__ void gather_cells_kernel(const T* __restrict__ in, size_t in_stride, int ns, const int32_t* __restrict__ idx,
                                    int64_t nw, T* __restrict__ out, size_t out_stride) {
    const int s = blockIdx.y;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x)
        out[(size_t)s * out_stride + w] = in[(size_t)s * in_stride + idx[w]];
}

}  // namespace ps

cudaError_t ps_gather_cells(int is_double, const void* in, size_t in_stride, int ns, const int32_t* idx, int64_t nw,
                            void* out, size_t out_stride, cudaStream_t st) {
    if (nw <= 0 || ns <= 0) return cudaSuccess;
    dim3 grid((unsigned)((nw + 255) / 256 < 2048 ? (nw + 255) / 256 : 2048), ns);
    if (is_double)
        ps::gather_cells_kernel<double><<<grid, 256, 0, st>>>((const double*)in, in_stride, ns, idx, nw, (double*)out,
                                                              out_stride);
    else
        ps::gather_cells_kernel<float><<<grid, 256, 0, st>>>((const float*)in, in_stride, ns, idx, nw, (float*)out,
                                                             out_stride);
    return cudaGetLastError();
}
