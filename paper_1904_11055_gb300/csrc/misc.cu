// Small helper kernels.
#include <algorithm>

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

// L_ell(mu) by Bonnet's recurrence, (n+1) P_{n+1} = (2n+1) mu P_n - n P_{n-1}
PS_DEV double legendre(int ell, double mu) {
    double p0 = 1.0, p1 = mu;
    if (ell == 0) return p0;
    for (int n = 1; n < ell; n++) {
        const double p2 = ((2.0 * n + 1.0) * mu * p1 - n * p0) / (n + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// Redshift-space multipoles: every mode of the pruned half spectrum
// fhat[((ky+K)(K+1) + kz)(2K+1) + kx+K] times L_ell(kz/|q|) (line of sight along z).
template <typename T>
__global__ void legendre_weight_kernel(const Cx<T>* __restrict__ fhat, int K, int ell, Cx<T>* __restrict__ out) {
    const int nk = 2 * K + 1;
    const int64_t n = (int64_t)nk * (K + 1) * nk;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % nk) - K;
        const int64_t line = i / nk;
        const int kz = (int)(line % (K + 1)), ky = (int)(line / (K + 1)) - K;
        const double q2 = (double)kx * kx + (double)ky * ky + (double)kz * kz;
        const double w = q2 > 0.0 ? legendre(ell, kz / sqrt(q2)) : 0.0;
        const Cx<T> v = fhat[i];
        out[i] = cx<T>((T)(w * v.re), (T)(w * v.im));
    }
}

}  // namespace ps

cudaError_t ps_legendre_weight(int is_double, const void* fhat, int K, int ell, void* out, cudaStream_t st) {
    const int64_t n = (int64_t)(2 * K + 1) * (K + 1) * (2 * K + 1);
    const unsigned nb = (unsigned)std::min<int64_t>(2048, (n + 255) / 256);
    if (is_double)
        ps::legendre_weight_kernel<double><<<nb, 256, 0, st>>>((const ps::Cx<double>*)fhat, K, ell,
                                                               (ps::Cx<double>*)out);
    else
        ps::legendre_weight_kernel<float><<<nb, 256, 0, st>>>((const ps::Cx<float>*)fhat, K, ell, (ps::Cx<float>*)out);
    return cudaGetLastError();
}

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
