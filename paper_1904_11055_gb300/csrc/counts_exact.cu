// Exact polygon counts from integer closure maps (count_b of App. A and Eq. Ncalc,
// the number of closed n-gons of grid modes, evaluated without a long FP64 sum).
//
// A bin's legs split into a first group A (n - 3 legs, at least one) and the rest
// B (at most three).  The closure map of a group, G(p) = #{tuples of its shells'
// modes with q_1 + ... = p}, is the forward transform of the product of its
// counting fields divided by N^3; it is an integer, so the FP64 transform is
// rounded to it (and the rounding checked).  With no closure wrapping around the
// grid, count_b = sum_p G_A(p) G_B(-p) = sum_p G_A(p) G_B(p) (shells are symmetric
// under q -> -q), summed exactly in 64-bit integers over the cube |p_c| <= K'
// that holds A's support; the maps are real and even, so the half spectrum
// kz >= 0 serves with weight 2 off the kz = 0 plane.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace ps {

// out[x] = prod_t F[slot_t][x] over up to three slots (-1: none), natural layout, FP64
__global__ void prod_fields_kernel(const double* __restrict__ F, size_t n3, int s0, int s1, int s2,
                                   double* __restrict__ out) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n3; x += (size_t)gridDim.x * blockDim.x) {
        double v = F[(size_t)s0 * n3 + x];
        if (s1 >= 0) v *= F[(size_t)s1 * n3 + x];
        if (s2 >= 0) v *= F[(size_t)s2 * n3 + x];
        out[x] = v;
    }
}

// G[i] = round(Re fhat[i] / N^3); err set when a value lies 0.25 or more from an integer or the
// imaginary part is 0.25 or more (in units of N^3)
__global__ void round_map_kernel(const Cx<double>* __restrict__ fhat, size_t n, double inv_n3,
                                 long long* __restrict__ G, int* __restrict__ err) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double re = fhat[i].re * inv_n3, im = fhat[i].im * inv_n3;
        const double r = rint(re);
        if (fabs(re - r) >= 0.25 || fabs(im) >= 0.25 || r < 0.0) atomicExch(err, 1);
        G[i] = (long long)r;
    }
}

// count[b] = sum over the half cube of w(kz) GA[a_b][i] GB[b_b][i], w = 1 on kz = 0, else 2
__global__ void __launch_bounds__(256) dot_maps_kernel(const long long* __restrict__ maps, size_t mapsz,
                                                       const int2* __restrict__ which, int Kp,
                                                       unsigned long long* __restrict__ out) {
    __shared__ unsigned long long s_part[8];
    const int2 w = which[blockIdx.x];
    const long long* A = maps + (size_t)w.x * mapsz;
    const long long* B = maps + (size_t)w.y * mapsz;
    const int nk = 2 * Kp + 1;
    unsigned long long acc = 0;
    for (size_t i = threadIdx.x; i < mapsz; i += blockDim.x) {
        const long long a = A[i];
        if (!a) continue;
        const int kz = (int)((i / nk) % (Kp + 1));
        const unsigned long long v = (unsigned long long)a * (unsigned long long)B[i];
        acc += kz == 0 ? v : 2 * v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < 8; k++) t += s_part[k];
        out[blockIdx.x] = t;
    }
}

}  // namespace ps

cudaError_t ps_prod_fields(const double* F, size_t n3, int s0, int s1, int s2, double* out, cudaStream_t st) {
    const unsigned blocks = (unsigned)std::min<size_t>((n3 + 255) / 256, 4096);
    ps::prod_fields_kernel<<<blocks, 256, 0, st>>>(F, n3, s0, s1, s2, out);
    return cudaGetLastError();
}

cudaError_t ps_round_map(const void* fhat, size_t n, double inv_n3, long long* G, int* err, cudaStream_t st) {
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
    ps::round_map_kernel<<<blocks, 256, 0, st>>>((const ps::Cx<double>*)fhat, n, inv_n3, G, err);
    return cudaGetLastError();
}

cudaError_t ps_dot_maps(const long long* maps, size_t mapsz, const int2* which, int nbins, int Kp,
                        unsigned long long* out, cudaStream_t st) {
    if (nbins <= 0) return cudaSuccess;
    ps::dot_maps_kernel<<<nbins, 256, 0, st>>>(maps, mapsz, which, Kp, out);
    return cudaGetLastError();
}
