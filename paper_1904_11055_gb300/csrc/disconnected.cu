// Disconnected (Wick-paired) part of the trispectrum estimator (n = 4).  The
// estimator of Eq. estimator keeps it; this is an optional separate output.
//
// The closed quadrilaterals that split into two zero-sum pairs, summed over the
// three pairings with the measured per-mode power |dhat(q)|^2 (real delta:
// dhat(-q) = conj dhat(q)).  A pairing (a b)(c d) needs q_b = -q_a and
// q_d = -q_c, i.e. equal shells k_a = k_b and k_c = k_d, so with the shell
// powers P(k) = sum_{q in S_k} |dhat(q)|^2:
//   S_disc_b = N^3 [d(k1,k2) d(k3,k4) P(k1) P(k3) + d(k1,k3) d(k2,k4) P(k1) P(k2)
//                   + d(k1,k4) d(k2,k3) P(k1) P(k2)],
//   B_disc_b = c_4 S_disc_b / (N^3 count_b),
// normalised like B_b (App. A).  The shell powers come from the pruned half
// spectrum of the forward transform through the shells' line tables: a mode
// with kz > 0 stands for itself and its conjugate partner (weight 2); the kz = 0
// plane is stored whole (weight 1).
#include "common.cuh"
#include "kernels.h"

namespace ps {

constexpr int kPowThreads = 256;

// P[s] for shell s = blockIdx.x (line records: ky, kz, |kx| run [a, b])
template <typename T>
__global__ void __launch_bounds__(kPowThreads) shell_power_kernel(const Cx<T>* __restrict__ fhat,
                                                                  const short4* __restrict__ lines,
                                                                  const int* __restrict__ line_off, int K,
                                                                  double* __restrict__ P) {
    __shared__ double s_part[kPowThreads / 32];
    const int s = blockIdx.x;
    const int nk = 2 * K + 1;
    double acc = 0.0;
    for (int li = line_off[s] + threadIdx.x; li < line_off[s + 1]; li += kPowThreads) {
        const short4 L = lines[li];
        const Cx<T>* Fl = fhat + ((size_t)(L.x + K) * (K + 1) + L.y) * nk + K;
        double sum = 0.0;
        for (int kx = L.z; kx <= L.w; kx++) {
            const Cx<T> v = Fl[kx];
            sum += (double)v.re * v.re + (double)v.im * v.im;
        }
        for (int kx = L.z > 0 ? L.z : 1; kx <= L.w; kx++) {
            const Cx<T> v = Fl[-kx];
            sum += (double)v.re * v.re + (double)v.im * v.im;
        }
        acc += L.y > 0 ? 2.0 * sum : sum;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kPowThreads / 32; w++) t += s_part[w];
        P[s] = t;
    }
}

__global__ void disconnected_kernel(const double* __restrict__ P, const int32_t* __restrict__ bins,
                                    const int64_t* __restrict__ counts, int64_t nbins, double norm, double n3,
                                    double* __restrict__ out) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbins; b += (int64_t)gridDim.x * blockDim.x) {
        const int32_t* k = bins + 4 * b;
        const double p1 = P[k[0] - 1], p2 = P[k[1] - 1], p3 = P[k[2] - 1];
        double sd = 0.0;
        if (k[0] == k[1] && k[2] == k[3]) sd += p1 * p3;
        if (k[0] == k[2] && k[1] == k[3]) sd += p1 * p2;
        if (k[0] == k[3] && k[1] == k[2]) sd += p1 * p2;
        const int64_t c = counts[b];
        out[b] = c > 0 ? norm * (n3 * sd) / (n3 * (double)c) : 0.0;
    }
}

}  // namespace ps

cudaError_t ps_disconnected(int is_double, const void* fhat, const void* lines, const int* line_off, int nshell, int K,
                            const int32_t* bins, const int64_t* counts, int64_t nbins, double norm, double n3,
                            double* P, double* out, cudaStream_t st) {
    if (is_double)
        ps::shell_power_kernel<double><<<nshell, ps::kPowThreads, 0, st>>>((const ps::Cx<double>*)fhat,
                                                                           (const short4*)lines, line_off, K, P);
    else
        ps::shell_power_kernel<float><<<nshell, ps::kPowThreads, 0, st>>>((const ps::Cx<float>*)fhat,
                                                                          (const short4*)lines, line_off, K, P);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    const unsigned nb = (unsigned)(nbins > 0 ? (nbins + 255) / 256 < 1024 ? (nbins + 255) / 256 : 1024 : 1);
    ps::disconnected_kernel<<<nb, 256, 0, st>>>(P, bins, counts, nbins, norm, n3, out);
    return cudaGetLastError();
}
