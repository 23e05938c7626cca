// double instantiations of the field kernels (compiled separately for build parallelism).
#include "fields_impl.cuh"

using namespace ps;

cudaError_t ps_forward_f64(int n, const void* delta, int K, const void* tw_fwd, void* W, void* fhat, void* spill,
                            cudaStream_t st, int nfields) {
#define PS_CASE(NN)                                                                                             \
    case NN:                                                                                                    \
        return forward_n<double, NN>((const double*)delta, K, (const Cx<double>*)tw_fwd, (Cx<double>*)W, (Cx<double>*)fhat,  \
                                 (Cx<double>*)spill, st, nfields);
    switch (n) { PS_FOR_EACH_N(PS_CASE) }
#undef PS_CASE
    return cudaErrorInvalidValue;
}

cudaError_t ps_inverse_f64(int n, int unity, const void* fhat, const void* lines, const int* line_off, int s0, int ns,
                            int K, int x0, int nx, const void* tw_inv, void* out, size_t out_stride, void* spill,
                            void* xpre, int max_lines, int tile_ns, cudaStream_t st) {
#define PS_CASE(NN) \
    case NN:        \
        if (unity)                                                                                                 \
            return inverse_n<double, NN, true>((const Cx<double>*)fhat, (const short4*)lines, line_off, s0, ns, K, \
                                               x0, nx, (const Cx<double>*)tw_inv, (double*)out, out_stride,       \
                                               (Cx<double>*)spill, nullptr, 0, tile_ns, st);                                \
        return inverse_n<double, NN, false>((const Cx<double>*)fhat, (const short4*)lines, line_off, s0, ns, K,   \
                                            x0, nx, (const Cx<double>*)tw_inv, (double*)out, out_stride,          \
                                            (Cx<double>*)spill, (Cx<double>*)xpre, max_lines, tile_ns, st);
    switch (n) { PS_FOR_EACH_N(PS_CASE) }
#undef PS_CASE
    return cudaErrorInvalidValue;
}

size_t ps_plane_smem_f64(int n, int K, int spill) {
#define PS_CASE(NN) \
    case NN:        \
        return plane_smem_n<double, NN>(K, spill != 0);
    switch (n) { PS_FOR_EACH_N(PS_CASE) }
#undef PS_CASE
    return 0;
}
