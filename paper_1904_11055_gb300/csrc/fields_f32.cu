// float instantiations of the field kernels (compiled separately for build parallelism).
#include "fields_impl.cuh"

using namespace ps;

cudaError_t ps_forward_f32(int n, const void* delta, int K, const void* tw_fwd, void* W, void* fhat, void* spill,
                            cudaStream_t st, int nfields) {
#define PS_CASE(NN)                                                                                             \
    case NN:                                                                                                    \
        return forward_n<float, NN>((const float*)delta, K, (const Cx<double>*)tw_fwd, (Cx<float>*)W, (Cx<float>*)fhat,  \
                                 (Cx<float>*)spill, st, nfields);
    switch (n) { PS_FOR_EACH_N(PS_CASE) }
#undef PS_CASE
    return cudaErrorInvalidValue;
}

cudaError_t ps_inverse_f32(int n, int unity, const void* fhat, const void* lines, const int* line_off, int s0, int ns,
                            int K, int x0, int nx, const void* tw_inv, void* out, size_t out_stride, void* spill,
                            void* xpre, int max_lines, int tile_ns, cudaStream_t st) {
#define PS_CASE(NN) \
    case NN:        \
        if (unity) return cudaErrorInvalidValue;                                                                   \
        return inverse_n<float, NN, false>((const Cx<float>*)fhat, (const short4*)lines, line_off, s0, ns, K, x0,  \
                                           nx, (const Cx<double>*)tw_inv, (float*)out, out_stride,                  \
                                           (Cx<float>*)spill, (Cx<float>*)xpre, max_lines, tile_ns, st);
    switch (n) { PS_FOR_EACH_N(PS_CASE) }
#undef PS_CASE
    return cudaErrorInvalidValue;
}

cudaError_t ps_inverse_ranged_f32(int n, const void* fhat, const void* lines, const int* line_off, int s0, int ns, int K,
                                  const void* tw_inv, void* out, size_t out_stride, void* xpre, int max_lines,
                                  int tile_ns, const int* kz_host, const int* kz_dev, cudaStream_t st) {
#define PS_CASE(NN) \
    case NN:        \
        return inverse_ranged_n<float, NN>((const Cx<float>*)fhat, (const short4*)lines, line_off, s0, ns, K,      \
                                           (const Cx<double>*)tw_inv, (float*)out, out_stride, (Cx<float>*)xpre,    \
                                           max_lines, tile_ns, kz_host, kz_dev, st);
    switch (n) { PS_FOR_EACH_N(PS_CASE) }
#undef PS_CASE
    return cudaErrorInvalidValue;
}

size_t ps_plane_smem_f32(int n, int K, int spill) {
#define PS_CASE(NN) \
    case NN:        \
        return plane_smem_n<float, NN>(K, spill != 0);
    switch (n) { PS_FOR_EACH_N(PS_CASE) }
#undef PS_CASE
    return 0;
}
