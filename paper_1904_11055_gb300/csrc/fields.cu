// Type dispatch of the field kernels (FP32 and FP64 instantiations live in
// fields_f32.cu / fields_f64.cu; the kernels themselves in fields_impl.cuh).
#include "common.cuh"
#include "kernels.h"

cudaError_t ps_forward_f32(int n, const void* delta, int K, const void* tw_fwd, void* W, void* fhat, void* spill,
                           cudaStream_t st, int nfields);
cudaError_t ps_forward_f64(int n, const void* delta, int K, const void* tw_fwd, void* W, void* fhat, void* spill,
                           cudaStream_t st, int nfields);
cudaError_t ps_inverse_f32(int n, int unity, const void* fhat, const void* lines, const int* line_off, int s0, int ns,
                           int K, int x0, int nx, const void* tw_inv, void* out, size_t out_stride, void* spill,
                           void* xpre, int max_lines, int tile_ns, cudaStream_t st);
cudaError_t ps_inverse_f64(int n, int unity, const void* fhat, const void* lines, const int* line_off, int s0, int ns,
                           int K, int x0, int nx, const void* tw_inv, void* out, size_t out_stride, void* spill,
                           void* xpre, int max_lines, int tile_ns, cudaStream_t st);
size_t ps_plane_smem_f32(int n, int K, int spill);
size_t ps_plane_smem_f64(int n, int K, int spill);

static const size_t kMaxPlaneSmem = 227 * 1024;

size_t ps_spill_elems(int n, int K, int nblocks, int is_double) {
    // per block (K+1) lines of ls complex elements, only needed when smem does not fit
    size_t ls = is_double ? ps::line_stride<double>(n) : ps::line_stride<float>(n);
    return (size_t)nblocks * (K + 1) * ls;
}

int ps_plane_needs_spill(int n, int K, int is_double) {
    if (!ps_supported_n(n)) return -1;
    const size_t b = is_double ? ps_plane_smem_f64(n, K, 0) : ps_plane_smem_f32(n, K, 0);
    return b > kMaxPlaneSmem ? 1 : 0;
}

int ps_supported_n(int n) {
#define PS_CASE(NN) \
    case NN:        \
        return 1;
    switch (n) { PS_FOR_EACH_N(PS_CASE) }
#undef PS_CASE
    return 0;
}

cudaError_t ps_forward(int n, int is_double, const void* delta, int K, const void* tw_fwd, void* W, void* fhat,
                       void* spill, cudaStream_t st) {
    return ps_forward_batched(n, is_double, delta, 1, K, tw_fwd, W, fhat, spill, st);
}

cudaError_t ps_forward_batched(int n, int is_double, const void* delta, int nfields, int K, const void* tw_fwd, void* W,
                               void* fhat, void* spill, cudaStream_t st) {
    if (nfields < 1 || nfields > 65535) return cudaErrorInvalidValue;
    return is_double ? ps_forward_f64(n, delta, K, tw_fwd, W, fhat, spill, st, nfields)
                     : ps_forward_f32(n, delta, K, tw_fwd, W, fhat, spill, st, nfields);
}

cudaError_t ps_inverse(int n, int is_double, int unity, const void* fhat, const void* lines, const int* line_off, int s0,
                       int ns, int K, int x0, int nx, const void* tw_inv, void* out, size_t out_stride, void* spill,
                       void* xpre, int max_lines, int tile_ns, cudaStream_t st) {
    return is_double ? ps_inverse_f64(n, unity, fhat, lines, line_off, s0, ns, K, x0, nx, tw_inv, out, out_stride,
                                      spill, xpre, max_lines, tile_ns, st)
                     : ps_inverse_f32(n, unity, fhat, lines, line_off, s0, ns, K, x0, nx, tw_inv, out, out_stride,
                                      spill, xpre, max_lines, tile_ns, st);
}
