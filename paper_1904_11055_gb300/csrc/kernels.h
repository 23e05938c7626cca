// Internal launch interface between the plan code and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

// ---- fields.cu --------------------------------------------------------------
int ps_supported_n(int n);
int ps_plane_needs_spill(int n, int K, int is_double);
size_t ps_spill_elems(int n, int K, int nblocks, int is_double);
// delta [N^3] real -> W [N][(2K+1)(K+1)] -> fhat [(2K+1)(K+1)][2K+1] (complex, same precision)
cudaError_t ps_forward(int n, int is_double, const void* delta, int K, const void* tw_fwd, void* W, void* fhat,
                       void* spill, cudaStream_t st);
// the same for nfields fields N^3 apart in one launch pair: W and fhat hold one output per field, N (2K+1)(K+1)
// and (2K+1)(K+1)(2K+1) complex values apart; spill (when needed) nfields * N blocks
cudaError_t ps_forward_batched(int n, int is_double, const void* delta, int nfields, int K, const void* tw_fwd, void* W,
                               void* fhat, void* spill, cudaStream_t st);
// shells s0..s0+ns-1, planes x0..x0+nx-1 -> out[(s-s0)*out_stride + (x-x0)*N*N + y*N + z].
// xpre != NULL (and not unity): first run the x pass into xpre (sum over shells of lines * N complex values;
// max_lines = the largest line count of the shells), then scatter; otherwise gather along x in the plane kernel.
// tile_ns > 0: write the cell-tiled layout out[(cell/32) * tile_ns * 32 + s * 32 + cell % 32] (absolute shell s,
// x0 must be 0) instead of the natural one.
cudaError_t ps_inverse(int n, int is_double, int unity, const void* fhat, const void* lines, const int* line_off,
                       int s0, int ns, int K, int x0, int nx, const void* tw_inv, void* out, size_t out_stride,
                       void* spill, void* xpre, int max_lines, int tile_ns, cudaStream_t st);
// The FP32 estimate-path inverse in runs of shells sized by each shell's largest
// kz (kz_host: host array indexed by shell; kz_dev: the same on the device, or
// NULL); see inverse_ranged_n.
cudaError_t ps_inverse_ranged_f32(int n, const void* fhat, const void* lines, const int* line_off, int s0, int ns, int K,
                                  const void* tw_inv, void* out, size_t out_stride, void* xpre, int max_lines,
                                  int tile_ns, const int* kz_host, const int* kz_dev, cudaStream_t st);

// ---- contract_cc.cu -----------------------------------------------------------
// One GEMM tile of the CUDA-core contraction: up to 64 rows x 64 cols, each row
// (col) the product of one or two of the tile's local fields.
struct PsTile {
    int row_off, nrow, col_off, ncol, field_off, nfield;
    unsigned region_mask;  // bit w: warp w's 32x16 region holds at least one needed entry
    int pad_;
};
constexpr int kCcTM = 64, kCcTN = 64, kCcMaxFields = 128;
// cells per chunk of the CUDA-core contraction
inline int ps_cc_chunk(int is_double) { return is_double ? 16 : 32; }

// partial[(split * ntiles + tile) * 64 * 64 + r * 64 + c] = sum over the split's cells
// fields: natural [s][cell] with stride field_stride (tile_ns == 0) or cell-tiled over tile_ns shells
// nf: factors per row or column at most (2 for n <= 4, 3 for n = 5, 6)
cudaError_t ps_contract_cc(int is_double, int weighted, int absval, int nf, const void* fields, size_t field_stride,
                           int tile_ns, int64_t ncell, const void* weight, const PsTile* tiles, int ntiles, const int* field_ids,
                           const short4* rowf, const short4* colf, int nsplit, int64_t chunks_per_split,
                           double* partial, cudaStream_t st);
// S[b] = sum_split partial[split * slot_stride + slot[b]]
cudaError_t ps_reduce_slots(const double* partial, int nsplit, int64_t slot_stride, const int64_t* slot,
                            int64_t nbins, double* S, cudaStream_t st);
// out[b] = norm * S[b] / (N^3 count[b])  (0 where count == 0)
// disconnected part of the trispectrum: shell powers P (device, nshell) from the pruned spectrum, then B_disc per bin
cudaError_t ps_disconnected(int is_double, const void* fhat, const void* lines, const int* line_off, int nshell, int K,
                            const int32_t* bins, const int64_t* counts, int64_t nbins, double norm, double n3,
                            double* P, double* out, cudaStream_t st);
// out = L_ell(kz/|q|) * fhat over the pruned half spectrum (even ell; the mode q = 0 gets weight 0)
cudaError_t ps_legendre_weight(int is_double, const void* fhat, int K, int ell, void* out, cudaStream_t st);
cudaError_t ps_normalise(const double* S, const int64_t* counts, int64_t nbins, double norm, double n3, double* out,
                         cudaStream_t st);

// ---- misc.cu -------------------------------------------------------------------
// out[s * out_stride + w] = in[s * in_stride + idx[w]] for s < ns, w < nw
// ---- counts_exact.cu ---------------------------------------------------------
// out = F[s0] F[s1] F[s2] (slots -1: none), FP64 fields of n3 cells in natural layout
cudaError_t ps_prod_fields(const double* F, size_t n3, int s0, int s1, int s2, double* out, cudaStream_t st);
// G[i] = round(Re fhat[i] * inv_n3) for n complex FP64 values; *err = 1 if any is not near an integer
cudaError_t ps_round_map(const void* fhat, size_t n, double inv_n3, long long* G, int* err, cudaStream_t st);
// out[b] = sum over the half cube |p_c| <= Kp of w(kz) maps[which[b].x][i] maps[which[b].y][i]
cudaError_t ps_dot_maps(const long long* maps, size_t mapsz, const int2* which, int nbins, int Kp,
                        unsigned long long* out, cudaStream_t st);

cudaError_t ps_gather_cells(int is_double, const void* in, size_t in_stride, int ns, const int32_t* idx, int64_t nw,
                            void* out, size_t out_stride, cudaStream_t st);
