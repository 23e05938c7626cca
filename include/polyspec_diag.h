/*
 * polyspec_diag.h -- diagnostic entry points of the polyspectrum library.
 *
 * These exist to check this implementation, not the method, and are not part of
 * the estimator (the paper has no counterpart): on the GPU, the hardware
 * layouts the tensor-core contraction relies on, the limit of its device waits
 * and the shell fields it computes; with no device, the host tables that plan
 * creation builds (bins, shell lines, contraction tiles, adjoint entries, the
 * cells the counts are summed over).
 */
#ifndef POLYSPEC_DIAG_H
#define POLYSPEC_DIAG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * One-block tcgen05 GEMM on the current device, built exactly like the
 * contraction's MMA step: D[128][N] = sum_{k<32} A[m][k] * B[n][k] with A
 * (host, 128 x 32 bf16 bit patterns, row-major) placed in tensor memory by
 * tcgen05.st, B (host, N x 32 bf16 bit patterns, row-major) placed in shared
 * memory in the K-major core-matrix layout, FP32 accumulation.  N in
 * {16, 32, ..., 256}.  D (host, 128 x N float, row-major) receives the result.
 * Returns 0 on success, 1 for a bad N, 3 allocation failure, 4 CUDA error,
 * 5 a bounded wait gave up.  Synchronises the device.
 */
int poly_diag_tc_gemm(const uint16_t* A_host, const uint16_t* B_host, int N, float* D_host);

/*
 * A stalled producer, simulated: one warp waits on a shared-memory barrier
 * that nothing arrives on, through the same bounded wait the pipelines use
 * (a clock64 budget of about 2 s).  The wait gives up, the kernel sets the
 * error word and returns, and the host reports what the pipelines report for
 * it.  Returns 5 (POLY_ERR_TIMEOUT) when the wait gave up as designed, 0 if
 * it completed (which would be a defect), 4 on a CUDA error.  ms_out
 * (nullable) receives the kernel's duration.  Synchronises the device.
 */
int poly_diag_stalled_wait(double* ms_out);

/*
 * Peak FMA rate of the CUDA cores of the current device, measured: every
 * thread of 16 blocks of 256 threads per SM runs 8 independent FMA chains
 * (FP32, or FP64 when is_double) for `iters` steps; the kernel is timed with
 * CUDA events after one untimed launch.  tflops_out receives
 * 2 x threads x 8 x iters / time in TFLOP/s; ms_out (nullable) the kernel's
 * duration.  iters in [1, 2^24].  Returns 0, 1 for bad arguments, 4 on a CUDA
 * error.  Synchronises the device.
 */
int poly_diag_fma_peak(int is_double, int iters, double* tflops_out, double* ms_out);

/*
 * The plan's shell fields of delta_x (device, N^3 real of the plan's type):
 * runs the forward transform and the shell-field stage exactly as
 * poly_estimate does, synchronises `stream`, and copies the fields to
 * fields_host (host, nfield x N^3 of the plan's real type, natural layout
 * [slot][x][y][z]; nfield = nshell, or 2 nshell for a multipole plan, the
 * Legendre-weighted fields after the plain ones).  `plan` is a poly_plan.
 * Returns a poly_status.
 */
int poly_diag_fields(void* plan, const void* delta_x, void* fields_host, void* stream);

/*
 * The host tables a plan builds, computed on the host alone (no device call):
 * the bins (Sec. 4.2 ordering, App. B polygon rule unless POLY_BINS_ALL_SORTED),
 * the shell line tables of the pruned inverse transforms and the CUDA-core
 * contraction tiles.  Arguments N, order, edges (nshell + 1 values), flags and
 * ell are those of poly_plan_create_multipole and are checked the same way
 * (precision taken as FP64); the tiles are the final ones, so for ell > 0 the
 * first leg reads the weighted slot k_1 - 1 + nshell.
 *   sizes[7] (required) receives the element counts: bins (tuples), tiles,
 *   field ids, row factor records, column factor records, lines, line offsets.
 *   Each other pointer may be NULL (not written) or a caller-owned host buffer:
 *   bins      int32 [nbins][order], 1-based shells;
 *   tiles     int32 [ntiles][8]: row_off, nrow, col_off, ncol, field_off, nfield,
 *             region_mask (bit (r / 32) * 4 + c / 16), padding;
 *   field_ids int32, 0-based field slots, tile t's at field_off .. + nfield;
 *   rowf/colf int16 [][4]: up to three tile-local field indices (-1: none),
 *             row r of tile t at rowf[row_off + r], column c at colf[col_off + c];
 *   slot      int64 [nbins]: t * 4096 + r * 64 + c, the product that is bin b;
 *   lines     int16 [nlines][4]: ky, kz >= 0, a, b: shell s's modes on the line
 *             (ky, kz) are those with a <= |kx| <= b; lines line_off[s] ..
 *             line_off[s + 1] - 1, and slot nshell holds the union of all shells.
 * Returns a poly_status.
 */
/*
 * The cells and weights the exact counts are summed over (count_b = N^-3 sum_x
 * prod iota, App. A): the counting fields are invariant under the cube's 48
 * symmetries, so the sum runs over 0 <= x <= y <= z <= N/2 with each cell
 * weighted by the size of its orbit.  N even.  ncell (required) receives the
 * number of cells; cells (int32, linear index (x N + y) N + z) and weights
 * (double) are NULL or host buffers of that length.  Returns a poly_status.
 */
int poly_diag_count_wedge(int N, int64_t* ncell, int32_t* cells, double* weights);

/*
 * poly_plan_bin_wraps computed on the host alone for the plan that N, order,
 * edges (nshell + 1), nshell and flags would give: nbins (required) receives
 * the bin count, wraps (NULL or host, nbins uint8) the flags.  Returns a
 * poly_status.
 */
int poly_diag_bin_wraps(int N, int order, const double* edges, int nshell, unsigned flags, int64_t* nbins,
                        uint8_t* wraps);

int poly_diag_host_tables(int N, int order, const double* edges, int nshell, unsigned flags, int ell,
                          int64_t* sizes, int32_t* bins, int32_t* tiles, int32_t* field_ids, int16_t* rowf,
                          int16_t* colf, int64_t* slot, int16_t* lines, int32_t* line_off);

/*
 * The tensor-core contraction's host tables for a split-BF16 plan, computed on
 * the host alone: which products of fields (rows: the first legs, as a pair for
 * n >= 3; columns: the remaining legs) each block accumulates where, and where
 * the reduction finds each bin.  N, order (2..6), edges, nshell and flags as in
 * poly_plan_create, ell as in poly_plan_create_multipole (for ell > 0 the rows'
 * first factor is the weighted field slot k1 - 1 + nshell, and the groups are
 * held to fewer accumulator columns: the chunk stages 2 nshell field rows);
 * sms (the device's SM count), max_mt (M tiles per group) and
 * cta_mult (the block budget is sms x cta_mult / 2) as poly_plan_set_config
 * and the device would set them.
 *   sizes[9] (required) receives the counts: bins, blocks, groups, M tiles,
 *   runs, row factor records, column factor records, then the launch's
 *   producer teams (2 or 3) and its A/B slot cap (what shared memory holds;
 *   a group's slots are also bounded by tensor memory: (512 - its
 *   accumulator columns rounded up to 32) / (32 x its M tiles)).  Other pointers may be
 *   NULL or caller-owned host buffers:
 *   ctas   int64 [nblocks][3]: group, first chunk, end chunk (chunks of 32 cells);
 *   groups int32 [ngroups][5]: first M tile, M tiles, first column record,
 *          columns (a multiple of 16), accumulator columns;
 *   mtiles int32 [][3]: first row record (128 rows), first run, runs;
 *   runs   int32 [][4]: first local column n0, columns nn, first accumulator
 *          column acc, M tile within the group: accumulator column acc + j of
 *          that M tile's row r is the product of row r and column n0 + j;
 *   rowf, colf int16 [][3]: 0-based field slots (-1: none);
 *   binmap int32 [nbins][3]: first block, blocks, slot = accumulator column x
 *          128 + row; bin b is the sum of that slot over those blocks.
 * Returns a poly_status.
 */
int poly_diag_tc_tables(int N, int order, const double* edges, int nshell, unsigned flags, int ell, int sms,
                        int max_mt, int cta_mult, int64_t* sizes, int64_t* ctas, int32_t* groups, int32_t* mtiles,
                        int32_t* runs, int16_t* rowf, int16_t* colf, int32_t* binmap);

/*
 * The adjoint's host tables (poly_backward), computed on the host alone.  The
 * gradient of B_b with respect to the field D_m at a cell is the sum, over the
 * positions of m in b, of the product of b's other fields there (Eq. estimator
 * differentiated); the adjoint gathers these by entry: (m, the other shells
 * sorted), each listing the bins that produce it.  N, order (2..4), edges,
 * nshell, flags and prec as in poly_plan_create; sms as the device would set it.
 *   sizes[10] (required): entries, entry-bin records, then for the tensor-core
 *   form (order 3, split-BF16; 0 groups when it does not apply): groups, chunks,
 *   K (shells padded to 32), accumulator columns per buffer, bytes of one B
 *   array, cell ranges per pair of groups, shells without entries, largest
 *   chunk count of a group.  Other pointers may be NULL or host buffers:
 *   moff   int32 [nshell + 1]: entries of shell m are moff[m] .. moff[m+1]-1;
 *   ent    int16 [nent][3]: the other shells, 0-based, ascending (-1: none);
 *   eoff   int32 [nent + 1], ebins int32: entry e's bins at ebins[eoff[e] ..
 *          eoff[e+1]-1], a bin once per position of m in it;
 *   at_groups int32 [][6]: first chunk, chunks, first chunk of the second
 *          half, B byte offset, K-block masks of the two column runs;
 *   at_chunks int32: j block | m << 8 | (last chunk of m) << 16;
 *   at_pos int32 [nent]: byte offset of entry e's weight in the B arrays
 *          (column = chunk x 16 + j % 16 of its group, row = first other shell).
 * Returns a poly_status.
 */
int poly_diag_adj_tables(int N, int order, const double* edges, int nshell, unsigned flags, int prec, int sms,
                         int64_t* sizes, int32_t* moff, int16_t* ent, int32_t* eoff, int32_t* ebins,
                         int32_t* at_groups, int32_t* at_chunks, int32_t* at_pos);

#ifdef __cplusplus
}
#endif

#endif /* POLYSPEC_DIAG_H */
