/*
 * polyspec_diag.h -- diagnostic entry points of the polyspectrum library.
 *
 * These exist to check, on the GPU, the hardware layouts the tensor-core
 * contraction relies on; they are not part of the estimator.  The paper has no
 * counterpart: they test this implementation, not the method.
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
 * The plan's shell fields of delta_x (device, N^3 real of the plan's type):
 * runs the forward transform and the shell-field stage exactly as
 * poly_estimate does, synchronises `stream`, and copies the fields to
 * fields_host (host, nfield x N^3 of the plan's real type, natural layout
 * [slot][x][y][z]; nfield = nshell, or 2 nshell for a multipole plan, the
 * Legendre-weighted fields after the plain ones).  `plan` is a poly_plan.
 * Returns a poly_status.
 */
int poly_diag_fields(void* plan, const void* delta_x, void* fields_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* POLYSPEC_DIAG_H */
