/*
 * polyspec.h -- C ABI of the GB300 (sm_103a) polyspectrum library.
 *
 * The library computes the FFT-based (Scoccimarro-type) angle-averaged
 * polyspectrum estimator of Tomlinson, Jeong & Kim, arXiv:1904.11055:
 *
 *   B_b = (V^{n-1} / N^{3n}) * S_b / (N^3 count_b),                      (App. A)
 *   S_b = sum_x prod_{t=1..n} D_{k_t}(x),                                (Eq. estimator)
 *   D_k(x) = sum_{q in shell k} dhat(q) e^{+2 pi i q.x / N},             (Eq. Bkfast; App. A)
 *   count_b = N^{-3} sum_x prod_t iota_{k_t}(x),                         (Eqs. volume, Vn, Ncalc)
 *   iota_k(x) = sum_{q in shell k} e^{+2 pi i q.x / N},
 *
 * for one real N^3 field delta(x) in a periodic box of side L (V = L^3),
 * dhat(q) = sum_x delta(x) e^{-2 pi i q.x / N} (the unnormalised FFTW
 * convention of App. A), integer wavevectors q in units of k_F = 2 pi / L,
 * shell k = {q != 0 : edges[k-1]^2 <= |q|^2 < edges[k]^2} (the half-width
 * binning |q - k_i| < dk/2 of Sec. 2 written with explicit edges), and bins
 * b = (k_1 >= k_2 >= ... >= k_n) in the row-major order of Sec. 4.2 (k_n
 * fastest) that satisfy the polygon inequality k_1 <= k_2 + ... + k_n on the
 * shell centres (App. B, Eq. polygon).  count_b is the exact number of closed
 * n-gons of grid modes (an integer, returned bit-exact).
 *
 * Conventions of every entry point:
 *  - Arrays are plain pointers.  "device" means memory of the plan's CUDA
 *    device; "host" means ordinary (pageable or pinned) host memory.
 *  - Real grids are C order [x][y][z], z fastest, N^3 elements.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *    calls are stream-ordered and asynchronous unless stated otherwise.
 *  - The caller owns every buffer it passes; the plan owns its workspace and
 *    its cached counts.  Output buffers must not alias inputs.
 *  - Argument errors return synchronously and leave outputs untouched.
 *    Errors raised on the device surface as POLY_ERR_CUDA / POLY_ERR_TIMEOUT
 *    from poly_plan_sync() or the next call on the plan.
 *  - No exception or longjmp crosses this boundary.  A plan is not
 *    thread-safe: serialise calls on one plan.
 */
#ifndef POLYSPEC_H
#define POLYSPEC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct poly_plan_s* poly_plan;

typedef enum {
    POLY_OK = 0,
    POLY_ERR_ARG = 1,         /* bad argument (NULL, sizes, unsorted edges, bad order, ...) */
    POLY_ERR_ALIAS = 2,       /* n * K >= N: closures wrap around the periodic grid (Sec. 4.3) */
    POLY_ERR_ALLOC = 3,       /* device or host allocation failed */
    POLY_ERR_CUDA = 4,        /* a CUDA runtime call or kernel failed */
    POLY_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (see poly_plan_sync) */
    POLY_ERR_UNSUPPORTED = 6, /* valid request outside what the library implements */
    POLY_ERR_COUNT = 7        /* a polygon count came out non-integral (numerical failure) */
} poly_status;

typedef enum {
    POLY_FP32 = 0,       /* FP32 input and fields; FP32 CUDA-core products, FP64 reduction */
    POLY_SPLIT_BF16 = 1, /* FP32 input and fields; split-BF16 (hi+lo, 3 products) tcgen05 contraction */
    POLY_TF32X3 = 2,     /* reserved; returns POLY_ERR_UNSUPPORTED */
    POLY_FP64 = 3        /* FP64 input, fields and contraction (the plain method) */
} poly_precision;

/* plan flags */
#define POLY_BINS_ALL_SORTED 0x1u /* every sorted tuple instead of the polygon-inequality set */
#define POLY_ALLOW_ALIAS 0x2u     /* accept n*K >= N; the periodic (mod N) estimator is returned */

/*
 * Create a plan for grid size N (one of 16, 24, 32, 48, 64, 96, 128, 160, 256),
 * box side L > 0, order n in [2, 6] (split-BF16 plans run the tensor-core
 * contraction with rows of one to three fields against columns of one to
 * three; FP32 and FP64 plans the CUDA-core one), `nshell` shells with `nshell + 1`
 * strictly increasing edges (host array, units of k_F, edges[0] >= 0).
 * K = the largest integer with K^2 < edges[nshell]^2 must satisfy 2K+1 <= N,
 * and n*K < N unless POLY_ALLOW_ALIAS.  The sorted shell tuples the bins are
 * drawn from, C(nshell + n - 1, n) of them, may number at most 2^26
 * (POLY_ERR_UNSUPPORTED above; e.g. n = 5 with 120 shells).  Argument checks
 * and the host tables come before any device call.  Plan creation enumerates the bins,
 * builds the shell tables and tiles, allocates the workspace (nshell * N^3
 * fields of the plan's precision plus small buffers) on the current CUDA
 * device and computes the exact counts (FP64 counting fields on the
 * 1/48 symmetry wedge, cached per (N, edges, n, flags) in the process).  Where
 * those FP64 sums can no longer be rounded safely (large n = 5, 6 plans) the
 * counts come from integer closure maps instead (the product of the first
 * max(1, n - 3) legs' counting fields and of the rest, each transformed and
 * rounded to its integer map, then summed in 64-bit integers); plans with
 * POLY_ALLOW_ALIAS cannot take that route and return POLY_ERR_COUNT there.
 * It synchronises the device.  On failure *out is set to NULL.
 */
poly_status poly_plan_create(poly_plan* out, int N, double L, int order, int nshell, const double* edges,
                             poly_precision prec, unsigned flags);

/*
 * Number of bins the plan outputs (*nbins, host): the sorted shell tuples
 * b = (k_1 >= ... >= k_n) of Sec. 4.2 that satisfy the polygon inequality on
 * the shell centres (App. B, Eq. polygon), or every sorted tuple with
 * POLY_BINS_ALL_SORTED.  Host only; POLY_ERR_ARG for a NULL argument.
 */
poly_status poly_plan_nbins(poly_plan plan, int64_t* nbins);

/*
 * Redshift-space multipoles (the extension Sec. 5 points to): the same as
 * poly_plan_create, but the first leg k1 of every bin carries the Legendre
 * weight L_ell(q_z/|q|) (plane-parallel line of sight along the grid's z
 * axis), and poly_estimate returns
 *   B^ell_b = (2 ell + 1) c_n sum_x D^ell_{k1}(x) prod_{t>1} D_{kt}(x) / (N^3 count_b),
 *   D^ell_k(x) = sum_{q in S_k} L_ell(q_z/|q|) dhat(q) e^{+2 pi i q.x/N}.
 * ell even in [0, 8] (POLY_ERR_ARG otherwise; odd multipoles of a real field
 * are not real); ell = 0 is poly_plan_create.  All three precisions; a
 * split-BF16 plan runs the tensor-core contraction with the weighted fields as
 * its rows' first factor (orders 2 to 4, as for monopole plans; 64 unit shells
 * fit, the chunk stages 2 * nshell field rows, and a shell count whose stages
 * leave no shared memory for accumulators is POLY_ERR_UNSUPPORTED).  The plan
 * holds 2 * nshell fields;
 * counts are the plain polygon counts.  poly_backward and
 * poly_trispectrum_disconnected return POLY_ERR_UNSUPPORTED for ell > 0.
 */
poly_status poly_plan_create_multipole(poly_plan* out, int N, double L, int order, int nshell, const double* edges,
                                       poly_precision prec, unsigned flags, int ell);

/*
 * The bins (Sec. 4.2 order: row-major over k_1 >= k_2 >= ... >= k_n, k_n
 * fastest) as 1-based shell numbers: idx, host, caller-owned, nbins * order
 * int32, bin b at idx[b * order ..].  Host only; POLY_ERR_ARG for NULL.
 */
poly_status poly_plan_bins(poly_plan plan, int32_t* idx);

/*
 * Exact polygon counts count_b = N^{-3} sum_x prod_t iota_{k_t}(x) (Eqs. Vn,
 * Ncalc; the number of closed n-gons of grid modes), computed at plan creation:
 * counts, host, caller-owned, nbins int64, in poly_plan_bins order.  Host only;
 * POLY_ERR_ARG for NULL.
 */
poly_status poly_plan_counts(poly_plan plan, int64_t* counts);

/*
 * Which bins may hold closures that wrap around the grid (the aliasing the
 * paper avoids by asking N > n N_max, Sec. 4.3): wraps (host, nbins uint8)
 * receives 1 where sum_t K_{k_t} >= N, K_k being the largest component |q_c|
 * of a mode of shell k, else 0.  A bin marked 0 counts and sums exact closures
 * q_1 + ... + q_n = 0 only; a bin marked 1 may also hold closures that sum to a
 * nonzero multiple of N (the periodic estimator the FFT computes).  Without
 * POLY_ALLOW_ALIAS every bin is 0.  Host only.
 */
poly_status poly_plan_bin_wraps(poly_plan plan, uint8_t* wraps);

/*
 * Device memory the plan holds now, in bytes (*bytes, host).  Sec. 1 sizes the
 * method's memory as N_max fields of (n N_max)^3 cells, growing like
 * n^3 N_max^4; here that is the workspace
 * (nfield x N^3 shell fields of the plan's real type, about 4.3 GB at 256^3
 * with 64 FP32 fields, plus the transform buffers, tables and partial sums),
 * and the adjoint's buffers once poly_backward has run (another nshell x N^3
 * fields).  Plan creation's transient count buffers are freed before it
 * returns and are not included.  Host only.
 */
poly_status poly_plan_device_bytes(poly_plan plan, int64_t* bytes);

/*
 * Estimate B_b for one field: the forward transform of delta_x, the shell
 * fields D_k (Eq. Bkfast), the product sums S_b (Eq. estimator) and the
 * normalisation by the plan's counts (App. A, final discrete form).
 * delta_x: device, N^3 real (float for POLY_FP32 /
 * POLY_SPLIT_BF16, double for POLY_FP64).  out: device, nbins double, B_b.
 * scale_or_null: device, nbins double or NULL; if given, receives
 * sum_x |prod_t D_{k_t}(x)| / (N^3 count_b) (the scale of the stated error
 * bound), at the cost of a second contraction.  Asynchronous on `stream`.  Both
 * buffers are caller-owned and must not alias delta_x or each other
 * (POLY_ERR_ARG); kernel faults and bounded-wait timeouts of the contraction
 * surface from poly_plan_sync or the next call on the plan.
 */
poly_status poly_estimate(poly_plan plan, const void* delta_x, double* out, double* scale_or_null, void* stream);

/*
 * Disconnected (Gaussian, Wick-paired) part of the trispectrum estimate of
 * delta_x, for order-4 plans (POLY_ERR_UNSUPPORTED otherwise).  The paper's
 * estimator keeps it; subtract it from poly_estimate's B_b for the connected
 * part.  Per bin b = (k1 >= k2 >= k3 >= k4), the closed quadrilaterals that
 * split into two zero-sum pairs, summed over the three pairings with the
 * measured mode power: with P(k) = sum_{q in S_k} |dhat(q)|^2,
 *   B_disc_b = c_4 N^3 [d(k1,k2)d(k3,k4) P(k1)P(k3) + d(k1,k3)d(k2,k4) P(k1)P(k2)
 *                       + d(k1,k4)d(k2,k3) P(k1)P(k2)] / (N^3 count_b),
 * c_4 = V^3/N^12 as for B_b; zero for bins without two equal pairs.
 * delta_x: device, N^3 real of the plan's input type.  out: device, nbins
 * double.  shell_power_or_null: device, nshell double (P(k)), or NULL.
 * Uses the plan's spectrum workspace (stream-ordered with poly_estimate);
 * the first call allocates two small device tables.  Asynchronous on `stream`.
 */
poly_status poly_trispectrum_disconnected(poly_plan plan, const void* delta_x, double* out, double* shell_power_or_null,
                                          void* stream);

/*
 * Full-shape trispectrum of one shell quadruple (Eq. Tkfull, Sec. 2.1; the
 * paper leaves it as future work): the closed quadrilaterals
 * q1 + q2 + q3 + q4 = 0 (mod N), q_t in S_{k_t}, split by their diagonals
 * p1 = q1 - q2 and p2 = q1 - q3 into bins j: dedges[j]^2 <= |p|^2 <
 * dedges[j+1]^2 (components of p: differences of the signed representatives
 * -N/2 .. N/2-1; p = 0 falls in bin 0 when dedges[0] = 0):
 *   T[j1 * ndiag + j2] = c_4 sum Re prod_t dhat(q_t) / count[j1][j2]
 * (0 where the count is 0), c_4 = V^3/N^12 as for B_b.  Summed over diagonal
 * bins that cover every |p|, c_4^{-1} T * count and count give the
 * angle-averaged trispectrum's sums and counts of that bin.
 * Any plan (any order, precision and multipole) serves: its shells, grid and
 * forward transform are used.  delta_x: device, N^3 real of the plan's input
 * type, or NULL for counts only (then T_out and scale_or_null must be NULL).
 * k: host, 4 shell numbers, 1-based, in [1, nshell], any order.  ndiag in
 * [1, 128]; dedges: host, ndiag + 1 finite, non-negative, strictly increasing.
 * T_out, counts_out (int64), scale_or_null: device, ndiag^2 each, or NULL (at
 * least one given; none may alias another or delta_x).  scale_or_null
 * receives c_4 sum prod_t |dhat(q_t)| / count (the scale of the rounding error
 * of T).  Products and per-bin partial sums are in the plan's precision
 * (FP32 for FP32 and split-BF16 plans), accumulation in FP64; counts are
 * exact.  Work grows as |S_k1| |S_k2| |S_k3|: more than 4.4e12 triples is
 * POLY_ERR_UNSUPPORTED.  Grows a per-plan scratch buffer on demand (freed
 * with the plan) and overwrites the plan's spectrum workspace
 * (stream-ordered with poly_estimate).  Asynchronous on `stream`.
 */
poly_status poly_trispectrum_full(poly_plan plan, const void* delta_x, const int32_t* k, int ndiag, const double* dedges,
                                  double* T_out, int64_t* counts_out, double* scale_or_null, void* stream);

/*
 * The same as poly_estimate (Eq. estimator, App. A) with HOST buffers: copies
 * delta_x (host, N^3 real of the plan's input type, caller-owned; pinned
 * memory makes the copy asynchronous to other host work) into the plan's
 * workspace, estimates, copies B_b to out (host, nbins double, caller-owned)
 * and synchronises `stream` before returning, so device errors are reported
 * by this call.
 */
poly_status poly_estimate_host(poly_plan plan, const void* delta_x_host, double* out_host, void* stream);

/*
 * Gradient of L = sum_b dL_dB[b] * B_b with respect to delta(x) (no
 * counterpart in the paper: the adjoint of Eq. estimator and Eq. Bkfast,
 * dL/ddelta = sum_q mask_{m(q)} Ghat_{m(q)}(q) e^{+2 pi i q.x/N} with
 * G_m = dL/dD_m).
 * dL_dB: device, nbins double.  dL_ddelta: device, N^3 real of the plan's
 * input type, overwritten.  Recomputes the shell fields from delta_x (it
 * never stores pair products), contracts dL/dB with products of the other
 * fields, transforms each result forward, keeps its own shell and applies one
 * inverse transform (the adjoint of the estimator).  Asynchronous on `stream`.
 * Orders 2 to 4 (POLY_ERR_UNSUPPORTED above).
 */
poly_status poly_backward(poly_plan plan, const void* delta_x, const double* dL_dB, void* dL_ddelta, void* stream);

/*
 * Estimate `count` fields (Eq. estimator for each; the batching has no
 * counterpart in the paper), possibly of different plans (e.g. mock catalogues
 * on different grid sizes), in one stream-ordered batch: fields[i] is a device
 * pointer for plans[i] and outs[i] a device array of plans[i]'s nbins doubles.
 * Results are bit-identical to calling poly_estimate on each field.
 *
 * The first call with a given (plans, fields, outs) list captures all the
 * launches into one CUDA graph, which later calls with the same list replay
 * with a single launch (the library keeps the 8 most recently used graphs).
 * Fields of one plan run in order on one branch of the graph (they share the
 * plan's workspace); different plans run on parallel branches.  A cached graph
 * reads the fields and writes the outputs at the addresses it was captured
 * with, so keep those buffers alive (or pass a new list); destroying or
 * retuning a plan drops the graphs that use it.  Calls with the same list
 * from several host threads at once are not supported.
 */
poly_status poly_estimate_batched(const poly_plan* plans, const void* const* fields, double* const* outs, int count,
                                  void* stream);

/*
 * Autotuner for the plan's contraction shape (no counterpart in the paper).
 * For a POLY_SPLIT_BF16 plan it times the tensor-core contraction on the
 * shell fields of delta_x (device, N^3 float) for each candidate shape:
 * at most 2, 3 or 4 M tiles per CTA group, and a CTA budget of 1/2, 1, 2, 3 or 4
 * times the SM count.  The plan keeps the fastest.  config_out receives an
 * opaque code for it (give it to poly_plan_set_config to restore the choice
 * without timing, e.g. from a cache on disk) and ms_out the contraction time
 * it measured.  Other precisions have nothing to tune: config 0, 0 ms.
 * Synchronises `stream`.  Results after tuning differ from the untuned plan
 * only in the order of the final FP64 sums (last bits); repeated estimates of
 * one tuned plan are bit-identical.
 */
poly_status poly_plan_tune(poly_plan plan, const void* delta_x, int* config_out, double* ms_out, void* stream);

/*
 * Apply a configuration code from poly_plan_tune (0: keep the current one).
 * POLY_ERR_ARG for a code poly_plan_tune does not produce.  A shape that
 * fails to build (shared memory, allocation) returns its error and rebuilds
 * the previous shape; if that fails too, later estimates of the plan return
 * POLY_ERR_UNSUPPORTED.
 */
poly_status poly_plan_set_config(poly_plan plan, int config);

/*
 * Wait for the plan's work on `stream` (host blocks) and report device-side
 * errors: POLY_ERR_CUDA for a failed kernel or runtime call,
 * POLY_ERR_TIMEOUT when a bounded wait inside a pipeline gave up (the
 * context stays usable; the estimate's outputs are then undefined).
 */
poly_status poly_plan_sync(poly_plan plan, void* stream);

/*
 * Release the plan, its workspace and the batched graphs that use it (NULL
 * is ignored).  The workspace is freed with cudaFree, which waits for the
 * device's outstanding work; buffers passed to the plan stay the caller's.
 */
void poly_plan_destroy(poly_plan plan);

/* Per-plan instrumentation: launch counter and CUDA events per stage. */
typedef struct {
    int64_t launches;   /* kernels this plan has launched since creation (excluding plan-time work) */
    float ms_forward;   /* last timed estimate: forward R2C transform */
    float ms_fields;    /* last timed estimate: shell gather + inverse transforms (all shells) */
    float ms_contract;  /* last timed estimate: the product-sum contraction kernel */
    float ms_reduce;    /* last timed estimate: cross-tile reduction + normalisation */
    double contract_flops; /* flops the contraction kernel executes per estimate (dense tiles; the tensor
                              path counts its three split products) */
} poly_stats;

/*
 * enable != 0: every following estimate records CUDA events between its
 * stages on its stream (a few microseconds of overhead); 0 disables.
 */
poly_status poly_plan_set_timing(poly_plan plan, int enable);

/* Launch count and stage durations of the last timed estimate (waits for its events). */
poly_status poly_plan_stats(poly_plan plan, poly_stats* out);

/*
 * Bispectrum of one small field without allocating any device memory.
 *
 * The paper has no counterpart; this is for callers that cannot call
 * cudaMalloc at the moment they need an estimate: code running after its
 * device-memory budget has been fixed, or code inside a framework that owns the
 * device allocator.  It computes what poly_estimate
 * computes for a POLY_FP32 plan of order 3 with the default (polygon) bins,
 * with the same kernels, but keeps every intermediate in one static device
 * array of 32 MiB that belongs to the library.  Every GPU that loads the
 * library holds those 32 MiB until the process exits.
 *
 *  N, L, nshell, edges: as for poly_plan_create (order is 3, flags 0).
 *  delta_x: device, N^3 float.   out: device, nbins double (B_b, paper order).
 *  counts: HOST, nbins int64: the exact polygon counts of these bins, e.g. from
 *          poly_plan_counts of a plan with the same N and edges, made earlier.
 *  stream: cudaStream_t; the call is asynchronous on it.
 *
 * Problems whose intermediates do not fit in 32 MiB (roughly nshell * N^3 * 4
 * bytes of fields plus a few MiB) are rejected with POLY_ERR_UNSUPPORTED and a
 * message from poly_last_error(); e.g. N = 64 with 16 shells fits, 256^3 does
 * not.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current: make it before any stream
 * capture.  Every call copies its host tables and `counts` into the array from
 * pageable host memory (cudaMemcpyAsync), so a call can wait for its stream
 * before it returns.  All calls share the array, and each overwrites it: calls
 * whose work overlaps on the GPU (other streams or host threads) race, so
 * serialise them.
 */
poly_status poly_estimate_noalloc(int N, double L, int nshell, const double* edges, const float* delta_x,
                                  const int64_t* counts, double* out, void* stream);

/* Static description of a status code. */
const char* poly_status_string(poly_status status);

/* Message of the last error on the calling thread ("" if none). */
const char* poly_last_error(void);

/*
 * Test hook: make the n-th following workspace allocation of poly_plan_create
 * fail (n >= 1; 0 disables).  Exercises the allocation-failure path on the
 * host without touching the device.
 */
void poly_debug_fail_alloc_after(int n);

#ifdef __cplusplus
}
#endif

#endif /* POLYSPEC_H */
