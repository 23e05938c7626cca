/*
 * oracle.c -- plain, slow FP64 CPU oracle for the FFT-based (Scoccimarro-type)
 * polyspectrum estimator of Tomlinson, Jeong & Kim, arXiv:1904.11055.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file.
 * Only tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline leg and
 * its --impl reference arm) load the shared library built from it.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Conventions (paper Sec. 1 for the transform pair, App. A for the discrete
 * FFTW form):
 *   forward  dhat(q) = sum_x delta(x) exp(-2 pi i q.x / N)      (unnormalised)
 *   inverse  D(x)    = sum_q F(q)     exp(+2 pi i q.x / N)      (unnormalised)
 *   grid index m in [0,N) carries the integer wavevector component
 *   q = m for m < ceil(N/2), q = m - N otherwise.
 *   Shell s (0-based) holds the q != 0 with edges[s]^2 <= |q|^2 < edges[s+1]^2,
 *   the half-width binning |q - k_s| < dk/2 of Sec. 2 and App. A written as
 *   edges k_s -/+ dk/2.
 *
 * Every routine is written in the order of the paper's equations; no blocking,
 * fusion or reordering beyond what the definitions state.  Sums over grid cells
 * are accumulated in FP64 in blocks of ORC_BLOCK cells (plain summation inside a
 * block, plain summation of block totals), which is a rounding-order choice only.
 *
 * Return codes: 0 ok, negative on bad arguments / allocation failure / a check
 * that failed (see orc_last_error()).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BLOCK 4096
#define ORC_PI 3.14159265358979323846

typedef struct {
    double re, im;
} cplx;

static char g_err[256] = "";
static int g_threads = 1;

static int fail(int code, const char* msg) {
    snprintf(g_err, sizeof g_err, "%s", msg);
    return code;
}

const char* orc_last_error(void) { return g_err; }

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------- */
/* a tiny static-chunk parallel-for over [0, n) on g_threads pthreads         */
/* ------------------------------------------------------------------------- */
typedef void (*range_fn)(void* ctx, int64_t begin, int64_t end, int tid);

typedef struct {
    range_fn fn;
    void* ctx;
    int64_t begin, end;
    int tid;
} par_job;

static void* par_trampoline(void* p) {
    par_job* j = (par_job*)p;
    j->fn(j->ctx, j->begin, j->end, j->tid);
    return NULL;
}

static void par_for(int64_t n, range_fn fn, void* ctx) {
    int nt = g_threads;
    if (nt > n) nt = (int)(n > 0 ? n : 1);
    if (nt <= 1) {
        fn(ctx, 0, n, 0);
        return;
    }
    pthread_t th[256];
    par_job jobs[256];
    if (nt > 256) nt = 256;
    for (int t = 0; t < nt; t++) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].begin = n * t / nt;
        jobs[t].end = n * (t + 1) / nt;
        jobs[t].tid = t;
        pthread_create(&th[t], NULL, par_trampoline, &jobs[t]);
    }
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------- */
/* own FFT: recursive mixed-radix decimation in time, any length              */
/* X[k] = sum_{r<p} W_n^{r k} Y_r[k mod m],  Y_r = DFT_m(x[r], x[r+p], ...)  */
/* with W_n = exp(sign * 2 pi i / n) and p the smallest prime factor of n.    */
/* ------------------------------------------------------------------------- */
static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

static void fft_rec(cplx* out, const cplx* in, int n, int is, const cplx* tw, int ntw, cplx* tmp) {
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int p = smallest_factor(n), m = n / p;
    for (int r = 0; r < p; r++) fft_rec(out + (size_t)r * m, in + (size_t)r * is, m, is * p, tw, ntw, tmp);
    int step = ntw / n;
    for (int k = 0; k < n; k++) {
        double ar = 0.0, ai = 0.0;
        for (int r = 0; r < p; r++) {
            cplx y = out[(size_t)r * m + (k % m)];
            cplx w = tw[(size_t)(((int64_t)r * k) % n) * step];
            ar += w.re * y.re - w.im * y.im;
            ai += w.re * y.im + w.im * y.re;
        }
        tmp[k].re = ar;
        tmp[k].im = ai;
    }
    memcpy(out, tmp, sizeof(cplx) * (size_t)n);
}

static cplx* twiddles(int n, int sign) {
    cplx* tw = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    if (!tw) return NULL;
    for (int j = 0; j < n; j++) {
        double a = 2.0 * ORC_PI * (double)j / (double)n;
        tw[j].re = cos(a);
        tw[j].im = sign * sin(a);
    }
    return tw;
}

/* in-place 1-D transform of n complex values spaced `stride` apart */
int orc_fft1d(double* data, int n, int sign) {
    if (n < 1 || (sign != 1 && sign != -1)) return fail(-1, "orc_fft1d: bad n or sign");
    cplx* a = (cplx*)data;
    cplx* tw = twiddles(n, sign);
    cplx* buf = (cplx*)malloc(sizeof(cplx) * 2 * (size_t)n);
    if (!tw || !buf) return fail(-2, "orc_fft1d: out of memory");
    fft_rec(buf, a, n, 1, tw, n, buf + n);
    memcpy(a, buf, sizeof(cplx) * (size_t)n);
    free(tw);
    free(buf);
    return 0;
}

typedef struct {
    cplx* a;
    int n[3];
    int axis;
    const cplx* tw;
    cplx* scratch; /* per thread: 3 * n[axis] */
} fft3_ctx;

static void fft3_lines(void* vctx, int64_t begin, int64_t end, int tid) {
    fft3_ctx* c = (fft3_ctx*)vctx;
    int n0 = c->n[0], n1 = c->n[1], n2 = c->n[2];
    int len = c->n[c->axis];
    cplx* line = c->scratch + (size_t)tid * 3 * len;
    cplx* out = line + len;
    cplx* tmp = out + len;
    for (int64_t L = begin; L < end; L++) {
        /* enumerate lines orthogonal to `axis` and their element stride */
        size_t base, stride;
        if (c->axis == 2) {
            base = (size_t)L * n2;
            stride = 1;
        } else if (c->axis == 1) {
            size_t i0 = (size_t)(L / n2), i2 = (size_t)(L % n2);
            base = i0 * n1 * n2 + i2;
            stride = (size_t)n2;
        } else {
            base = (size_t)L;
            stride = (size_t)n1 * n2;
        }
        for (int t = 0; t < len; t++) line[t] = c->a[base + (size_t)t * stride];
        fft_rec(out, line, len, 1, c->tw, len, tmp);
        for (int t = 0; t < len; t++) c->a[base + (size_t)t * stride] = out[t];
    }
    (void)n0;
}

/* in-place 3-D transform of an n0 x n1 x n2 complex array (last index fastest) */
int orc_fft3d(double* data, int n0, int n1, int n2, int sign) {
    if (n0 < 1 || n1 < 1 || n2 < 1 || (sign != 1 && sign != -1)) return fail(-1, "orc_fft3d: bad args");
    fft3_ctx c;
    c.a = (cplx*)data;
    c.n[0] = n0;
    c.n[1] = n1;
    c.n[2] = n2;
    for (int axis = 0; axis < 3; axis++) {
        int len = c.n[axis];
        cplx* tw = twiddles(len, sign);
        cplx* scratch = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)len * (size_t)(g_threads > 0 ? g_threads : 1));
        if (!tw || !scratch) {
            free(tw);
            free(scratch);
            return fail(-2, "orc_fft3d: out of memory");
        }
        c.axis = axis;
        c.tw = tw;
        c.scratch = scratch;
        int64_t nlines = ((int64_t)n0 * n1 * n2) / len;
        par_for(nlines, fft3_lines, &c);
        free(tw);
        free(scratch);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* shells (Sec. 2: |q - k_i| < dk/2, written with explicit edges)             */
/* ------------------------------------------------------------------------- */
static int freq_of(int m, int N) { return (m < (N + 1) / 2) ? m : m - N; }

static int shell_of_q2(int64_t q2, int nshell, const double* edges) {
    if (q2 == 0) return -1;
    double d = (double)q2;
    for (int s = 0; s < nshell; s++)
        if (edges[s] * edges[s] <= d && d < edges[s + 1] * edges[s + 1]) return s;
    return -1;
}

/* shell index (or -1) of every grid mode, laid out like the N^3 grid */
int orc_shell_map(int N, int nshell, const double* edges, int32_t* shell) {
    if (N < 2 || nshell < 1) return fail(-1, "orc_shell_map: bad args");
    for (int s = 0; s < nshell; s++)
        if (!(edges[s] >= 0.0 && edges[s + 1] > edges[s])) return fail(-1, "orc_shell_map: edges must increase");
    for (int a = 0; a < N; a++)
        for (int b = 0; b < N; b++)
            for (int c = 0; c < N; c++) {
                int64_t qa = freq_of(a, N), qb = freq_of(b, N), qc = freq_of(c, N);
                shell[((size_t)a * N + b) * N + c] = shell_of_q2(qa * qa + qb * qb + qc * qc, nshell, edges);
            }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* bins: k_1 >= k_2 >= ... >= k_n, row-major with k_n fastest (Sec. 4.2),     */
/* kept when the polygon inequality k_1 <= k_2 + ... + k_n holds on the       */
/* shell centres (App. B, Eq. polygon).  rule 1 keeps every sorted tuple.     */
/* Bins are reported with 1-based shell numbers, as in the paper.             */
/* ------------------------------------------------------------------------- */
static int64_t bins_rec(int order, int nshell, int rule, const double* centre, int depth, int* cur, int* out,
                        int64_t nb) {
    if (depth == order) {
        double rest = 0.0;
        for (int t = 1; t < order; t++) rest += centre[cur[t] - 1];
        if (rule == 1 || centre[cur[0] - 1] <= rest + 1e-9 * centre[cur[0] - 1]) {
            if (out)
                for (int t = 0; t < order; t++) out[nb * order + t] = cur[t];
            nb++;
        }
        return nb;
    }
    int hi = depth == 0 ? nshell : cur[depth - 1];
    for (int v = 1; v <= hi; v++) {
        cur[depth] = v;
        nb = bins_rec(order, nshell, rule, centre, depth + 1, cur, out, nb);
    }
    return nb;
}

int64_t orc_enumerate_bins(int nshell, const double* edges, int order, int rule, int32_t* out) {
    if (nshell < 1 || order < 2 || order > 8) return fail(-1, "orc_enumerate_bins: bad args");
    double* centre = (double*)malloc(sizeof(double) * (size_t)nshell);
    int cur[8];
    for (int s = 0; s < nshell; s++) centre[s] = 0.5 * (edges[s] + edges[s + 1]);
    int64_t nb = bins_rec(order, nshell, rule, centre, 0, cur, (int*)out, 0);
    free(centre);
    return nb;
}

/* ------------------------------------------------------------------------- */
/* forward transform of a real field: dhat(q) = sum_x delta(x) e^{-i q.x}     */
/* ------------------------------------------------------------------------- */
int orc_forward(int N, const double* delta, double* dhat /* 2*N^3, interleaved complex */) {
    size_t n3 = (size_t)N * N * N;
    cplx* a = (cplx*)dhat;
    for (size_t i = 0; i < n3; i++) {
        a[i].re = delta[i];
        a[i].im = 0.0;
    }
    return orc_fft3d(dhat, N, N, N, -1);
}

/* ------------------------------------------------------------------------- */
/* shell fields: D_s(x) = sum_{q in S_s} F(q) e^{+i q.x}  (Eq. Bkfast; App. A) */
/* With F = dhat this is I_{k_s}[x] up to the (2 pi)^3/N^3 factor of App. A;  */
/* with F = 1 it is the counting field iota_{k_s}[x] (Eq. Vn).                 */
/* `imag_max` (optional) receives max |Im D| / max |Re D| over the shells.     */
/* ------------------------------------------------------------------------- */
int orc_shell_fields(int N, const double* dhat /* complex N^3, or NULL for F = 1 */, const int32_t* shell_map,
                     int nsel, const int32_t* shells /* 0-based shells to build */,
                     double* fields /* nsel * N^3 */, double* imag_max) {
    size_t n3 = (size_t)N * N * N;
    cplx* work = (cplx*)malloc(sizeof(cplx) * n3);
    if (!work) return fail(-2, "orc_shell_fields: out of memory");
    double worst = 0.0;
    for (int t = 0; t < nsel; t++) {
        int s = shells[t];
        const cplx* F = (const cplx*)dhat;
        for (size_t i = 0; i < n3; i++) {
            if (shell_map[i] == s) {
                work[i].re = F ? F[i].re : 1.0;
                work[i].im = F ? F[i].im : 0.0;
            } else {
                work[i].re = 0.0;
                work[i].im = 0.0;
            }
        }
        int rc = orc_fft3d((double*)work, N, N, N, +1);
        if (rc) {
            free(work);
            return rc;
        }
        double mre = 0.0, mim = 0.0;
        double* f = fields + (size_t)t * n3;
        for (size_t i = 0; i < n3; i++) {
            f[i] = work[i].re;
            if (fabs(work[i].re) > mre) mre = fabs(work[i].re);
            if (fabs(work[i].im) > mim) mim = fabs(work[i].im);
        }
        double r = mre > 0.0 ? mim / mre : mim;
        if (r > worst) worst = r;
    }
    if (imag_max) *imag_max = worst;
    free(work);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* product sums over the grid (Eq. estimator, discrete form of App. A):       */
/*   S_b = sum_x prod_t D_{b_t}(x),   A_b = sum_x |prod_t D_{b_t}(x)|        */
/* `slot` maps a 1-based shell number to its row in `fields` (or -1).         */
/* ------------------------------------------------------------------------- */
typedef struct {
    size_t n3;
    int order;
    const double* fields;
    const int32_t* slot;
    const int32_t* bins;
    double* S;
    double* A;
} sums_ctx;

static void sums_range(void* vctx, int64_t begin, int64_t end, int tid) {
    sums_ctx* c = (sums_ctx*)vctx;
    (void)tid;
    for (int64_t b = begin; b < end; b++) {
        const double* f[8];
        for (int t = 0; t < c->order; t++) f[t] = c->fields + (size_t)c->slot[c->bins[b * c->order + t]] * c->n3;
        double tot = 0.0, atot = 0.0;
        for (size_t x0 = 0; x0 < c->n3; x0 += ORC_BLOCK) {
            size_t x1 = x0 + ORC_BLOCK < c->n3 ? x0 + ORC_BLOCK : c->n3;
            double blk = 0.0, ablk = 0.0;
            for (size_t x = x0; x < x1; x++) {
                double p = 1.0;
                for (int t = 0; t < c->order; t++) p *= f[t][x];
                blk += p;
                ablk += fabs(p);
            }
            tot += blk;
            atot += ablk;
        }
        c->S[b] = tot;
        if (c->A) c->A[b] = atot;
    }
}

int orc_product_sums(int N, const double* fields, const int32_t* slot, int order, int64_t nbins, const int32_t* bins,
                     double* S, double* A) {
    sums_ctx c = {(size_t)N * N * N, order, fields, slot, bins, S, A};
    for (int64_t b = 0; b < nbins * order; b++)
        if (slot[bins[b]] < 0) return fail(-1, "orc_product_sums: bin uses a shell with no field");
    par_for(nbins, sums_range, &c);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* exact polygon counts by pair convolutions, n = 2, 3, 4: the plain          */
/* definition (App. A), the number of n-tuples of grid modes q_t in shell k_t */
/* with q_1 + ... + q_n = 0 (mod N).  With                                    */
/*   P_ij(p) = #{(q, q') in S_i x S_j : q + q' = p (mod N)}                   */
/*           = round(IDFT(DFT(1_Si) DFT(1_Sj))(p) / N^3),                     */
/* integers of at most |S_i||S_j| (far below 2^52, so the FP64 transforms     */
/* round to them exactly; each is checked to lie within 1e-3 of one):         */
/*   n = 2: count = sum_p 1_S1(p) 1_S2(-p)                                    */
/*   n = 3: count = sum_p P_12(p) 1_S3(-p)                                    */
/*   n = 4: count = sum_p P_12(p) P_34(-p)                                    */
/* summed in 64-bit integers.  Shell numbers in `bins` are 1-based.           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int N, ka, kb;
    const int32_t* smap;
    const int32_t* pa; /* NULL: the indicator of shell ka */
    const int32_t* pb; /* NULL: the indicator of shell kb */
    int64_t part[256];
} cnt_ctx;

static void count_range(void* vctx, int64_t begin, int64_t end, int tid) {
    cnt_ctx* c = (cnt_ctx*)vctx;
    const int N = c->N;
    int64_t acc = 0;
    for (int64_t i = begin; i < end; i++) {
        const int a = (int)(i / ((int64_t)N * N)), b = (int)((i / N) % N), z = (int)(i % N);
        const int64_t j = ((int64_t)((N - a) % N) * N + (N - b) % N) * N + (N - z) % N; /* -p */
        const int64_t va = c->pa ? c->pa[i] : (c->smap[i] == c->ka);
        if (!va) continue;
        const int64_t vb = c->pb ? c->pb[j] : (c->smap[j] == c->kb);
        acc += va * vb;
    }
    c->part[tid] = acc;
}

static int64_t count_sum(int N, const int32_t* smap, const int32_t* pa, int ka, const int32_t* pb, int kb) {
    cnt_ctx c;
    memset(&c, 0, sizeof c);
    c.N = N;
    c.ka = ka;
    c.kb = kb;
    c.smap = smap;
    c.pa = pa;
    c.pb = pb;
    par_for((int64_t)N * N * N, count_range, &c);
    int64_t s = 0;
    for (int t = 0; t < 256; t++) s += c.part[t];
    return s;
}

/* DFT of the indicator of shell k (0-based), interleaved complex */
static int shell_dft(int N, const int32_t* smap, int k, double* F) {
    const size_t n3 = (size_t)N * N * N;
    for (size_t i = 0; i < n3; i++) {
        F[2 * i] = smap[i] == k ? 1.0 : 0.0;
        F[2 * i + 1] = 0.0;
    }
    return orc_fft3d(F, N, N, N, -1);
}

static int pair_conv(int N, const double* Fa, const double* Fb, double* work, int32_t* out) {
    const size_t n3 = (size_t)N * N * N;
    for (size_t i = 0; i < n3; i++) {
        const double ar = Fa[2 * i], ai = Fa[2 * i + 1], br = Fb[2 * i], bi = Fb[2 * i + 1];
        work[2 * i] = ar * br - ai * bi;
        work[2 * i + 1] = ar * bi + ai * br;
    }
    int rc = orc_fft3d(work, N, N, N, +1);
    if (rc) return rc;
    for (size_t i = 0; i < n3; i++) {
        const double v = work[2 * i] / (double)n3, r = nearbyint(v);
        if (fabs(v - r) > 1e-3 || fabs(work[2 * i + 1] / (double)n3) > 1e-3)
            return fail(-3, "orc_counts_exact: pair convolution is not an integer");
        out[i] = (int32_t)r;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* exact triangle counts (n = 3) for many bins at once: the same definition   */
/* and pair convolutions as above (count = sum_p P_12(p) 1_S3(-p)), with the  */
/* sum over p taken for every third shell in one pass over the grid,          */
/*   H_12(k) = sum_p P_12(p) [-p in S_k],  count(k1, k2, k3) = H_12(k3),      */
/* so that each pair (k1, k2) costs one convolution and one pass whatever the */
/* number of its bins.                                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
    int N, nshell;
    const int32_t* smap;
    const int32_t* P;
    int64_t* hist; /* [256][nshell + 1], indexed by 1-based shell */
} hist_ctx;

static void hist_range(void* vctx, int64_t begin, int64_t end, int tid) {
    hist_ctx* c = (hist_ctx*)vctx;
    const int N = c->N;
    int64_t* h = c->hist + (size_t)tid * (size_t)(c->nshell + 1);
    for (int64_t i = begin; i < end; i++) {
        const int32_t v = c->P[i];
        if (!v) continue;
        const int a = (int)(i / ((int64_t)N * N)), b = (int)((i / N) % N), z = (int)(i % N);
        const int64_t j = ((int64_t)((N - a) % N) * N + (N - b) % N) * N + (N - z) % N; /* -p */
        const int32_t k = c->smap[j];
        if (k >= 0) h[k + 1] += v;
    }
}

int orc_counts_triangles(int N, int nshell, const double* edges, int64_t nbins, const int32_t* bins, int64_t* counts) {
    if (N < 2 || nbins < 0) return fail(-1, "orc_counts_triangles: bad args");
    const size_t n3 = (size_t)N * N * N;
    int32_t* smap = (int32_t*)malloc(sizeof(int32_t) * n3);
    int* fslot = (int*)malloc(sizeof(int) * (size_t)(nshell + 1));
    int64_t* hist = (int64_t*)calloc((size_t)256 * (size_t)(nshell + 1), sizeof(int64_t));
    int64_t* tot = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nshell + 1));
    int rc = (!smap || !fslot || !hist || !tot) ? fail(-2, "orc_counts_triangles: out of memory")
                                                : orc_shell_map(N, nshell, edges, smap);
    int nf = 0;
    for (int s = 0; s <= nshell && fslot; s++) fslot[s] = -1;
    for (int64_t b = 0; b < nbins && !rc; b++) {
        const int32_t* k = bins + 3 * b;
        for (int t = 0; t < 3; t++)
            if (k[t] < 1 || k[t] > nshell) rc = fail(-1, "orc_counts_triangles: bin shell out of range");
        for (int t = 0; t < 2 && !rc; t++)
            if (fslot[k[t]] < 0) fslot[k[t]] = nf++;
    }
    double* F = rc || nf == 0 ? NULL : (double*)malloc(sizeof(double) * 2 * n3 * (size_t)nf);
    double* work = rc || nf == 0 ? NULL : (double*)malloc(sizeof(double) * 2 * n3);
    int32_t* P = rc || nf == 0 ? NULL : (int32_t*)malloc(sizeof(int32_t) * n3);
    if (!rc && nf > 0 && (!F || !work || !P)) rc = fail(-2, "orc_counts_triangles: out of memory");
    for (int s = 1; s <= nshell && !rc; s++)
        if (fslot[s] >= 0) rc = shell_dft(N, smap, s - 1, F + 2 * n3 * (size_t)fslot[s]);
    for (int64_t b = 0; b < nbins; b++) counts[b] = -1;
    /* pairs in the order of first appearance; every bin of a pair is filled from its histogram */
    for (int64_t b0 = 0; b0 < nbins && !rc; b0++) {
        if (counts[b0] >= 0) continue;
        const int k1 = bins[3 * b0], k2 = bins[3 * b0 + 1];
        rc = pair_conv(N, F + 2 * n3 * (size_t)fslot[k1], F + 2 * n3 * (size_t)fslot[k2], work, P);
        if (rc) break;
        memset(hist, 0, sizeof(int64_t) * 256 * (size_t)(nshell + 1));
        hist_ctx c = {N, nshell, smap, P, hist};
        par_for((int64_t)n3, hist_range, &c);
        for (int s = 0; s <= nshell; s++) {
            tot[s] = 0;
            for (int t = 0; t < 256; t++) tot[s] += hist[(size_t)t * (size_t)(nshell + 1) + s];
        }
        for (int64_t b = b0; b < nbins; b++)
            if (bins[3 * b] == k1 && bins[3 * b + 1] == k2) counts[b] = tot[bins[3 * b + 2]];
    }
    free(smap);
    free(fslot);
    free(hist);
    free(tot);
    free(F);
    free(work);
    free(P);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* exact counts for n = 5, 6 by group convolutions: the bin's shells split    */
/* into a first group of n - 3 (two for n = 5, three for n = 6) and a second  */
/* group of three.  With the closure map of a group g of shells,              */
/*   G_g(p) = #{one grid mode in each shell of g, the modes summing to p}     */
/*          = round(IDFT(prod_{s in g} DFT(1_Ss))(p) / N^3),                  */
/* integers of at most prod |S_s| (each checked to lie within 1e-3 of one),   */
/*   count = sum_p G_first(p) G_second(-p),  summed in 64-bit integers.       */
/* ------------------------------------------------------------------------- */
typedef struct {
    int N;
    const int64_t* a;
    const int64_t* b;
    int64_t part[256];
} cnt64_ctx;

static void count64_range(void* vctx, int64_t begin, int64_t end, int tid) {
    cnt64_ctx* c = (cnt64_ctx*)vctx;
    const int N = c->N;
    int64_t acc = 0;
    for (int64_t i = begin; i < end; i++) {
        if (!c->a[i]) continue;
        const int x = (int)(i / ((int64_t)N * N)), y = (int)((i / N) % N), z = (int)(i % N);
        const int64_t j = ((int64_t)((N - x) % N) * N + (N - y) % N) * N + (N - z) % N; /* -p */
        acc += c->a[i] * c->b[j];
    }
    c->part[tid] = acc;
}

static int group_map(int N, const double* const* F, int nf, double* work, int64_t* out) {
    const size_t n3 = (size_t)N * N * N;
    for (size_t i = 0; i < n3; i++) {
        double re = F[0][2 * i], im = F[0][2 * i + 1];
        for (int f = 1; f < nf; f++) {
            const double br = F[f][2 * i], bi = F[f][2 * i + 1];
            const double t = re * br - im * bi;
            im = re * bi + im * br;
            re = t;
        }
        work[2 * i] = re;
        work[2 * i + 1] = im;
    }
    int rc = orc_fft3d(work, N, N, N, +1);
    if (rc) return rc;
    for (size_t i = 0; i < n3; i++) {
        const double v = work[2 * i] / (double)n3, r = nearbyint(v);
        if (fabs(v - r) > 1e-3 || fabs(work[2 * i + 1] / (double)n3) > 1e-3)
            return fail(-3, "orc_counts_exact: group convolution is not an integer");
        out[i] = (int64_t)r;
    }
    return 0;
}

static int counts_exact_groups(int N, int nshell, const double* edges, int order, int64_t nbins, const int32_t* bins,
                               int64_t* counts) {
    const size_t n3 = (size_t)N * N * N;
    const int g1 = order - 3; /* size of the first group; the second has three shells */
    int32_t* smap = (int32_t*)malloc(sizeof(int32_t) * n3);
    int* fslot = (int*)malloc(sizeof(int) * (size_t)(nshell + 1));
    /* distinct groups: key = shells (1-based) padded with 0, stored 3 per group */
    int32_t* gkey = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(2 * nbins + 1));
    int64_t* bg = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)(nbins + 1)); /* per bin: its two group ids */
    int rc = (!smap || !fslot || !gkey || !bg) ? fail(-2, "orc_counts_exact: out of memory")
                                                : orc_shell_map(N, nshell, edges, smap);
    int nf = 0;
    int64_t ng = 0;
    for (int s = 0; s <= nshell && fslot; s++) fslot[s] = -1;
    for (int64_t b = 0; b < nbins && !rc; b++) {
        const int32_t* k = bins + b * order;
        for (int t = 0; t < order; t++) {
            if (k[t] < 1 || k[t] > nshell) rc = fail(-1, "orc_counts_exact: bin shell out of range");
            else if (fslot[k[t]] < 0) fslot[k[t]] = nf++;
        }
        for (int h = 0; h < 2 && !rc; h++) {
            int32_t key[3] = {0, 0, 0};
            const int first = h == 0 ? 0 : g1, size = h == 0 ? g1 : 3;
            for (int t = 0; t < size; t++) key[t] = k[first + t];
            int64_t g = 0;
            while (g < ng && memcmp(gkey + 3 * g, key, sizeof key)) g++;
            if (g == ng) memcpy(gkey + 3 * ng++, key, sizeof key);
            bg[2 * b + h] = g;
        }
    }
    double* F = rc ? NULL : (double*)malloc(sizeof(double) * 2 * n3 * (size_t)(nf > 0 ? nf : 1));
    double* work = rc ? NULL : (double*)malloc(sizeof(double) * 2 * n3);
    int64_t* G = rc ? NULL : (int64_t*)malloc(sizeof(int64_t) * n3 * (size_t)(ng > 0 ? ng : 1));
    if (!rc && (!F || !work || !G)) rc = fail(-2, "orc_counts_exact: out of memory");
    for (int s = 1; s <= nshell && !rc; s++)
        if (fslot[s] >= 0) rc = shell_dft(N, smap, s - 1, F + 2 * n3 * (size_t)fslot[s]);
    for (int64_t g = 0; g < ng && !rc; g++) {
        const double* Fs[3];
        int nfg = 0;
        for (int t = 0; t < 3; t++)
            if (gkey[3 * g + t] > 0) Fs[nfg++] = F + 2 * n3 * (size_t)fslot[gkey[3 * g + t]];
        rc = group_map(N, Fs, nfg, work, G + n3 * (size_t)g);
    }
    for (int64_t b = 0; b < nbins && !rc; b++) {
        cnt64_ctx c;
        memset(&c, 0, sizeof c);
        c.N = N;
        c.a = G + n3 * (size_t)bg[2 * b];
        c.b = G + n3 * (size_t)bg[2 * b + 1];
        par_for((int64_t)n3, count64_range, &c);
        int64_t sum = 0;
        for (int t = 0; t < 256; t++) sum += c.part[t];
        counts[b] = sum;
    }
    free(smap);
    free(fslot);
    free(gkey);
    free(bg);
    free(F);
    free(work);
    free(G);
    return rc;
}

int orc_counts_exact(int N, int nshell, const double* edges, int order, int64_t nbins, const int32_t* bins,
                     int64_t* counts) {
    if (N < 2 || order < 2 || order > 6 || nbins < 0) return fail(-1, "orc_counts_exact: bad args (order 2..6)");
    if (order >= 5) return counts_exact_groups(N, nshell, edges, order, nbins, bins, counts);
    const size_t n3 = (size_t)N * N * N;
    int32_t* smap = (int32_t*)malloc(sizeof(int32_t) * n3);
    if (!smap) return fail(-2, "orc_counts_exact: out of memory");
    int rc = orc_shell_map(N, nshell, edges, smap);
    /* shells whose DFT is needed: the members of every pair (k1, k2) and, for n = 4, (k3, k4) */
    int* fslot = (int*)malloc(sizeof(int) * (size_t)(nshell + 1));
    int* pslot = (int*)malloc(sizeof(int) * (size_t)(nshell + 1) * (size_t)(nshell + 1));
    int nf = 0, np = 0;
    for (int s = 0; s <= nshell; s++) fslot[s] = -1;
    for (int64_t i = 0; i < (int64_t)(nshell + 1) * (nshell + 1); i++) pslot[i] = -1;
    for (int64_t b = 0; b < nbins && !rc; b++) {
        const int32_t* k = bins + b * order;
        for (int t = 0; t < order; t++)
            if (k[t] < 1 || k[t] > nshell) rc = fail(-1, "orc_counts_exact: bin shell out of range");
        if (rc || order == 2) continue;
        for (int h = 0; h + 1 < (order == 4 ? 4 : 2); h += 2) {
            const int a = k[h], c = k[h + 1];
            if (fslot[a] < 0) fslot[a] = nf++;
            if (fslot[c] < 0) fslot[c] = nf++;
            if (pslot[a * (nshell + 1) + c] < 0) pslot[a * (nshell + 1) + c] = np++;
        }
    }
    double* F = NULL;
    double* work = NULL;
    int32_t* P = NULL;
    if (!rc && np > 0) {
        F = (double*)malloc(sizeof(double) * 2 * n3 * (size_t)nf);
        work = (double*)malloc(sizeof(double) * 2 * n3);
        P = (int32_t*)malloc(sizeof(int32_t) * n3 * (size_t)np);
        if (!F || !work || !P) rc = fail(-2, "orc_counts_exact: out of memory");
        for (int s = 1; s <= nshell && !rc; s++)
            if (fslot[s] >= 0) rc = shell_dft(N, smap, s - 1, F + 2 * n3 * (size_t)fslot[s]);
        for (int a = 1; a <= nshell && !rc; a++)
            for (int c = 1; c <= nshell && !rc; c++) {
                const int q = pslot[a * (nshell + 1) + c];
                if (q >= 0)
                    rc = pair_conv(N, F + 2 * n3 * (size_t)fslot[a], F + 2 * n3 * (size_t)fslot[c], work,
                                   P + n3 * (size_t)q);
            }
    }
    for (int64_t b = 0; b < nbins && !rc; b++) {
        const int32_t* k = bins + b * order;
        if (order == 2) {
            counts[b] = count_sum(N, smap, NULL, k[0] - 1, NULL, k[1] - 1);
        } else {
            const int32_t* p12 = P + n3 * (size_t)pslot[k[0] * (nshell + 1) + k[1]];
            if (order == 3) counts[b] = count_sum(N, smap, p12, 0, NULL, k[2] - 1);
            else counts[b] = count_sum(N, smap, p12, 0, P + n3 * (size_t)pslot[k[2] * (nshell + 1) + k[3]], 0);
        }
    }
    free(smap);
    free(fslot);
    free(pslot);
    free(F);
    free(work);
    free(P);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* redshift-space multipoles (the extension the paper points to in Sec. 5,    */
/* following Scoccimarro 2015): the first leg of each bin carries the         */
/* Legendre weight L_ell(mu), mu = q_z/|q| (plane-parallel line of sight      */
/* along the grid's z axis):                                                  */
/*   D^ell_k(x) = sum_{q in S_k} L_ell(mu_q) dhat(q) e^{+2 pi i q.x/N}         */
/*   S^ell_b    = sum_x D^ell_{k1}(x) prod_{t > 1} D_{kt}(x)                   */
/*   B^ell_b    = (2 ell + 1) (V^{n-1}/N^{3n}) S^ell_b / (N^3 count_b)         */
/* Even ell only: L_ell(-mu) = L_ell(mu) keeps the weighted fields real.      */
/* ell = 0 is the monopole B_b.                                               */
/* ------------------------------------------------------------------------- */
static double legendre(int ell, double mu) {
    double p0 = 1.0, p1 = mu;
    if (ell == 0) return p0;
    for (int n = 1; n < ell; n++) { /* Bonnet: (n+1) P_{n+1} = (2n+1) mu P_n - n P_{n-1} */
        const double p2 = ((2.0 * n + 1.0) * mu * p1 - n * p0) / (n + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

static int shell_fields_weighted(int N, const double* dhat, const int32_t* smap, int nsel, const int32_t* shells,
                                 int ell, double* fields) {
    const size_t n3 = (size_t)N * N * N;
    cplx* work = (cplx*)malloc(sizeof(cplx) * n3);
    if (!work) return fail(-2, "orc_estimate_ell: out of memory");
    const cplx* F = (const cplx*)dhat;
    for (int t = 0; t < nsel; t++) {
        for (size_t i = 0; i < n3; i++) {
            work[i].re = work[i].im = 0.0;
            if (smap[i] != shells[t]) continue;
            const int x = (int)(i / ((size_t)N * N)), y = (int)((i / N) % N), z = (int)(i % N);
            const double qx = x < (N + 1) / 2 ? x : x - N, qy = y < (N + 1) / 2 ? y : y - N,
                         qz = z < (N + 1) / 2 ? z : z - N;
            const double w = legendre(ell, qz / sqrt(qx * qx + qy * qy + qz * qz));
            work[i].re = w * F[i].re;
            work[i].im = w * F[i].im;
        }
        int rc = orc_fft3d((double*)work, N, N, N, +1);
        if (rc) {
            free(work);
            return rc;
        }
        for (size_t i = 0; i < n3; i++) fields[(size_t)t * n3 + i] = work[i].re;
    }
    free(work);
    return 0;
}

int orc_estimate(int N, double L, const double* delta, int nshell, const double* edges, int order, int64_t nbins,
                 const int32_t* bins, double* B, double* R, double* scale, int64_t* counts, double* S_out,
                 double* imag_max);

int orc_estimate_ell(int N, double L, const double* delta, int nshell, const double* edges, int order, int ell,
                     int64_t nbins, const int32_t* bins, double* B, double* scale, int64_t* counts) {
    if (N < 2 || L <= 0.0 || order < 2 || order > 8 || nbins < 0 || ell < 0 || ell > 8 || (ell & 1))
        return fail(-1, "orc_estimate_ell: bad args (even ell in [0, 8])");
    const size_t n3 = (size_t)N * N * N;
    /* counts: those of the monopole estimator (they do not depend on the weight) */
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nbins > 0 ? nbins : 1));
    int32_t* smap = (int32_t*)malloc(sizeof(int32_t) * n3);
    int32_t* slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * nshell + 1));
    int32_t* sel = (int32_t*)malloc(sizeof(int32_t) * (size_t)nshell);
    int32_t* bins2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nbins * order > 0 ? nbins * order : 1));
    double* dhat = (double*)malloc(sizeof(double) * 2 * n3);
    double* S = (double*)malloc(sizeof(double) * (size_t)(nbins > 0 ? nbins : 1));
    double* A = (double*)malloc(sizeof(double) * (size_t)(nbins > 0 ? nbins : 1));
    if (!cnt || !smap || !slot || !sel || !bins2 || !dhat || !S || !A) return fail(-2, "orc_estimate_ell: out of memory");
    int rc = orc_estimate(N, L, delta, nshell, edges, order, nbins, bins, NULL, NULL, NULL, cnt, NULL, NULL);
    if (!rc) rc = orc_shell_map(N, nshell, edges, smap);
    /* fields: [unweighted | weighted] per used shell; the first leg reads "shell" k1 + nshell */
    int nsel = 0;
    for (int s = 0; s <= 2 * nshell; s++) slot[s] = -1;
    for (int64_t i = 0; i < nbins * order && !rc; i++) {
        const int k = bins[i];
        if (k < 1 || k > nshell) rc = fail(-1, "orc_estimate_ell: bin shell out of range");
        else if (slot[k] < 0) {
            slot[k] = nsel;
            sel[nsel++] = k - 1;
        }
    }
    for (int s = 1; s <= nshell; s++)
        if (slot[s] >= 0) slot[s + nshell] = nsel + slot[s];
    for (int64_t b = 0; b < nbins; b++)
        for (int t = 0; t < order; t++) bins2[b * order + t] = bins[b * order + t] + (t == 0 ? nshell : 0);
    double* fields = rc ? NULL : (double*)malloc(sizeof(double) * n3 * (size_t)(2 * (nsel > 0 ? nsel : 1)));
    if (!rc && !fields) rc = fail(-2, "orc_estimate_ell: out of memory");
    double im = 0.0;
    if (!rc) rc = orc_forward(N, delta, dhat);
    if (!rc) rc = orc_shell_fields(N, dhat, smap, nsel, sel, fields, &im);
    if (!rc) rc = shell_fields_weighted(N, dhat, smap, nsel, sel, ell, fields + n3 * (size_t)nsel);
    if (!rc) rc = orc_product_sums(N, fields, slot, order, nbins, bins2, S, A);
    if (!rc) {
        const double n3d = (double)n3, norm = (2.0 * ell + 1.0) * pow(L * L * L, order - 1) / pow(n3d, order);
        for (int64_t b = 0; b < nbins; b++) {
            const double den = n3d * (double)cnt[b];
            if (B) B[b] = cnt[b] > 0 ? norm * S[b] / den : 0.0;
            if (scale) scale[b] = cnt[b] > 0 ? A[b] / den : 0.0;
            if (counts) counts[b] = cnt[b];
        }
    }
    free(cnt);
    free(smap);
    free(slot);
    free(sel);
    free(bins2);
    free(dhat);
    free(S);
    free(A);
    free(fields);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* disconnected part of the trispectrum estimator (n = 4; not in the paper,   */
/* whose Eq. estimator keeps it): the closed quadrilaterals that split into   */
/* two zero-sum pairs, summed over the three pairings of Wick's theorem with  */
/* the measured per-mode power |dhat(q)|^2 (real delta: dhat(-q) = dhat(q)*). */
/* A pairing (a b)(c d) needs q_b = -q_a and q_d = -q_c, i.e. equal shells    */
/* k_a = k_b and k_c = k_d (disjoint shells, S = -S); with                    */
/*   P(k) = sum_{q in S_k} |dhat(q)|^2                                        */
/*   S_disc_b = N^3 [d(k1,k2) d(k3,k4) P(k1) P(k3) + d(k1,k3) d(k2,k4) P(k1) P(k2) */
/*                   + d(k1,k4) d(k2,k3) P(k1) P(k2)]                         */
/* and the estimator's normalisation B_disc_b = c_4 S_disc_b / (N^3 count_b). */
/* ------------------------------------------------------------------------- */
int orc_disconnected(int N, double L, const double* delta, int nshell, const double* edges, int64_t nbins,
                     const int32_t* bins, const int64_t* counts, double* B_disc, double* P_out) {
    if (N < 2 || L <= 0.0 || nbins < 0 || nshell < 1) return fail(-1, "orc_disconnected: bad args");
    const size_t n3 = (size_t)N * N * N;
    int32_t* smap = (int32_t*)malloc(sizeof(int32_t) * n3);
    double* dhat = (double*)malloc(sizeof(double) * 2 * n3);
    double* P = (double*)calloc((size_t)nshell, sizeof(double));
    if (!smap || !dhat || !P) return fail(-2, "orc_disconnected: out of memory");
    int rc = orc_shell_map(N, nshell, edges, smap);
    if (!rc) rc = orc_forward(N, delta, dhat);
    for (size_t i = 0; i < n3 && !rc; i++)
        if (smap[i] >= 0) P[smap[i]] += dhat[2 * i] * dhat[2 * i] + dhat[2 * i + 1] * dhat[2 * i + 1];
    const double n3d = (double)n3, norm = pow(L * L * L, 3) / pow(n3d, 4);
    for (int64_t b = 0; b < nbins && !rc; b++) {
        const int32_t* k = bins + 4 * b;
        for (int t = 0; t < 4; t++)
            if (k[t] < 1 || k[t] > nshell) rc = fail(-1, "orc_disconnected: bin shell out of range");
        if (rc) break;
        const double p1 = P[k[0] - 1], p2 = P[k[1] - 1], p3 = P[k[2] - 1];
        double sd = 0.0;
        if (k[0] == k[1] && k[2] == k[3]) sd += p1 * p3;
        if (k[0] == k[2] && k[1] == k[3]) sd += p1 * p2;
        if (k[0] == k[3] && k[1] == k[2]) sd += p1 * p2;
        sd *= n3d;
        B_disc[b] = counts[b] > 0 ? norm * sd / (n3d * (double)counts[b]) : 0.0;
    }
    if (!rc && P_out) memcpy(P_out, P, sizeof(double) * (size_t)nshell);
    free(smap);
    free(dhat);
    free(P);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* whole estimator (Eqs. estimator, volume, Vn; App. A):                      */
/*   count_b = (1/N^3) sum_x prod iota  (an integer: the number of closed     */
/*             n-gons of grid modes, Eq. Ncalc with V_f = k_F^3)              */
/*   B_b     = (V^{n-1}/N^{3n}) * S_b / (N^3 count_b)                         */
/*   R_b     = S_b / (N^3 count_b),  scale_b = A_b / (N^3 count_b)            */
/* Only the shells used by `bins` are transformed, so a sample of bins at a   */
/* large N costs one inverse FFT per distinct shell.                          */
/* ------------------------------------------------------------------------- */
int orc_estimate(int N, double L, const double* delta, int nshell, const double* edges, int order, int64_t nbins,
                 const int32_t* bins, double* B, double* R, double* scale, int64_t* counts, double* S_out,
                 double* imag_max) {
    if (N < 2 || L <= 0.0 || order < 2 || order > 8 || nbins < 0) return fail(-1, "orc_estimate: bad args");
    size_t n3 = (size_t)N * N * N;
    int32_t* smap = (int32_t*)malloc(sizeof(int32_t) * n3);
    int32_t* slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nshell + 1));
    int32_t* sel = (int32_t*)malloc(sizeof(int32_t) * (size_t)nshell);
    if (!smap || !slot || !sel) return fail(-2, "orc_estimate: out of memory");
    int rc = orc_shell_map(N, nshell, edges, smap);
    if (rc) return rc;
    for (int s = 0; s <= nshell; s++) slot[s] = -1;
    int nsel = 0;
    for (int64_t i = 0; i < nbins * order; i++) {
        int k = bins[i];
        if (k < 1 || k > nshell) return fail(-1, "orc_estimate: bin shell out of range");
        if (slot[k] < 0) {
            slot[k] = nsel;
            sel[nsel++] = k - 1;
        }
    }
    double* dhat = (double*)malloc(sizeof(double) * 2 * n3);
    double* fields = (double*)malloc(sizeof(double) * n3 * (size_t)(nsel > 0 ? nsel : 1));
    double* S = (double*)malloc(sizeof(double) * (size_t)(nbins > 0 ? nbins : 1));
    double* A = (double*)malloc(sizeof(double) * (size_t)(nbins > 0 ? nbins : 1));
    double* C = (double*)malloc(sizeof(double) * (size_t)(nbins > 0 ? nbins : 1));
    if (!dhat || !fields || !S || !A || !C) return fail(-2, "orc_estimate: out of memory");
    double im1 = 0.0, im2 = 0.0;
    rc = orc_forward(N, delta, dhat);
    if (!rc) rc = orc_shell_fields(N, dhat, smap, nsel, sel, fields, &im1);
    if (!rc) rc = orc_product_sums(N, fields, slot, order, nbins, bins, S, A);
    /* counting fields: the same pipeline on a grid of unity (Sec. 4) */
    if (!rc) rc = orc_shell_fields(N, NULL, smap, nsel, sel, fields, &im2);
    if (!rc) rc = orc_product_sums(N, fields, slot, order, nbins, bins, C, NULL);
    /* counts: the counting-field sum where FP64 keeps it within 1e-6 of an integer;     */
    /* otherwise (large counts at n >= 4) the exact convolution count of the same bin      */
    int64_t* exact = NULL;
    if (!rc) {
        int64_t nbad = 0;
        for (int64_t b = 0; b < nbins; b++)
            if (fabs(C[b] / (double)n3 - nearbyint(C[b] / (double)n3)) > 1e-6) nbad++;
        if (nbad > 0 && order > 6) rc = fail(-3, "orc_estimate: polygon count is not an integer");
        if (nbad > 0 && !rc) {
            int32_t* bad = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nbad * order));
            exact = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbins);
            if (!bad || !exact) rc = fail(-2, "orc_estimate: out of memory");
            int64_t j = 0;
            for (int64_t b = 0; b < nbins && !rc; b++)
                if (fabs(C[b] / (double)n3 - nearbyint(C[b] / (double)n3)) > 1e-6)
                    memcpy(bad + (j++) * order, bins + b * order, sizeof(int32_t) * (size_t)order);
            int64_t* cb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nbad > 0 ? nbad : 1));
            if (!rc && !cb) rc = fail(-2, "orc_estimate: out of memory");
            if (!rc) rc = orc_counts_exact(N, nshell, edges, order, nbad, bad, cb);
            j = 0;
            for (int64_t b = 0; b < nbins && !rc; b++)
                exact[b] = fabs(C[b] / (double)n3 - nearbyint(C[b] / (double)n3)) > 1e-6 ? cb[j++] : -1;
            free(bad);
            free(cb);
        }
    }
    if (!rc) {
        double n3d = (double)n3;
        double norm = pow(L * L * L, order - 1) / pow(n3d, order);
        for (int64_t b = 0; b < nbins; b++) {
            double v = C[b] / n3d;
            int64_t cnt = (exact && exact[b] >= 0) ? exact[b] : (int64_t)nearbyint(v);
            if (counts) counts[b] = cnt;
            if (S_out) S_out[b] = S[b];
            double den = n3d * (double)cnt;
            if (R) R[b] = cnt > 0 ? S[b] / den : 0.0;
            if (scale) scale[b] = cnt > 0 ? A[b] / den : 0.0;
            if (B) B[b] = cnt > 0 ? norm * S[b] / den : 0.0;
        }
    }
    if (imag_max) *imag_max = im1 > im2 ? im1 : im2;
    free(exact);
    free(smap);
    free(slot);
    free(sel);
    free(dhat);
    free(fields);
    free(S);
    free(A);
    free(C);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* direct sampling of polygons (Eq. estimateBk and its n-gon form): loop over */
/* q_1..q_{n-1} in their shells, close with q_n = -(q_1+...+q_{n-1}) mod N,  */
/* keep the tuple when q_n lies in shell k_n.                                 */
/*   S_b = N^3 * Re sum prod dhat(q_t),   count_b = number of such tuples    */
/* `dhat` may be NULL (a grid of unity: only counts).                         */
/* ------------------------------------------------------------------------- */
typedef struct {
    int N, order, nshell;
    const cplx* dhat;
    const int32_t* smap;
    const int32_t* bins;
    int32_t** modes; /* per shell: flat grid indices */
    int32_t* nmodes;
    double* S;
    int64_t* counts;
} direct_ctx;

static void direct_range(void* vctx, int64_t begin, int64_t end, int tid) {
    direct_ctx* c = (direct_ctx*)vctx;
    (void)tid;
    int N = c->N, n = c->order;
    for (int64_t b = begin; b < end; b++) {
        const int32_t* k = c->bins + b * n;
        int idx[8];
        int64_t cnt = 0;
        double sre = 0.0, sim = 0.0;
        int depth = 0;
        idx[0] = -1;
        /* iterative odometer over q_1 .. q_{n-1} */
        while (depth >= 0) {
            idx[depth]++;
            if (idx[depth] >= c->nmodes[k[depth] - 1]) {
                depth--;
                continue;
            }
            if (depth < n - 2) {
                depth++;
                idx[depth] = -1;
                continue;
            }
            int sa = 0, sb = 0, sc = 0;
            double pre = 1.0, pim = 0.0;
            for (int t = 0; t < n - 1; t++) {
                int32_t g = c->modes[k[t] - 1][idx[t]];
                int a = g / (N * N), bb = (g / N) % N, cc = g % N;
                sa += a;
                sb += bb;
                sc += cc;
                if (c->dhat) {
                    double r2 = pre * c->dhat[g].re - pim * c->dhat[g].im;
                    double i2 = pre * c->dhat[g].im + pim * c->dhat[g].re;
                    pre = r2;
                    pim = i2;
                }
            }
            int la = ((-sa) % N + N) % N, lb = ((-sb) % N + N) % N, lc = ((-sc) % N + N) % N;
            int32_t gl = ((int32_t)la * N + lb) * N + lc;
            if (c->smap[gl] == k[n - 1] - 1) {
                cnt++;
                if (c->dhat) {
                    sre += pre * c->dhat[gl].re - pim * c->dhat[gl].im;
                    sim += pre * c->dhat[gl].im + pim * c->dhat[gl].re;
                }
            }
        }
        c->counts[b] = cnt;
        if (c->S) c->S[b] = (double)N * N * N * sre;
        (void)sim;
    }
}

int orc_direct_sample(int N, const double* delta /* NULL: counts only */, int nshell, const double* edges, int order,
                      int64_t nbins, const int32_t* bins, double* S, int64_t* counts) {
    if (N < 2 || order < 2 || order > 8) return fail(-1, "orc_direct_sample: bad args");
    size_t n3 = (size_t)N * N * N;
    int32_t* smap = (int32_t*)malloc(sizeof(int32_t) * n3);
    int rc = orc_shell_map(N, nshell, edges, smap);
    if (rc) return rc;
    int32_t** modes = (int32_t**)calloc((size_t)nshell, sizeof(int32_t*));
    int32_t* nm = (int32_t*)calloc((size_t)nshell, sizeof(int32_t));
    for (size_t i = 0; i < n3; i++)
        if (smap[i] >= 0) nm[smap[i]]++;
    for (int s = 0; s < nshell; s++) modes[s] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nm[s] + 1));
    int32_t* fill = (int32_t*)calloc((size_t)nshell, sizeof(int32_t));
    for (size_t i = 0; i < n3; i++)
        if (smap[i] >= 0) modes[smap[i]][fill[smap[i]]++] = (int32_t)i;
    double* dhat = NULL;
    if (delta) {
        dhat = (double*)malloc(sizeof(double) * 2 * n3);
        rc = orc_forward(N, delta, dhat);
    }
    if (!rc) {
        direct_ctx c = {N, order, nshell, (const cplx*)dhat, smap, bins, modes, nm, delta ? S : NULL, counts};
        par_for(nbins, direct_range, &c);
    }
    for (int s = 0; s < nshell; s++) free(modes[s]);
    free(modes);
    free(nm);
    free(fill);
    free(smap);
    free(dhat);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* full-shape trispectrum (Eq. Tkfull, which the paper leaves as future       */
/* work): the closed quadrilaterals of one bin (k1, k2, k3, k4), split by the */
/* diagonals p1 = q1 - q2 and p2 = q1 - q3 (Eq. Tkfull's                      */
/* delta_D(p1 - q1 + q2) delta_D(p2 - q1 + q3)) into diagonal bins            */
/* j: de_j^2 <= |p|^2 < de_{j+1}^2 (p = 0 falls in bin 0 when de_0 = 0):      */
/*   S[j1][j2]     = N^3 Re sum prod_t dhat(q_t)                             */
/*   count[j1][j2] = the number of those quadrilaterals,                      */
/* over q_t in S_{k_t} with q1 + q2 + q3 + q4 = 0 (mod N); the components of  */
/* p are differences of the signed (-N/2 .. N/2 - 1) representatives.        */
/*   A[j1][j2]     = N^3 sum prod_t |dhat(q_t)|  (the scale of rounding       */
/*                   errors in S, for error bars; optional)                  */
/* Summed over diagonal bins that cover every |p| they give S_b and count_b   */
/* of the angle-averaged trispectrum.  Direct enumeration over q1, q2, q3.    */
/* `delta` may be NULL (counts only).                                         */
/* ------------------------------------------------------------------------- */
typedef struct {
    int N, ndiag;
    const double* de2;
    const cplx* dhat;
    const int32_t* smap;
    int32_t* modes[4];
    int32_t nm[4];
    int k4;
    double* S;   /* [256][ndiag * ndiag] */
    double* A;   /* [256][ndiag * ndiag] */
    int64_t* C;  /* [256][ndiag * ndiag] */
} tfull_ctx;

static int signed_freq(int i, int N) { return i < (N + 1) / 2 ? i : i - N; }

static int diag_bin(const double* de2, int nd, double p2) {
    for (int j = 0; j < nd; j++)
        if (de2[j] <= p2 && p2 < de2[j + 1]) return j;
    return -1;
}

static void tfull_range(void* vctx, int64_t begin, int64_t end, int tid) {
    tfull_ctx* c = (tfull_ctx*)vctx;
    const int N = c->N, nd = c->ndiag;
    double* S = c->S + (size_t)tid * nd * nd;
    double* A = c->A + (size_t)tid * nd * nd;
    int64_t* C = c->C + (size_t)tid * nd * nd;
    for (int64_t a = begin; a < end; a++) {
        const int32_t i1 = c->modes[0][a];
        const int x1 = (int)(i1 / (N * N)), y1 = (int)((i1 / N) % N), z1 = (int)(i1 % N);
        for (int32_t b = 0; b < c->nm[1]; b++) {
            const int32_t i2 = c->modes[1][b];
            const int x2 = (int)(i2 / (N * N)), y2 = (int)((i2 / N) % N), z2 = (int)(i2 % N);
            const double u0 = signed_freq(x1, N) - signed_freq(x2, N), u1 = signed_freq(y1, N) - signed_freq(y2, N),
                         u2 = signed_freq(z1, N) - signed_freq(z2, N);
            const int j1 = diag_bin(c->de2, nd, u0 * u0 + u1 * u1 + u2 * u2);
            if (j1 < 0) continue;
            for (int32_t g = 0; g < c->nm[2]; g++) {
                const int32_t i3 = c->modes[2][g];
                const int x3 = (int)(i3 / (N * N)), y3 = (int)((i3 / N) % N), z3 = (int)(i3 % N);
                const int x4 = ((-(x1 + x2 + x3)) % N + N) % N, y4 = ((-(y1 + y2 + y3)) % N + N) % N,
                          z4 = ((-(z1 + z2 + z3)) % N + N) % N;
                const int64_t i4 = ((int64_t)x4 * N + y4) * N + z4;
                if (c->smap[i4] != c->k4) continue;
                const double w0 = signed_freq(x1, N) - signed_freq(x3, N), w1 = signed_freq(y1, N) - signed_freq(y3, N),
                             w2 = signed_freq(z1, N) - signed_freq(z3, N);
                const int j2 = diag_bin(c->de2, nd, w0 * w0 + w1 * w1 + w2 * w2);
                if (j2 < 0) continue;
                C[j1 * nd + j2]++;
                if (c->dhat) {
                    const cplx f1 = c->dhat[i1], f2 = c->dhat[i2], f3 = c->dhat[i3], f4 = c->dhat[i4];
                    const double ar = f1.re * f2.re - f1.im * f2.im, ai = f1.re * f2.im + f1.im * f2.re;
                    const double br = f3.re * f4.re - f3.im * f4.im, bi = f3.re * f4.im + f3.im * f4.re;
                    S[j1 * nd + j2] += ar * br - ai * bi;
                    A[j1 * nd + j2] += hypot(f1.re, f1.im) * hypot(f2.re, f2.im) * hypot(f3.re, f3.im) *
                                       hypot(f4.re, f4.im);
                }
            }
        }
    }
}

int orc_trispectrum_full(int N, const double* delta, int nshell, const double* edges, const int32_t* k, int ndiag,
                         const double* dedges, double* S, double* A, int64_t* counts) {
    if (N < 2 || ndiag < 1 || !k) return fail(-1, "orc_trispectrum_full: bad args");
    for (int t = 0; t < 4; t++)
        if (k[t] < 1 || k[t] > nshell) return fail(-1, "orc_trispectrum_full: bin shell out of range");
    for (int j = 0; j < ndiag; j++)
        if (!(dedges[j] >= 0.0 && dedges[j + 1] > dedges[j])) return fail(-1, "orc_trispectrum_full: diagonal edges");
    const size_t n3 = (size_t)N * N * N;
    tfull_ctx c;
    memset(&c, 0, sizeof c);
    c.N = N;
    c.ndiag = ndiag;
    double* de2 = (double*)malloc(sizeof(double) * (size_t)(ndiag + 1));
    int32_t* smap = (int32_t*)malloc(sizeof(int32_t) * n3);
    double* dhat = delta ? (double*)malloc(sizeof(double) * 2 * n3) : NULL;
    c.S = (double*)calloc((size_t)256 * ndiag * ndiag, sizeof(double));
    c.A = (double*)calloc((size_t)256 * ndiag * ndiag, sizeof(double));
    c.C = (int64_t*)calloc((size_t)256 * ndiag * ndiag, sizeof(int64_t));
    int rc = (!de2 || !smap || (delta && !dhat) || !c.S || !c.A || !c.C) ? fail(-2, "orc_trispectrum_full: out of memory")
                                                                 : orc_shell_map(N, nshell, edges, smap);
    for (int j = 0; j <= ndiag && !rc; j++) de2[j] = dedges[j] * dedges[j];
    if (!rc && delta) rc = orc_forward(N, delta, dhat);
    for (int t = 0; t < 3 && !rc; t++) {
        int32_t cnt = 0;
        for (size_t i = 0; i < n3; i++) cnt += smap[i] == k[t] - 1;
        c.modes[t] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt + 1));
        if (!c.modes[t]) {
            rc = fail(-2, "orc_trispectrum_full: out of memory");
            break;
        }
        c.nm[t] = 0;
        for (size_t i = 0; i < n3; i++)
            if (smap[i] == k[t] - 1) c.modes[t][c.nm[t]++] = (int32_t)i;
    }
    if (!rc) {
        c.de2 = de2;
        c.dhat = (const cplx*)dhat;
        c.smap = smap;
        c.k4 = k[3] - 1;
        par_for(c.nm[0], tfull_range, &c);
        for (int j = 0; j < ndiag * ndiag; j++) {
            double sv = 0.0, av = 0.0;
            int64_t cv = 0;
            for (int t = 0; t < 256; t++) {
                sv += c.S[(size_t)t * ndiag * ndiag + j];
                av += c.A[(size_t)t * ndiag * ndiag + j];
                cv += c.C[(size_t)t * ndiag * ndiag + j];
            }
            if (S) S[j] = (double)n3 * sv;
            if (A) A[j] = (double)n3 * av;
            if (counts) counts[j] = cv;
        }
    }
    for (int t = 0; t < 3; t++) free(c.modes[t]);
    free(de2);
    free(smap);
    free(dhat);
    free(c.S);
    free(c.A);
    free(c.C);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* adjoint of the estimator for L = sum_b g_b B_b (g = dL/dB).                */
/* B_b = c_b S_b with c_b = V^{n-1}/N^{3n} / (N^3 count_b) and               */
/* S_b = sum_x prod_t D_{b_t}(x); D_m = inverse(mask_m * forward(delta)).    */
/*   G_m(x) = dL/dD_m(x) = sum_b g_b c_b sum_{t: b_t = m} prod_{u != t} D_{b_u}(x) */
/*   dL/ddelta(y) = sum_m sum_x G_m(x) K_m(x - y),  K_m(r) = sum_{q in S_m} e^{i q.r} */
/*               = sum_q [sum_m mask_m(q) Ghat_m(q)] e^{+i q.y}               */
/* with Ghat_m(q) = sum_x G_m(x) e^{-i q.x} (K_m is real and even).          */
/* `counts` must be the bins' exact polygon counts.                           */
/* ------------------------------------------------------------------------- */
int orc_gradient(int N, double L, const double* delta, int nshell, const double* edges, int order, int64_t nbins,
                 const int32_t* bins, const int64_t* counts, const double* dLdB, double* grad) {
    if (N < 2 || order < 2 || order > 8) return fail(-1, "orc_gradient: bad args");
    size_t n3 = (size_t)N * N * N;
    int32_t* smap = (int32_t*)malloc(sizeof(int32_t) * n3);
    int rc = orc_shell_map(N, nshell, edges, smap);
    if (rc) return rc;
    int32_t* all = (int32_t*)malloc(sizeof(int32_t) * (size_t)nshell);
    int32_t* slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nshell + 1));
    slot[0] = -1;
    for (int s = 0; s < nshell; s++) {
        all[s] = s;
        slot[s + 1] = s;
    }
    double* dhat = (double*)malloc(sizeof(double) * 2 * n3);
    double* D = (double*)malloc(sizeof(double) * n3 * (size_t)nshell);
    double* G = (double*)calloc(n3 * (size_t)nshell, sizeof(double));
    cplx* H = (cplx*)calloc(n3, sizeof(cplx));
    cplx* work = (cplx*)malloc(sizeof(cplx) * n3);
    if (!dhat || !D || !G || !H || !work) return fail(-2, "orc_gradient: out of memory");
    rc = orc_forward(N, delta, dhat);
    if (!rc) rc = orc_shell_fields(N, dhat, smap, nshell, all, D, NULL);
    if (!rc) {
        double n3d = (double)n3;
        double norm = pow(L * L * L, order - 1) / pow(n3d, order);
        for (int64_t b = 0; b < nbins; b++) {
            if (counts[b] <= 0) continue;
            double w = dLdB[b] * norm / (n3d * (double)counts[b]);
            const int32_t* k = bins + b * order;
            for (int t = 0; t < order; t++) {
                double* g = G + (size_t)(k[t] - 1) * n3;
                for (size_t x = 0; x < n3; x++) {
                    double p = w;
                    for (int u = 0; u < order; u++)
                        if (u != t) p *= D[(size_t)(k[u] - 1) * n3 + x];
                    g[x] += p;
                }
            }
        }
        for (int m = 0; m < nshell && !rc; m++) {
            const double* g = G + (size_t)m * n3;
            for (size_t x = 0; x < n3; x++) {
                work[x].re = g[x];
                work[x].im = 0.0;
            }
            rc = orc_fft3d((double*)work, N, N, N, -1);
            for (size_t q = 0; q < n3 && !rc; q++)
                if (smap[q] == m) H[q] = work[q];
        }
    }
    if (!rc) rc = orc_fft3d((double*)H, N, N, N, +1);
    if (!rc)
        for (size_t x = 0; x < n3; x++) grad[x] = H[x].re;
    free(smap);
    free(all);
    free(slot);
    free(dhat);
    free(D);
    free(G);
    free(H);
    free(work);
    return rc;
}
