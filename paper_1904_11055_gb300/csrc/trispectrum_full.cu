// Full-shape trispectrum T(k1, k2, k3, k4; d1, d2) (Eq. Tkfull, Sec. 2.1).
//
// Besides the four side lengths, a closed quadrilateral q1 + q2 + q3 + q4 = 0
// has two more degrees of freedom; Eq. Tkfull takes them as the diagonals
// p1 = q1 - q2 and p2 = q1 - q3, binned like the shells.  Per pair of diagonal
// bins (j1, j2):
//   T[j1][j2] = c_4 sum Re prod_t dhat(q_t) / count[j1][j2],   c_4 = V^3 / N^12,
// over q_t in S_{k_t} with q1 + q2 + q3 + q4 = 0 (mod N), d_{j} <= |p| < d_{j+1};
// count[j1][j2] is the number of those quadrilaterals.  Summed over diagonal
// bins that cover every |p|, sums and counts are the angle-averaged
// trispectrum's (Eq. estimator at n = 4).  The paper leaves this estimator as
// future work; it names the double convolution of Eq. Tkfull.  Here the sum is
// taken on the Fourier side over the mode lists of S_{k1}, S_{k2}, S_{k3}, with
// q4 = -(q1 + q2 + q3) reduced to the grid's signed representatives and tested
// against S_{k4}.
//
// Work split: one block per (q1, run of 256 q2); a thread owns one q2, so d1 is
// fixed per thread.  The q3 list is staged through shared memory in tiles,
// each tile counting-sorted by d2's bin (d2 depends on q1 and q3 only, so the
// sort is shared by the block); a thread then sums Re prod_t dhat over one
// d2 bin at a time in registers and adds the sum to the (d1, d2) accumulator
// once per bin and tile.  Accumulators are FP64 (block-local in shared memory
// up to 32 diagonal bins, else global); products and per-bin sums are in the
// plan's precision.  Which q3 of a bin a thread visits first depends on
// shared-memory atomics, so the rounding (not the counts) can differ between
// runs.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "plan_internal.h"

namespace ps {

constexpr int kTfThreads = 256;
constexpr int kTfTile = 1024;      // q3 entries per shared-memory tile
constexpr int kTfSmemDiag = 32;    // block-local accumulators up to this many diagonal bins
constexpr int kTfMaxDiag = 128;

struct TfArgs {
    const int4* m1;  // mode lists (x, y, z, |q|^2) of S_{k1}, S_{k2}, S_{k3}
    const int4* m2;
    const int4* m3;
    int n2, n3;
    const short* dl;  // |p|^2 -> diagonal bin, -1 outside every bin; 12 K^2 + 1 entries
    int nd;
    int a4, w4;       // q4 in S_{k4} iff a4 <= |q4|^2 < a4 + w4
    int N, K, hi;     // signed representatives run [hi - N + 1, hi]
    double* S;        // [nd * nd] sum Re prod dhat
    double* A;        // [nd * nd] sum prod |dhat| (SCALE)
    unsigned long long* C;  // [nd * nd] counts
};

PS_DEV Cx<float> ldg_cx(const Cx<float>* p) {
    const float2 v = __ldg((const float2*)p);
    return cx<float>(v.x, v.y);
}
PS_DEV Cx<double> ldg_cx(const Cx<double>* p) {
    const double2 v = __ldg((const double2*)p);
    return cx<double>(v.x, v.y);
}

// dhat(q) from the pruned half spectrum (kz >= 0; the kz = 0 plane is stored whole).
template <typename T>
PS_DEV Cx<T> mode_value(const Cx<T>* __restrict__ fhat, int K, int x, int y, int z) {
    const bool cj = z < 0;
    if (cj) {
        x = -x;
        y = -y;
        z = -z;
    }
    Cx<T> v = ldg_cx(&fhat[((size_t)(y + K) * (K + 1) + z) * (2 * K + 1) + (x + K)]);
    if (cj) v.im = -v.im;
    return v;
}

PS_DEV int signed_rep(int v, int N, int hi) { return v > hi ? v - N : (v < hi - N + 1 ? v + N : v); }

PS_DEV int sq3(int x, int y, int z) { return x * x + y * y + z * z; }

template <typename T, bool WRAP, bool PROD, bool SCALE>
__global__ void __launch_bounds__(kTfThreads) tfull_kernel(const Cx<T>* __restrict__ fhat, TfArgs a) {
    extern __shared__ __align__(16) unsigned char tf_smem[];
    int4* sq = (int4*)tf_smem;                                   // [kTfTile] sorted q3
    Cx<T>* sf = (Cx<T>*)(sq + kTfTile);                          // [kTfTile] dhat(q3)       (PROD)
    T* smag = (T*)(sf + (PROD ? kTfTile : 0));                   // [kTfTile] |dhat(q3)|     (SCALE)
    short* skey = (short*)(smag + (SCALE ? kTfTile : 0));        // [kTfTile] d2 bin
    short* spos = skey + kTfTile;                                // [kTfTile] rank in its bin
    int* soff = (int*)(spos + kTfTile);                          // [kTfMaxDiag + 1] bin offsets / histogram
    double* accS = (double*)(soff + kTfMaxDiag + 2);             // [nd * nd] block-local (nd <= kTfSmemDiag)
    double* accA = accS + kTfSmemDiag * kTfSmemDiag;
    unsigned long long* accC = (unsigned long long*)(accA + kTfSmemDiag * kTfSmemDiag);

    const int nd = a.nd, tid = threadIdx.x;
    const bool local = nd <= kTfSmemDiag;
    if (local) {
        for (int j = tid; j < nd * nd; j += kTfThreads) {
            accS[j] = 0.0;
            accA[j] = 0.0;
            accC[j] = 0ull;
        }
    } else {
        accS = a.S;
        accA = a.A;
        accC = a.C;
    }

    const int4 q1 = a.m1[blockIdx.x];
    const int i2 = blockIdx.y * kTfThreads + tid;
    int j1 = -1, nsx = 0, nsy = 0, nsz = 0;
    T ar = 0, ai = 0, am = 0;
    if (i2 < a.n2) {
        const int4 q2 = a.m2[i2];
        j1 = a.dl[sq3(q1.x - q2.x, q1.y - q2.y, q1.z - q2.z)];
        nsx = -(q1.x + q2.x);
        nsy = -(q1.y + q2.y);
        nsz = -(q1.z + q2.z);
        if (PROD) {
            const Cx<T> f1 = mode_value(fhat, a.K, q1.x, q1.y, q1.z), f2 = mode_value(fhat, a.K, q2.x, q2.y, q2.z);
            ar = f1.re * f2.re - f1.im * f2.im;
            ai = f1.re * f2.im + f1.im * f2.re;
            if (SCALE) am = sqrt(ar * ar + ai * ai);
        }
    }
    const bool active = j1 >= 0;

    for (int t0 = 0; t0 < a.n3; t0 += kTfTile) {
        const int nt = min(kTfTile, a.n3 - t0);
        __syncthreads();  // the previous tile's readers are done with soff, sq, sf, smag
        for (int j = tid; j <= nd; j += kTfThreads) soff[j] = 0;
        __syncthreads();
        for (int e = tid; e < nt; e += kTfThreads) {
            const int4 q3 = a.m3[t0 + e];
            const int j2 = a.dl[sq3(q1.x - q3.x, q1.y - q3.y, q1.z - q3.z)];
            skey[e] = (short)j2;
            if (j2 >= 0) spos[e] = (short)atomicAdd(&soff[j2 + 1], 1);
        }
        __syncthreads();
        if (tid == 0)
            for (int j = 1; j <= nd; j++) soff[j] += soff[j - 1];
        __syncthreads();
        for (int e = tid; e < nt; e += kTfThreads) {
            const int j2 = skey[e];
            if (j2 < 0) continue;
            const int d = soff[j2] + spos[e];
            const int4 q3 = a.m3[t0 + e];
            sq[d] = q3;
            if (PROD) {
                const Cx<T> f3 = mode_value(fhat, a.K, q3.x, q3.y, q3.z);
                sf[d] = f3;
                if (SCALE) smag[d] = sqrt(f3.re * f3.re + f3.im * f3.im);
            }
        }
        __syncthreads();
        if (active) {
            for (int g = 0; g < nd; g++) {
                const int beg = soff[g], end = soff[g + 1];
                if (beg == end) continue;
                T acc = 0, acca = 0;
                unsigned cnt = 0;
                for (int e = beg; e < end; e++) {
                    const int4 q3 = sq[e];
                    int vx = nsx - q3.x, vy = nsy - q3.y, vz = nsz - q3.z;
                    if (WRAP) {
                        vx = signed_rep(vx, a.N, a.hi);
                        vy = signed_rep(vy, a.N, a.hi);
                        vz = signed_rep(vz, a.N, a.hi);
                    }
                    if ((unsigned)(sq3(vx, vy, vz) - a.a4) < (unsigned)a.w4) {
                        cnt++;
                        if (PROD) {
                            // |q4| < the outer shell edge, so every component lies in [-K, K]
                            const Cx<T> f4 = mode_value(fhat, a.K, vx, vy, vz), f3 = sf[e];
                            const T br = f3.re * f4.re - f3.im * f4.im, bi = f3.re * f4.im + f3.im * f4.re;
                            acc += ar * br - ai * bi;
                            if (SCALE) acca += am * smag[e] * sqrt(f4.re * f4.re + f4.im * f4.im);
                        }
                    }
                }
                if (cnt) {
                    const int j = j1 * nd + g;
                    atomicAdd(&accC[j], (unsigned long long)cnt);
                    if (PROD) atomicAdd(&accS[j], (double)acc);
                    if (SCALE) atomicAdd(&accA[j], (double)acca);
                }
            }
        }
    }
    if (local) {
        __syncthreads();
        for (int j = tid; j < nd * nd; j += kTfThreads) {
            if (accC[j] == 0ull) continue;
            atomicAdd(&a.C[j], accC[j]);
            if (PROD) atomicAdd(&a.S[j], accS[j]);
            if (SCALE) atomicAdd(&a.A[j], accA[j]);
        }
    }
}

__global__ void tfull_finish_kernel(const double* __restrict__ S, const double* __restrict__ A,
                                    const unsigned long long* __restrict__ C, int n, double norm, double* T,
                                    double* scale, int64_t* counts) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const unsigned long long c = C[j];
        if (T) T[j] = c ? norm * S[j] / (double)c : 0.0;
        if (scale) scale[j] = c ? norm * A[j] / (double)c : 0.0;
        if (counts) counts[j] = (int64_t)c;
    }
}

static size_t tfull_smem_bytes(int es, bool prod, bool scale) {
    return (size_t)kTfTile * (sizeof(int4) + (prod ? 2 * es : 0) + (scale ? es : 0) + 2 * sizeof(short)) +
           (kTfMaxDiag + 2) * sizeof(int) + (size_t)kTfSmemDiag * kTfSmemDiag * 3 * sizeof(double);
}

template <typename T, bool WRAP, bool PROD, bool SCALE>
static cudaError_t launch_tfull(const void* fhat, const TfArgs& a, int n1, cudaStream_t st) {
    const size_t smem = tfull_smem_bytes((int)sizeof(T), PROD, SCALE);
    auto k = tfull_kernel<T, WRAP, PROD, SCALE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    const dim3 grid((unsigned)n1, (unsigned)((a.n2 + kTfThreads - 1) / kTfThreads));
    k<<<grid, kTfThreads, smem, st>>>((const Cx<T>*)fhat, a);
    return cudaGetLastError();
}

template <typename T, bool WRAP>
static cudaError_t launch_tfull_p(const void* fhat, const TfArgs& a, int n1, bool prod, bool scale, cudaStream_t st) {
    if (!prod) return launch_tfull<T, WRAP, false, false>(fhat, a, n1, st);
    return scale ? launch_tfull<T, WRAP, true, true>(fhat, a, n1, st) : launch_tfull<T, WRAP, true, false>(fhat, a, n1, st);
}

}  // namespace ps

using namespace ps;

// Host side.  Mode lists, the diagonal-bin table and the q4 test use the same
// FP64 comparisons of integer |q|^2 against squared edges as the shell tables:
// e_lo^2 <= |q|^2 < e_hi^2.
namespace {

poly_status fail(poly_status s, const std::string& msg) {
    ps_set_last_error(msg);
    return s;
}

void shell_modes(int K, double lo, double hi, std::vector<int4>& out) {
    out.clear();
    const double lo2 = lo * lo, hi2 = hi * hi;
    for (int x = -K; x <= K; x++)
        for (int y = -K; y <= K; y++)
            for (int z = -K; z <= K; z++) {
                const int r = x * x + y * y + z * z;
                if (lo2 <= (double)r && (double)r < hi2) out.push_back(make_int4(x, y, z, r));
            }
}

// smallest integer r >= 0 with (double)r >= e2
int first_at_least(double e2) {
    if (!(e2 > 0.0)) return 0;
    long long r = (long long)std::ceil(e2);
    while (r > 0 && (double)(r - 1) >= e2) r--;
    while ((double)r < e2) r++;
    return (int)std::min<long long>(r, 1 << 30);
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

poly_status ps_trispectrum_full_impl(PsPlan* p, const void* delta, const int32_t* k, int nd, const double* dedges,
                                     double* T_out, int64_t* counts_out, double* scale_out, cudaStream_t st) {
    if (!k || !dedges) return fail(POLY_ERR_ARG, "NULL argument");
    if (!T_out && !counts_out && !scale_out) return fail(POLY_ERR_ARG, "no output requested");
    if (!delta && (T_out || scale_out)) return fail(POLY_ERR_ARG, "T and scale need delta_x (NULL: counts only)");
    if (nd < 1 || nd > kTfMaxDiag) return fail(POLY_ERR_ARG, "ndiag must be in [1, 128]");
    for (int t = 0; t < 4; t++)
        if (k[t] < 1 || k[t] > p->nshell) return fail(POLY_ERR_ARG, "shell index out of [1, nshell]");
    for (int j = 0; j <= nd; j++)
        if (!std::isfinite(dedges[j]) || dedges[j] < 0.0) return fail(POLY_ERR_ARG, "diagonal edges must be finite, >= 0");
    for (int j = 0; j < nd; j++)
        if (!(dedges[j + 1] > dedges[j])) return fail(POLY_ERR_ARG, "diagonal edges must increase strictly");
    const void* outs[3] = {T_out, counts_out, scale_out};
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            if (i != j && outs[i] && outs[i] == outs[j]) return fail(POLY_ERR_ARG, "outputs alias each other");
    for (int i = 0; i < 3; i++)
        if (outs[i] && outs[i] == delta) return fail(POLY_ERR_ARG, "output aliases delta_x");

    const int K = p->K, N = p->N;
    const double* e = p->edges.data();
    std::vector<int4> m[3];
    for (int t = 0; t < 3; t++) shell_modes(K, e[k[t] - 1], e[k[t]], m[t]);
    const double tests = (double)m[0].size() * (double)m[1].size() * (double)m[2].size();
    if (tests > 4.4e12) return fail(POLY_ERR_UNSUPPORTED, "more than 4.4e12 (q1, q2, q3) triples");
    if ((m[1].size() + kTfThreads - 1) / kTfThreads > 65535)
        return fail(POLY_ERR_UNSUPPORTED, "S_k2 holds more than 65535 * 256 modes");
    const int ndl = 12 * K * K + 1;  // |q1 - q2|^2 <= 3 (2K)^2
    std::vector<short> dl(ndl, (short)-1);
    for (int r = 0; r < ndl; r++)
        for (int j = 0; j < nd; j++)
            if (dedges[j] * dedges[j] <= (double)r && (double)r < dedges[j + 1] * dedges[j + 1]) {
                dl[r] = (short)j;
                break;
            }
    const double lo4 = e[k[3] - 1], hi4 = e[k[3]];
    const int a4 = first_at_least(lo4 * lo4), b4 = first_at_least(hi4 * hi4);

    // scratch: lists, diagonal table, accumulators (grown on demand, freed with the plan)
    const size_t nacc = (size_t)nd * nd;
    size_t off_m[3], off_dl, off_S, off_A, off_C, bytes = 0;
    for (int t = 0; t < 3; t++) {
        off_m[t] = bytes;
        bytes = align256(bytes + std::max<size_t>(m[t].size(), 1) * sizeof(int4));
    }
    off_dl = bytes;
    bytes = align256(bytes + dl.size() * sizeof(short));
    off_S = bytes;
    bytes = align256(bytes + nacc * sizeof(double));
    off_A = bytes;
    bytes = align256(bytes + nacc * sizeof(double));
    off_C = bytes;
    bytes = align256(bytes + nacc * sizeof(unsigned long long));
    if (bytes > p->tf_bytes) {
        ps_free(p, p->d_tf);
        p->d_tf = nullptr;
        p->tf_bytes = 0;
        void* d = nullptr;
        poly_status s = ps_alloc(p, &d, bytes);
        if (s) return s;
        p->d_tf = d;
        p->tf_bytes = bytes;
    }
    unsigned char* B = (unsigned char*)p->d_tf;
    cudaError_t ce;
    for (int t = 0; t < 3; t++)
        if (!m[t].empty() &&
            (ce = cudaMemcpyAsync(B + off_m[t], m[t].data(), m[t].size() * sizeof(int4), cudaMemcpyHostToDevice, st)))
            return fail(POLY_ERR_CUDA, std::string("mode list upload: ") + cudaGetErrorString(ce));
    if ((ce = cudaMemcpyAsync(B + off_dl, dl.data(), dl.size() * sizeof(short), cudaMemcpyHostToDevice, st)) ||
        (ce = cudaMemsetAsync(B + off_S, 0, bytes - off_S, st)))
        return fail(POLY_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(ce));
    const bool prod = delta != nullptr;
    if (prod && (ce = ps_forward(N, p->is_double, delta, K, p->d_tw_fwd, p->d_W, p->d_fhat, p->d_spill, st)))
        return fail(POLY_ERR_CUDA, std::string("forward transform: ") + cudaGetErrorString(ce));
    p->launches += prod ? 2 : 0;

    TfArgs a;
    a.m1 = (const int4*)(B + off_m[0]);
    a.m2 = (const int4*)(B + off_m[1]);
    a.m3 = (const int4*)(B + off_m[2]);
    a.n2 = (int)m[1].size();
    a.n3 = (int)m[2].size();
    a.dl = (const short*)(B + off_dl);
    a.nd = nd;
    a.a4 = a4;
    a.w4 = std::max(b4 - a4, 0);
    a.N = N;
    a.K = K;
    a.hi = (N - 1) / 2;
    a.S = (double*)(B + off_S);
    a.A = (double*)(B + off_A);
    a.C = (unsigned long long*)(B + off_C);
    // no q_t sum leaves the signed range when 3K <= (N - 1) / 2
    const bool wrap = 3 * K > (N - 1) / 2;
    const bool scale = scale_out != nullptr;
    if (!m[0].empty() && !m[1].empty() && !m[2].empty() && a.w4 > 0) {
        if (p->is_double)
            ce = wrap ? launch_tfull_p<double, true>(p->d_fhat, a, (int)m[0].size(), prod, scale, st)
                      : launch_tfull_p<double, false>(p->d_fhat, a, (int)m[0].size(), prod, scale, st);
        else
            ce = wrap ? launch_tfull_p<float, true>(p->d_fhat, a, (int)m[0].size(), prod, scale, st)
                      : launch_tfull_p<float, false>(p->d_fhat, a, (int)m[0].size(), prod, scale, st);
        if (ce) return fail(POLY_ERR_CUDA, std::string("full-shape trispectrum kernel: ") + cudaGetErrorString(ce));
        p->launches++;
    }
    const double n3 = (double)N * N * N, V = p->L * p->L * p->L;
    const double norm = V * V * V / (n3 * n3 * n3 * n3);
    tfull_finish_kernel<<<(int)((nacc + 255) / 256), 256, 0, st>>>(a.S, a.A, a.C, (int)nacc, norm, T_out, scale_out,
                                                                   counts_out);
    if ((ce = cudaGetLastError())) return fail(POLY_ERR_CUDA, std::string("finish kernel: ") + cudaGetErrorString(ce));
    p->launches++;
    return POLY_OK;
}
