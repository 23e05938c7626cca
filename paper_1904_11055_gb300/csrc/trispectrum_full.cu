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
// future work.  Each of its two diagonal constraints ties q1 to another leg, so
// no Gram of diagonal-filtered fields separates them; the sum is taken on the
// Fourier side instead, visiting closed quadrilaterals only:
//   1. the pairs (q1, q2) in S_k1 x S_k2 whose first diagonal falls in a bin, and
//      the pairs (q3, q4) in S_k3 x S_k4, are counting-sorted by the sum
//      s = q1 + q2 and by -(q3 + q4), taken mod N (a quadrilateral closes iff the
//      two keys agree);
//   2. a persistent kernel takes work items (one key, up to 256 of its (q1, q2)
//      pairs); a thread holds one pair, dhat(q1) dhat(q2) and its first
//      diagonal's bin, and walks the key's (q3, q4) pairs, staged through shared
//      memory with dhat(q3) dhat(q4) precomputed, binning each by |q1 - q3|.
// Sums and counts of one work item are added into per-item tables in shared
// memory (in the plan's precision, with shared-memory atomics), folded into
// FP64 block tables after the item and into FP64 global sums at the end.  The
// pairs' order inside a key comes from atomics, so the rounding (not the
// counts) can differ between runs.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "plan_internal.h"

namespace ps {

constexpr int kTfThreads = 256;
constexpr int kTfItem = 32;         // (q1, q2) pairs per work item: one warp, one pair per lane
constexpr int kTfMaxDiag = 128;
constexpr int kTfSmemDl = 16384;    // diagonal-bin table entries held in shared memory
constexpr int kTfScan = 1024;       // elements per block of the key scan

// One pair: the first mode's components and a diagonal bin (q1 and j1 for (q1, q2); q3 for (q3, q4)) in
// four signed bytes, the product of the two modes' dhat and its modulus.
template <typename T>
struct alignas(2 * sizeof(T)) TfPair {
    char4 q;
    T m;
    Cx<T> v;
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

PS_DEV int sq3(int x, int y, int z) { return x * x + y * y + z * z; }

struct TfKeys {
    int side, off, N;  // side = 4K + 1 (components + 2K) when no sum wraps, else N (components mod N)
    PS_DEV int operator()(int x, int y, int z) const {
        if (side == N) {
            x = ((x % N) + N) % N;
            y = ((y % N) + N) % N;
            z = ((z % N) + N) % N;
        } else {
            x += off;
            y += off;
            z += off;
        }
        return (x * side + y) * side + z;
    }
};

// Pairs of two mode lists: FIRST = (q1, q2) (kept when the diagonal q1 - q2 is in a bin; key q1 + q2), else
// (q3, q4) (key -(q3 + q4)).  cursor == NULL: histogram of the keys; else scatter at the cursors.
template <typename T, bool FIRST, bool PROD>
__global__ void __launch_bounds__(kTfThreads) tf_pairs_kernel(const int4* __restrict__ ma, const int4* __restrict__ mb,
                                                              int nb, long long npairs, const short* __restrict__ dl,
                                                              TfKeys key, int* __restrict__ hist, int* cursor,
                                                              TfPair<T>* __restrict__ out,
                                                              const Cx<T>* __restrict__ fhat, int K) {
    const long long idx = (long long)blockIdx.x * kTfThreads + threadIdx.x;
    if (idx >= npairs) return;
    const int ia = (int)(idx / nb), ib = (int)(idx - (long long)ia * nb);
    const int4 qa = ma[ia], qb = mb[ib];
    int j = 0, kk;
    if (FIRST) {
        j = dl[sq3(qa.x - qb.x, qa.y - qb.y, qa.z - qb.z)];
        if (j < 0) return;
        kk = key(qa.x + qb.x, qa.y + qb.y, qa.z + qb.z);
    } else {
        kk = key(-(qa.x + qb.x), -(qa.y + qb.y), -(qa.z + qb.z));
    }
    if (!cursor) {
        atomicAdd(&hist[kk], 1);
        return;
    }
    const int pos = atomicAdd(&cursor[kk], 1);
    TfPair<T> e;
    e.q = make_char4((signed char)qa.x, (signed char)qa.y, (signed char)qa.z, (signed char)j);
    e.m = 0;
    e.v = cx<T>(0, 0);
    if (PROD) {
        const Cx<T> fa = mode_value(fhat, K, qa.x, qa.y, qa.z), fb = mode_value(fhat, K, qb.x, qb.y, qb.z);
        e.v = cmul(fa, fb);
        e.m = sqrt(e.v.re * e.v.re + e.v.im * e.v.im);
    }
    out[pos] = e;
}

// Exclusive scan of n ints in three launches: per-block scans (block totals to bsum), a scan of the block
// totals in one block, and the add of each block's offset.
__global__ void __launch_bounds__(kTfScan) tf_scan_blocks_kernel(const int* __restrict__ in, int* __restrict__ out,
                                                                 int n, int* __restrict__ bsum) {
    __shared__ int s_w[kTfScan / 32];
    const int i = blockIdx.x * kTfScan + threadIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = i < n ? in[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < kTfScan / 32 ? s_w[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kTfScan / 32) s_w[lane] = t;
    }
    __syncthreads();
    const int incl = x + (w > 0 ? s_w[w - 1] : 0);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == kTfScan - 1) bsum[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(kTfScan) tf_scan_sums_kernel(int* __restrict__ bsum, int nb) {
    __shared__ int s_w[kTfScan / 32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b0 = 0; b0 < nb; b0 += kTfScan) {
        const int i = b0 + threadIdx.x;
        const int v = i < nb ? bsum[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[w] = x;
        __syncthreads();
        if (w == 0) {
            int t = lane < kTfScan / 32 ? s_w[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < kTfScan / 32) s_w[lane] = t;
        }
        __syncthreads();
        const int incl = x + (w > 0 ? s_w[w - 1] : 0) + s_carry;
        if (i < nb) bsum[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == kTfScan - 1) s_carry = incl;
        __syncthreads();
    }
}

__global__ void tf_scan_add_kernel(int* __restrict__ out, int* __restrict__ cursor, int n,
                                   const int* __restrict__ bsum) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int v = out[i] + bsum[i / kTfScan];
    out[i] = v;
    cursor[i] = v;
}

// Work items: (key, run of kTfItem (q1, q2) pairs) for every key that has pairs on both sides.
__global__ void tf_items_kernel(const int* __restrict__ h12, const int* __restrict__ h34, int nkeys,
                                int2* __restrict__ items, int* __restrict__ nitems) {
    const int kk = blockIdx.x * blockDim.x + threadIdx.x;
    if (kk >= nkeys || h12[kk] == 0 || h34[kk] == 0) return;
    const int nit = (h12[kk] + kTfItem - 1) / kTfItem;
    const int base = atomicAdd(nitems, nit);
    for (int c = 0; c < nit; c++) items[base + c] = make_int2(kk, c);
}

struct TfQuadArgs {
    const int2* items;
    const int* nitems;
    int* next;
    const int *h12, *o12, *h34, *o34;
    const short* dl;
    int ndl_smem;  // entries of dl copied to shared memory (0: read from global)
    int nd;
    int local;  // per-lane columns and block tables in shared memory (else global atomics per quadrilateral)
    double* S;
    double* A;
    unsigned long long* C;
};

// Shared-memory layout of the quadrilateral kernel (byte offsets): per warp a buffer of 32 (q3, q4) pairs;
// with per-lane tables (`local`, when they fit): FP64 block sums and counts [nd^2], and per-lane columns of
// one work item's sums and counts [nd][kTfThreads]; then the diagonal-bin table.
struct TfQuadLayout {
    size_t bS, bA, bC, colS, colA, colC, dl, total;
};
PS_HD TfQuadLayout tf_quad_layout(int nd, bool local, int es, int pair_bytes, bool scale, int ndl_smem) {
    TfQuadLayout L;
    const size_t ncell = local ? (size_t)nd * nd : 0, ncol = local ? (size_t)nd * kTfThreads : 0;
    size_t o = (size_t)kTfThreads * pair_bytes;
    L.bS = o;
    o += ncell * 8;
    L.bA = o;
    o += scale ? ncell * 8 : 0;
    L.bC = o;
    o += ncell * 8;
    L.colS = o;
    o += ncol * es;
    L.colA = o;
    o += scale ? ncol * es : 0;
    L.colC = o;
    o += ncol * 4;
    L.dl = o;
    o += (size_t)ndl_smem * 2;
    L.total = (o + 15) / 16 * 16;
    return L;
}

// One warp per work item: its lanes hold the item's (q1, q2) pairs, sorted by the first diagonal's bin so that
// lanes of one bin are contiguous; the key's (q3, q4) pairs pass through the warp's buffer 32 at a time, and
// each lane adds Re dhat(q1)dhat(q2)dhat(q3)dhat(q4) to its own column at the second diagonal's bin (no
// atomics).  After the item the columns are reduced over each run of lanes of one first-diagonal bin and added
// to the block's FP64 table.
template <typename T, bool PROD, bool SCALE>
__global__ void __launch_bounds__(kTfThreads, 2) tf_quad_kernel(const TfPair<T>* __restrict__ p12,
                                                                const TfPair<T>* __restrict__ p34, TfQuadArgs a) {
    extern __shared__ __align__(16) unsigned char tf_smem[];
    constexpr unsigned kFull = 0xffffffffu;
    const int nd = a.nd, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool local = a.local != 0;
    const TfQuadLayout Lq = tf_quad_layout(nd, local, (int)sizeof(T), (int)sizeof(TfPair<T>), SCALE, a.ndl_smem);
    TfPair<T>* wb = (TfPair<T>*)tf_smem + warp * 32;
    double* bS = (double*)(tf_smem + Lq.bS);
    double* bA = (double*)(tf_smem + Lq.bA);
    unsigned long long* bC = (unsigned long long*)(tf_smem + Lq.bC);
    T* colS = (T*)(tf_smem + Lq.colS);
    T* colA = (T*)(tf_smem + Lq.colA);
    unsigned* colC = (unsigned*)(tf_smem + Lq.colC);
    short* sdl = (short*)(tf_smem + Lq.dl);
    const int ncell = local ? nd * nd : 0;
    for (int j = tid; j < ncell; j += kTfThreads) {
        bS[j] = 0.0;
        if (SCALE) bA[j] = 0.0;
        bC[j] = 0ull;
    }
    for (int j = tid; local && j < nd * kTfThreads; j += kTfThreads) {
        colS[j] = 0;
        if (SCALE) colA[j] = 0;
        colC[j] = 0u;
    }
    for (int j = tid; j < a.ndl_smem; j += kTfThreads) sdl[j] = a.dl[j];
    const short* dl = a.ndl_smem > 0 ? sdl : a.dl;
    __syncthreads();
    const int nitems = *a.nitems;
    while (true) {
        int it = 0;
        if (lane == 0) it = atomicAdd(a.next, 1);
        it = __shfl_sync(kFull, it, 0);
        if (it >= nitems) break;
        const int2 item = a.items[it];
        const int kk = item.x;
        const int n12 = min(kTfItem, a.h12[kk] - item.y * kTfItem);
        TfPair<T> mine;
        mine.q = make_char4(0, 0, 0, 0);
        mine.m = 0;
        mine.v = cx<T>(0, 0);
        if (lane < n12) mine = p12[a.o12[kk] + item.y * kTfItem + lane];
        // bitonic sort of the lanes by (first-diagonal bin, lane); lanes without a pair go last
        int key = ((lane < n12 ? (int)mine.q.w : 255) << 5) | lane;
        for (int k2 = 2; k2 <= 32; k2 <<= 1)
            for (int j = k2 >> 1; j > 0; j >>= 1) {
                const int other = __shfl_xor_sync(kFull, key, j);
                key = (((lane & j) == 0) == ((lane & k2) == 0)) ? min(key, other) : max(key, other);
            }
        const int src = key & 31;
        const bool active = src < n12;
        int qw;
        memcpy(&qw, &mine.q, 4);
        qw = __shfl_sync(kFull, qw, src);
        char4 q1;
        memcpy(&q1, &qw, 4);
        const T ar = __shfl_sync(kFull, mine.v.re, src), ai = __shfl_sync(kFull, mine.v.im, src);
        const T am = __shfl_sync(kFull, mine.m, src);
        const int j1 = active ? (int)q1.w : -1;
        const int b34 = a.o34[kk], n34 = a.h34[kk];
        for (int c0 = 0; c0 < n34; c0 += 32) {
            const int nc = min(32, n34 - c0);
            __syncwarp();
            if (lane < nc) wb[lane] = p34[b34 + c0 + lane];
            __syncwarp();
            if (!active) continue;
            for (int e = 0; e < nc; e++) {
                const TfPair<T> f = wb[e];
                const int j2 = dl[sq3(q1.x - f.q.x, q1.y - f.q.y, q1.z - f.q.z)];
                if (j2 < 0) continue;
                if (local) {
                    const int c = j2 * kTfThreads + tid;
                    colC[c] += 1u;
                    if (PROD) colS[c] += ar * f.v.re - ai * f.v.im;
                    if (SCALE) colA[c] += am * f.m;
                } else {
                    const int cell = j1 * nd + j2;
                    atomicAdd(&a.C[cell], 1ull);
                    if (PROD) atomicAdd(&a.S[cell], (double)(ar * f.v.re - ai * f.v.im));
                    if (SCALE) atomicAdd(&a.A[cell], (double)(am * f.m));
                }
            }
        }
        if (!local) continue;
        // reduce each column over the run of lanes with this lane's first-diagonal bin; the run's first lane
        // adds the sums to the block table
        const int jprev = __shfl_up_sync(kFull, j1, 1);  // every lane takes part in the shuffle
        const bool head = lane == 0 || jprev != j1;
        for (int j2 = 0; j2 < nd; j2++) {
            const int c = j2 * kTfThreads + tid;
            unsigned cn = colC[c];
            if (__ballot_sync(kFull, cn != 0u) == 0u) continue;
            T sv = 0, av = 0;
            if (PROD) {
                sv = colS[c];
                colS[c] = 0;
            }
            if (SCALE) {
                av = colA[c];
                colA[c] = 0;
            }
            colC[c] = 0u;
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned oc = __shfl_down_sync(kFull, cn, off);
                const T os = __shfl_down_sync(kFull, sv, off), oa = __shfl_down_sync(kFull, av, off);
                const int oj = __shfl_down_sync(kFull, j1, off);
                if (lane + off < 32 && oj == j1) {
                    cn += oc;
                    sv += os;
                    av += oa;
                }
            }
            if (head && j1 >= 0 && cn) {
                const int cell = j1 * nd + j2;
                atomicAdd(&bC[cell], (unsigned long long)cn);
                if (PROD) atomicAdd(&bS[cell], (double)sv);
                if (SCALE) atomicAdd(&bA[cell], (double)av);
            }
        }
    }
    __syncthreads();
    for (int j = tid; j < ncell; j += kTfThreads) {
        if (bC[j] == 0ull) continue;
        atomicAdd(&a.C[j], bC[j]);
        if (PROD) atomicAdd(&a.S[j], bS[j]);
        if (SCALE) atomicAdd(&a.A[j], bA[j]);
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

template <typename T, bool PROD, bool SCALE>
static cudaError_t launch_quads(const void* p12, const void* p34, const TfQuadArgs& a, int sms, cudaStream_t st,
                                int* blocks_out) {
    auto k = tf_quad_kernel<T, PROD, SCALE>;
    TfQuadArgs b = a;
    // per-lane tables when they fit next to the buffers (about 48 diagonal bins in FP32)
    b.local = tf_quad_layout(a.nd, true, (int)sizeof(T), (int)sizeof(TfPair<T>), SCALE, a.ndl_smem).total <=
              200 * 1024;
    const size_t smem = tf_quad_layout(a.nd, b.local != 0, (int)sizeof(T), (int)sizeof(TfPair<T>), SCALE,
                                       a.ndl_smem).total;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTfThreads, smem))) return e;
    const int blocks = sms * std::max(1, per_sm);
    k<<<blocks, kTfThreads, smem, st>>>((const TfPair<T>*)p12, (const TfPair<T>*)p34, b);
    *blocks_out = blocks;
    return cudaGetLastError();
}

template <typename T, bool PROD>
static cudaError_t launch_pairs(bool first, const int4* ma, const int4* mb, int na, int nb, const short* dl,
                                TfKeys key, int* hist, int* cursor, void* out, const void* fhat, int K,
                                cudaStream_t st) {
    const long long np = (long long)na * nb;
    if (np == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((np + kTfThreads - 1) / kTfThreads);
    if (first)
        tf_pairs_kernel<T, true, PROD><<<blocks, kTfThreads, 0, st>>>(ma, mb, nb, np, dl, key, hist, cursor,
                                                                        (TfPair<T>*)out, (const Cx<T>*)fhat, K);
    else
        tf_pairs_kernel<T, false, PROD><<<blocks, kTfThreads, 0, st>>>(ma, mb, nb, np, dl, key, hist, cursor,
                                                                         (TfPair<T>*)out, (const Cx<T>*)fhat, K);
    return cudaGetLastError();
}

static cudaError_t scan_keys(const int* h, int* o, int* cursor, int n, int* bsum, cudaStream_t st) {
    const int nb = (n + kTfScan - 1) / kTfScan;
    tf_scan_blocks_kernel<<<nb, kTfScan, 0, st>>>(h, o, n, bsum);
    tf_scan_sums_kernel<<<1, kTfScan, 0, st>>>(bsum, nb);
    tf_scan_add_kernel<<<(n + 255) / 256, 256, 0, st>>>(o, cursor, n, bsum);
    return cudaGetLastError();
}

}  // namespace ps

using namespace ps;

// Host side.  Mode lists and the diagonal-bin table use the same FP64 comparisons of integer |q|^2
// against squared edges as the shell tables: e_lo^2 <= |q|^2 < e_hi^2.
namespace {

poly_status fail(poly_status s, const std::string& msg) {
    ps_set_last_error(msg);
    return s;
}

// largest |component| of a mode of a shell with outer edge hi: the largest integer c with c^2 < hi^2
int shell_kmax(double hi) {
    int c = 0;
    while ((double)((long long)(c + 1) * (c + 1)) < hi * hi) c++;
    return c;
}

// the shell's modes, scanned over the cube that holds them (|q_c| <= the shell's largest component, <= K)
void shell_modes(int K, double lo, double hi, std::vector<int4>& out) {
    out.clear();
    const double lo2 = lo * lo, hi2 = hi * hi;
    const int c = std::min(K, shell_kmax(hi));
    for (int x = -c; x <= c; x++)
        for (int y = -c; y <= c; y++)
            for (int z = -c; z <= c; z++) {
                const int r = x * x + y * y + z * z;
                if (lo2 <= (double)r && (double)r < hi2) out.push_back(make_int4(x, y, z, r));
            }
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
    std::vector<int4> m[4];
    int kmax[4];
    for (int t = 0; t < 4; t++) {
        shell_modes(K, e[k[t] - 1], e[k[t]], m[t]);
        kmax[t] = shell_kmax(e[k[t]]);
    }
    const long long np12 = (long long)m[0].size() * (long long)m[1].size();
    const long long np34 = (long long)m[2].size() * (long long)m[3].size();
    if (np12 > (1LL << 29) || np34 > (1LL << 29))
        return fail(POLY_ERR_UNSUPPORTED, "more than 2^29 pairs of modes on one side");
    // diagonal bins of |p|^2 <= 3 (2K)^2
    const int ndl = 12 * K * K + 1;
    std::vector<short> dl(ndl, (short)-1);
    for (int r = 0; r < ndl; r++)
        for (int j = 0; j < nd; j++)
            if (dedges[j] * dedges[j] <= (double)r && (double)r < dedges[j + 1] * dedges[j + 1]) {
                dl[r] = (short)j;
                break;
            }
    // |q1 - q3| < e_hi(k1) + e_hi(k3): the entries the quadrilateral kernel can read
    const double r13 = e[k[0]] + e[k[2]];
    const long long need = std::min<long long>(ndl, (long long)std::floor(r13 * r13) + 1);
    const int ndl_smem = need <= kTfSmemDl ? (int)need : 0;
    // keys: the pair sums' components lie in [-R, R]; without a wrap (the four legs' largest components
    // sum below N) a quadrilateral closes iff q1 + q2 = -(q3 + q4) exactly, else iff they agree mod N
    const int R = std::max(kmax[0] + kmax[1], kmax[2] + kmax[3]);
    TfKeys key;
    key.N = N;
    key.off = R;
    key.side = kmax[0] + kmax[1] + kmax[2] + kmax[3] < N ? std::min(2 * R + 1, N) : N;
    if (key.side == 2 * R + 1 && 2 * R + 1 > N) key.side = N;  // unreachable: 2R < N whenever no sum wraps
    const long long nkeys = (long long)key.side * key.side * key.side;
    const size_t es = p->is_double ? 8 : 4, pair_bytes = p->is_double ? sizeof(TfPair<double>) : sizeof(TfPair<float>);
    const long long cap_items = np12 / kTfItem + nkeys + 1;
    const int nbs = (int)((nkeys + kTfScan - 1) / kTfScan);
    (void)es;

    // scratch (grown on demand, freed with the plan)
    const size_t nacc = (size_t)nd * nd;
    size_t off_m[4], off_dl, off_h[6], off_bs, off_p12, off_p34, off_it, off_cnt, off_S, off_A, off_C, bytes = 0;
    for (int t = 0; t < 4; t++) {
        off_m[t] = bytes;
        bytes = align256(bytes + std::max<size_t>(m[t].size(), 1) * sizeof(int4));
    }
    off_dl = bytes;
    bytes = align256(bytes + dl.size() * sizeof(short));
    for (int i = 0; i < 6; i++) {  // h12, h34, o12, o34, c12, c34
        off_h[i] = bytes;
        bytes = align256(bytes + (size_t)nkeys * sizeof(int));
    }
    off_bs = bytes;
    bytes = align256(bytes + (size_t)std::max(nbs, 1) * sizeof(int));
    off_p12 = bytes;
    bytes = align256(bytes + (size_t)std::max<long long>(np12, 1) * pair_bytes);
    off_p34 = bytes;
    bytes = align256(bytes + (size_t)std::max<long long>(np34, 1) * pair_bytes);
    off_it = bytes;
    bytes = align256(bytes + (size_t)cap_items * sizeof(int2));
    off_cnt = bytes;
    bytes = align256(bytes + 2 * sizeof(int));
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
    int* h12 = (int*)(B + off_h[0]);
    int* h34 = (int*)(B + off_h[1]);
    int* o12 = (int*)(B + off_h[2]);
    int* o34 = (int*)(B + off_h[3]);
    int* c12 = (int*)(B + off_h[4]);
    int* c34 = (int*)(B + off_h[5]);
    int* cnt = (int*)(B + off_cnt);  // [0] work items, [1] next item
    cudaError_t ce;
    for (int t = 0; t < 4; t++)
        if (!m[t].empty() &&
            (ce = cudaMemcpyAsync(B + off_m[t], m[t].data(), m[t].size() * sizeof(int4), cudaMemcpyHostToDevice, st)))
            return fail(POLY_ERR_CUDA, std::string("mode list upload: ") + cudaGetErrorString(ce));
    if ((ce = cudaMemcpyAsync(B + off_dl, dl.data(), dl.size() * sizeof(short), cudaMemcpyHostToDevice, st)) ||
        (ce = cudaMemsetAsync(h12, 0, (size_t)nkeys * sizeof(int), st)) ||
        (ce = cudaMemsetAsync(h34, 0, (size_t)nkeys * sizeof(int), st)) ||
        (ce = cudaMemsetAsync(cnt, 0, 2 * sizeof(int), st)) ||
        (ce = cudaMemsetAsync(B + off_S, 0, bytes - off_S, st)))
        return fail(POLY_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(ce));
    const bool prod = delta != nullptr, scale = scale_out != nullptr, dbl = p->is_double != 0;
    if (prod && (ce = ps_forward(N, p->is_double, delta, K, p->d_tw_fwd, p->d_W, p->d_fhat, p->d_spill, st)))
        return fail(POLY_ERR_CUDA, std::string("forward transform: ") + cudaGetErrorString(ce));
    p->launches += prod ? 2 : 0;
    const int4* md[4];
    for (int t = 0; t < 4; t++) md[t] = (const int4*)(B + off_m[t]);
    const short* d_dl = (const short*)(B + off_dl);
    const int n0 = (int)m[0].size(), n1 = (int)m[1].size(), n2 = (int)m[2].size(), n3m = (int)m[3].size();
    auto pairs = [&](bool first, int* hist, int* cursor, void* out) {
        const int4* ma = first ? md[0] : md[2];
        const int4* mb = first ? md[1] : md[3];
        const int na = first ? n0 : n2, nb = first ? n1 : n3m;
        if (dbl)
            return prod ? launch_pairs<double, true>(first, ma, mb, na, nb, d_dl, key, hist, cursor, out, p->d_fhat, K, st)
                        : launch_pairs<double, false>(first, ma, mb, na, nb, d_dl, key, hist, cursor, out, p->d_fhat, K, st);
        return prod ? launch_pairs<float, true>(first, ma, mb, na, nb, d_dl, key, hist, cursor, out, p->d_fhat, K, st)
                    : launch_pairs<float, false>(first, ma, mb, na, nb, d_dl, key, hist, cursor, out, p->d_fhat, K, st);
    };
    if ((ce = pairs(true, h12, nullptr, nullptr)) || (ce = pairs(false, h34, nullptr, nullptr)) ||
        (ce = scan_keys(h12, o12, c12, (int)nkeys, (int*)(B + off_bs), st)) ||
        (ce = scan_keys(h34, o34, c34, (int)nkeys, (int*)(B + off_bs), st)) ||
        (ce = pairs(true, h12, c12, B + off_p12)) || (ce = pairs(false, h34, c34, B + off_p34)))
        return fail(POLY_ERR_CUDA, std::string("pair tables: ") + cudaGetErrorString(ce));
    tf_items_kernel<<<(int)((nkeys + 255) / 256), 256, 0, st>>>(h12, h34, (int)nkeys, (int2*)(B + off_it), cnt);
    if ((ce = cudaGetLastError())) return fail(POLY_ERR_CUDA, std::string("work items: ") + cudaGetErrorString(ce));
    p->launches += 4 + 6 + 1;
    TfQuadArgs a;
    a.items = (const int2*)(B + off_it);
    a.nitems = cnt;
    a.next = cnt + 1;
    a.h12 = h12;
    a.o12 = o12;
    a.h34 = h34;
    a.o34 = o34;
    a.dl = d_dl;
    a.ndl_smem = ndl_smem;
    a.nd = nd;
    a.local = 0;
    a.S = (double*)(B + off_S);
    a.A = (double*)(B + off_A);
    a.C = (unsigned long long*)(B + off_C);
    int blocks = 0;
    const void* P12 = B + off_p12;
    const void* P34 = B + off_p34;
    if (np12 > 0 && np34 > 0) {
        if (dbl)
            ce = !prod ? launch_quads<double, false, false>(P12, P34, a, p->sms, st, &blocks)
                       : (scale ? launch_quads<double, true, true>(P12, P34, a, p->sms, st, &blocks)
                                : launch_quads<double, true, false>(P12, P34, a, p->sms, st, &blocks));
        else
            ce = !prod ? launch_quads<float, false, false>(P12, P34, a, p->sms, st, &blocks)
                       : (scale ? launch_quads<float, true, true>(P12, P34, a, p->sms, st, &blocks)
                                : launch_quads<float, true, false>(P12, P34, a, p->sms, st, &blocks));
        if (ce) return fail(POLY_ERR_CUDA, std::string("quadrilateral kernel: ") + cudaGetErrorString(ce));
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
