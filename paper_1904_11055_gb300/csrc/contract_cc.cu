// CUDA-core contraction over grid cells (Eq. estimator, discrete form of App. A):
//   S_b = sum_x prod_t D_{b_t}(x)
// recast per tile as a GEMM  C[r][c] = sum_x A_r(x) B_c(x), where a row A_r is a
// product of one to three shell fields (e.g. D_{k1} D_{k2}) and a column B_c the
// product of the remaining ones (D_{k3}, D_{k3} D_{k4}, or three for n = 5, 6).  Cells are split
// across blocks (split-K); every block writes its FP64 partial tile and a
// fixed-order reduction gathers the bins.
//
// FP32 instantiation: products and per-chunk accumulation in FP32, flushed to
// FP64 every kFlushChunks chunks.  FP64 instantiation: FP64 throughout (the
// plain method, and the exact polygon counts over the symmetry wedge).
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace ps {

constexpr int kCcThreads = 256;
constexpr int kFlushChunks = 32;  // 32 chunks x 32 cells = 1024 cells per FP32 partial sum

PS_DEV void load4(const float* p, float* v) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
PS_DEV void load4(const double* p, double* v) {
    const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
    v[0] = q0.x, v[1] = q0.y, v[2] = q1.x, v[3] = q1.y;
}

// NF: factors per row or column at most (2 for n <= 4, 3 for n = 5, 6); the third is never read for NF = 2.
template <typename T, bool WEIGHTED, bool ABS, int NF>
__global__ void __launch_bounds__(kCcThreads) contract_cc_kernel(
    const T* __restrict__ fields, size_t fstride, int tile_ns, int64_t ncell, const T* __restrict__ weight,
    const PsTile* __restrict__ tiles, int ntiles, const int* __restrict__ field_ids, const short4* __restrict__ rowf,
    const short4* __restrict__ colf, int64_t chunks_per_split, double* __restrict__ partial) {
    constexpr int CH = sizeof(T) == 8 ? 16 : 32, TM = kCcTM, TN = kCcTN;
    __shared__ T s_d[kCcMaxFields][CH + 1];
    __shared__ __align__(16) T s_a[CH][TM];
    __shared__ __align__(16) T s_b[CH][TN];
    using FT = typename std::conditional<NF == 3, short4, short2>::type;  // factor record in shared memory
    __shared__ FT s_rf[TM], s_cf[TN];
    __shared__ int s_fid[kCcMaxFields];

    const PsTile tile = tiles[blockIdx.x];
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // warp w owns the 32x16 region (rows 32*(w/4).., cols 16*(w%4)..), lane -> 4x4 sub-block
    const int r0 = 32 * (warp >> 2) + 4 * (lane >> 2);
    const int c0 = 16 * (warp & 3) + 4 * (lane & 3);
    const bool active = (tile.region_mask >> warp) & 1u;

    auto narrow = [](short4 f) {
        if constexpr (NF == 3) return f;
        else return make_short2(f.x, f.y);
    };
    const short4 none = make_short4(-1, -1, -1, -1);
    for (int i = tid; i < TM; i += kCcThreads) s_rf[i] = narrow(i < tile.nrow ? rowf[tile.row_off + i] : none);
    for (int i = tid; i < TN; i += kCcThreads) s_cf[i] = narrow(i < tile.ncol ? colf[tile.col_off + i] : none);
    for (int i = tid; i < tile.nfield; i += kCcThreads) s_fid[i] = field_ids[tile.field_off + i];

    T acc[4][4];
    double acc64[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            acc[i][j] = 0;
            acc64[i][j] = 0.0;
        }

    const int64_t nchunks = (ncell + CH - 1) / CH;
    const int64_t cbeg = (int64_t)blockIdx.y * chunks_per_split;
    const int64_t cend = min(nchunks, cbeg + chunks_per_split);
    __syncthreads();
    // register prefetch of the next chunk's field values (each thread owns a fixed set of (f, x))
    constexpr int PF = kCcMaxFields * CH / kCcThreads;
    const int nload = tile.nfield * CH;
    T pf[PF];
    auto fetch = [&](int64_t ch) {
#pragma unroll
        for (int k = 0; k < PF; k++) {
            const int e = tid + k * kCcThreads;
            if (e < nload) {
                const int f = e / CH, x = e - (e / CH) * CH;
                const int64_t cell = ch * CH + x;
                const size_t a = tile_ns > 0 ? (size_t)(cell >> 5) * tile_ns * 32 + (size_t)s_fid[f] * 32 + (cell & 31)
                                             : (size_t)s_fid[f] * fstride + cell;
                pf[k] = (ch < cend && cell < ncell) ? fields[a] : (T)0;
            }
        }
    };
    // the row and column this thread forms products for are the same in every chunk
    static_assert(kCcThreads % TM == 0 && kCcThreads % TN == 0, "rows and columns per thread must not vary");
    const int r = tid % TM, c = tid % TN;
    const FT frow = s_rf[r], fcol = s_cf[c];
    if (cbeg < cend) fetch(cbeg);
    int since_flush = 0;
    for (int64_t ch = cbeg; ch < cend; ch++) {
        const int64_t base = ch * CH;
        // 1. this chunk's field values into shared memory, then prefetch the next chunk
#pragma unroll
        for (int k = 0; k < PF; k++) {
            const int e = tid + k * kCcThreads;
            if (e < nload) s_d[e / CH][e - (e / CH) * CH] = pf[k];
        }
        __syncthreads();
        fetch(ch + 1);
        // 2. row and column products
        for (int x = tid / TM; x < CH; x += kCcThreads / TM) {  // this thread's row r, every cell x it owns
            const FT f = frow;
            T v = 0;
            if (f.x >= 0) {
                v = s_d[f.x][x];
                if (f.y >= 0) v *= s_d[f.y][x];
                if constexpr (NF == 3)
                    if (f.z >= 0) v *= s_d[f.z][x];
                if (WEIGHTED) {
                    const int64_t cell = base + x;
                    v *= cell < ncell ? weight[cell] : (T)0;
                }
                if (ABS) v = v < 0 ? -v : v;
            }
            s_a[x][r] = v;
        }
        for (int x = tid / TN; x < CH; x += kCcThreads / TN) {
            const FT f = fcol;
            T v = 0;
            if (f.x >= 0) {
                v = s_d[f.x][x];
                if (f.y >= 0) v *= s_d[f.y][x];
                if constexpr (NF == 3)
                    if (f.z >= 0) v *= s_d[f.z][x];
                if (ABS) v = v < 0 ? -v : v;
            }
            s_b[x][c] = v;
        }
        __syncthreads();
        // 3. 4x4 outer products per lane over the chunk (16-byte vector loads)
        if (active) {
#pragma unroll 8
            for (int x = 0; x < CH; x++) {
                T a[4], b[4];
                load4(&s_a[x][r0], a);
                load4(&s_b[x][c0], b);
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
        }
        if (sizeof(T) == 4 && ++since_flush == kFlushChunks) {
            since_flush = 0;
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    acc64[i][j] += (double)acc[i][j];
                    acc[i][j] = 0;
                }
        }
    }
    double* out = partial + ((size_t)blockIdx.y * ntiles + blockIdx.x) * (TM * TN);
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) out[(r0 + i) * TN + c0 + j] = acc64[i][j] + (double)acc[i][j];
}

__global__ void reduce_slots_kernel(const double* __restrict__ partial, int nsplit, int64_t slot_stride,
                                    const int64_t* __restrict__ slot, int64_t nbins, double* __restrict__ S) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbins; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = slot[b];
        double s = 0.0;
        for (int k = 0; k < nsplit; k++) s += partial[(size_t)k * slot_stride + o];
        S[b] = s;
    }
}

__global__ void normalise_kernel(const double* __restrict__ S, const int64_t* __restrict__ counts, int64_t nbins,
                                 double norm, double n3, double* __restrict__ out) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbins; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = counts[b];
        out[b] = c > 0 ? norm * S[b] / (n3 * (double)c) : 0.0;
    }
}

}  // namespace ps

using namespace ps;

template <int NF>
static cudaError_t contract_cc_launch(int is_double, int weighted, int absval, const void* fields, size_t field_stride,
                                      int tile_ns, int64_t ncell, const void* weight, const PsTile* tiles, int ntiles,
                                      const int* field_ids, const short4* rowf, const short4* colf, int nsplit,
                                      int64_t chunks_per_split, double* partial, cudaStream_t st) {
    dim3 grid(ntiles, nsplit);
    if (is_double) {
        if (weighted)
            contract_cc_kernel<double, true, false, NF><<<grid, kCcThreads, 0, st>>>(
                (const double*)fields, field_stride, tile_ns, ncell, (const double*)weight, tiles, ntiles, field_ids, rowf,
                colf, chunks_per_split, partial);
        else if (absval)
            contract_cc_kernel<double, false, true, NF><<<grid, kCcThreads, 0, st>>>(
                (const double*)fields, field_stride, tile_ns, ncell, nullptr, tiles, ntiles, field_ids, rowf, colf,
                chunks_per_split, partial);
        else
            contract_cc_kernel<double, false, false, NF><<<grid, kCcThreads, 0, st>>>(
                (const double*)fields, field_stride, tile_ns, ncell, nullptr, tiles, ntiles, field_ids, rowf, colf,
                chunks_per_split, partial);
    } else {
        if (weighted) return cudaErrorInvalidValue;
        if (absval)
            contract_cc_kernel<float, false, true, NF><<<grid, kCcThreads, 0, st>>>(
                (const float*)fields, field_stride, tile_ns, ncell, nullptr, tiles, ntiles, field_ids, rowf, colf,
                chunks_per_split, partial);
        else
            contract_cc_kernel<float, false, false, NF><<<grid, kCcThreads, 0, st>>>(
                (const float*)fields, field_stride, tile_ns, ncell, nullptr, tiles, ntiles, field_ids, rowf, colf,
                chunks_per_split, partial);
    }
    return cudaGetLastError();
}

cudaError_t ps_contract_cc(int is_double, int weighted, int absval, int nf, const void* fields, size_t field_stride,
                           int tile_ns, int64_t ncell, const void* weight, const PsTile* tiles, int ntiles, const int* field_ids,
                           const short4* rowf, const short4* colf, int nsplit, int64_t chunks_per_split,
                           double* partial, cudaStream_t st) {
    if (nf == 3)
        return contract_cc_launch<3>(is_double, weighted, absval, fields, field_stride, tile_ns, ncell, weight, tiles,
                                     ntiles, field_ids, rowf, colf, nsplit, chunks_per_split, partial, st);
    return contract_cc_launch<2>(is_double, weighted, absval, fields, field_stride, tile_ns, ncell, weight, tiles, ntiles,
                                 field_ids, rowf, colf, nsplit, chunks_per_split, partial, st);
}

cudaError_t ps_reduce_slots(const double* partial, int nsplit, int64_t slot_stride, const int64_t* slot,
                            int64_t nbins, double* S, cudaStream_t st) {
    if (nbins <= 0) return cudaSuccess;
    int blocks = (int)((nbins + 255) / 256 < 4096 ? (nbins + 255) / 256 : 4096);
    reduce_slots_kernel<<<blocks, 256, 0, st>>>(partial, nsplit, slot_stride, slot, nbins, S);
    return cudaGetLastError();
}

cudaError_t ps_normalise(const double* S, const int64_t* counts, int64_t nbins, double norm, double n3, double* out,
                         cudaStream_t st) {
    if (nbins <= 0) return cudaSuccess;
    int blocks = (int)((nbins + 255) / 256 < 4096 ? (nbins + 255) / 256 : 4096);
    normalise_kernel<<<blocks, 256, 0, st>>>(S, counts, nbins, norm, n3, out);
    return cudaGetLastError();
}
