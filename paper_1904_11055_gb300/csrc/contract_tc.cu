// Split-BF16 tensor-core contraction (tcgen05, sm_103a) of the product sums
//   S_b = sum_x prod_t D_{b_t}(x)                      (Eq. estimator, App. A)
// as Gram blocks C[r][c] = sum_x A_r(x) B_c(x): rows A_r are pair products
// D_{k1} D_{k2} (bispectrum, trispectrum) and columns B_c single fields D_{k3}
// (bispectrum) or pair products D_{k3} D_{k4} (trispectrum).
//
// Each FP32 factor is split into bf16 hi + lo and every Gram block accumulates
// hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory.  The
// accumulators are drained every `window` chunks into FP32 sums in shared memory
// (round-to-nearest adds), and the per-block sums are reduced in FP64 across
// blocks in a fixed order.
//
// Block layout: 16 producer warps + 1 control warp.  The control thread streams
// 32-cell chunks of all shell fields (one contiguous block of the cell-tiled
// field layout) into shared memory with TMA (128-byte swizzle) and issues the
// MMAs; the producers write the pair products of their TMEM lanes (A operand,
// M = 128 rows per tile) with tcgen05.st and the column factors (B operand)
// into shared memory in the K-major core-matrix layout.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "plan_internal.h"
#include "tc.cuh"
#include "../../include/polyspec_diag.h"

namespace ps {

constexpr int kTcChunk = 32;         // cells per chunk (K of one pipeline step)
constexpr int kTcStages = 6;         // TMA stages
constexpr int kTcProducers = 512;    // 16 warps: 4 per TMEM lane quadrant, each owning 8 cells of a chunk
constexpr int kTcThreads = kTcProducers + 32;
constexpr int kTcMaxMT = 4;          // M tiles per block
constexpr int kTcAccMax = 256;       // accumulator columns per block
constexpr int kTcABase = 256;        // first TMEM column of the A slots
constexpr int kTcMaxRuns = 64;       // N runs per block
constexpr int kTcMaxCols = 256;      // local B columns per block
constexpr uint32_t kLBO = 128, kSBO = 512;  // B layout: K-adjacent core matrices, 8-row groups (K = 32)

struct TcMTile {
    int row_off;  // 128 row factors at rowf[row_off ..]
    int run_off, nrun;
    int pad_;
};
struct TcGroup {
    int mt_off, nmt;
    int col_off, ncol;  // local column factors at colf[col_off ..], ncol a multiple of 16
    int acc_cols;
    int pad_[3];
};
struct TcCta {  // one block: a group and a chunk range
    int group;
    int pad_;
    long long c0, c1;
};

// ---------------------------------------------------------------------------------
// One MMA of a chunk, precomputed per block: accumulator column, A column within
// the slot, B byte offset within the slot's buffer, instruction descriptor, and
// flags (bit 0: B = lo part, bit 1: first product of a K-step pair (resets at a window start)).
struct TcMma {
    uint32_t d_col, a_col, b_off, idesc_flags;
};
constexpr int kTcMaxMma = 256;

template <int RA, int CA>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_contract_kernel(const __grid_constant__ CUtensorMap fmap, int nshell, int stage_bytes, int bbuf_bytes,
                       int slot_cap, int acc_max, int window, const TcCta* __restrict__ ctas,
                       const TcGroup* __restrict__ groups, const TcMTile* __restrict__ mtiles,
                       const int4* __restrict__ runs, const short2* __restrict__ rowf,
                       const short2* __restrict__ colf, double* __restrict__ partial, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* s_d = base;                                        // kTcStages x stage_bytes (1024-aligned)
    uint8_t* s_b = s_d + kTcStages * stage_bytes;               // [slot][hi, lo] x bbuf_bytes
    float* s_acc = (float*)(s_b + 2 * slot_cap * bbuf_bytes);   // [acc_max cols][128 rows]
    short2* s_rowf = (short2*)(s_acc + (size_t)acc_max * 128);  // [kTcMaxMT][128]
    short2* s_colf = s_rowf + kTcMaxMT * 128;                   // [kTcMaxCols]
    TcMma* s_mma = (TcMma*)(s_colf + kTcMaxCols);               // [kTcMaxMma]
    uint64_t* bars = (uint64_t*)(s_mma + kTcMaxMma);
    uint64_t* full = bars;                                      // [kTcStages]
    uint64_t* empty = full + kTcStages;                         // [kTcStages]
    uint64_t* produced = empty + kTcStages;                     // [4]
    uint64_t* mma_done = produced + 4;                          // [4]
    uint64_t* acc_ready = mma_done + 4;
    uint64_t* acc_free = acc_ready + 1;
    uint64_t* drain = acc_free + 1;
    uint32_t* s_tmem = (uint32_t*)(drain + 1);
    volatile int* s_abort = (volatile int*)(s_tmem + 1);
    int* s_meta = (int*)(s_tmem + 2);  // nmma, nslots, a0

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TcCta cta = ctas[blockIdx.x];
    const TcGroup grp = groups[cta.group];
    const int nch = (int)(cta.c1 - cta.c0);
    const int nmt = grp.nmt, ncol = grp.ncol, acc_cols = grp.acc_cols;

    if (tid == 0) {
        // TMEM columns: accumulators [0, acc_cols), then the A slots of nmt x 32 columns each
        const int a0 = (acc_cols + 31) / 32 * 32;
        int nslots = (512 - a0) / (nmt * 32);
        nslots = nslots < slot_cap ? nslots : slot_cap;
        nslots = nslots > 4 ? 4 : nslots;
        for (int st = 0; st < kTcStages; st++) {
            tc::mbar_init(&full[st], 1);
            tc::mbar_init(&empty[st], kTcProducers / 32);
        }
        for (int b = 0; b < 4; b++) {
            tc::mbar_init(&produced[b], kTcProducers / 32);
            tc::mbar_init(&mma_done[b], 1);
        }
        tc::mbar_init(acc_ready, 1);
        tc::mbar_init(acc_free, kTcProducers / 32);
        tc::mbar_init(drain, 1);
        tc::mbar_fence_init();
        *s_abort = 0;
        int nm = 0;
        for (int m = 0; m < nmt; m++) {
            const TcMTile mt = mtiles[grp.mt_off + m];
            for (int r = 0; r < mt.nrun; r++) {
                const int4 run = runs[mt.run_off + r];  // n0, nn, acc col
                const uint32_t idesc = tc::idesc_bf16(128, run.y);
                for (int ks = 0; ks < kTcChunk / 16; ks++) {
                    const uint32_t boff = (uint32_t)(run.x / 8) * kSBO + (uint32_t)ks * 2 * kLBO;
                    const uint32_t acol = (uint32_t)(m * 32 + ks * 8);
                    if (nm + 3 <= kTcMaxMma) {
                        s_mma[nm++] = TcMma{(uint32_t)run.z, acol, boff, idesc | (ks == 0 ? 2u : 0u)};  // hi x hi
                        s_mma[nm++] = TcMma{(uint32_t)run.z, acol, boff, idesc | 1u};                    // hi x lo
                        s_mma[nm++] = TcMma{(uint32_t)run.z, acol + 16, boff, idesc};                   // lo x hi
                    }
                }
            }
        }
        s_meta[0] = nm;
        s_meta[1] = nslots;
        s_meta[2] = a0;
    }
    for (int i = tid; i < kTcMaxMT * 128; i += kTcThreads) {
        const int m = i >> 7;
        s_rowf[i] = m < nmt ? rowf[mtiles[grp.mt_off + m].row_off + (i & 127)] : make_short2(-1, -1);
    }
    for (int i = tid; i < kTcMaxCols; i += kTcThreads) s_colf[i] = i < ncol ? colf[grp.col_off + i] : make_short2(-1, -1);
    for (int i = tid; i < acc_cols * 128; i += kTcThreads) s_acc[i] = 0.f;
    if (warp == kTcProducers / 32) {
        tc::tmem_alloc(s_tmem, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;
    const int nmma = s_meta[0], nslots = s_meta[1], a0 = s_meta[2];
    const uint32_t stage_tx = (uint32_t)nshell * kTcChunk * 4;
    const uint32_t slot_cols = (uint32_t)(nmt * 32);

    if (warp == kTcProducers / 32) {
        // ------------------------------------------------------------- control thread
        if (lane == 0 && nch > 0) {
            tc::prefetch_tensormap(&fmap);
            int issued = 0;
            for (; issued < kTcStages && issued < nch; issued++) {
                tc::mbar_arrive_expect_tx(&full[issued], stage_tx);
                tc::tma_load_2d(s_d + issued * stage_bytes, &fmap, 0, (int)((cta.c0 + issued) * nshell), &full[issued]);
            }
            const uint32_t desc_hi = (kSBO >> 4) | (1u << 14);  // stride byte offset, sm_100 descriptor version
            for (int i = 0; i < nch; i++) {
                const int slot = i % nslots, w = i / window;
                if (!tc::mbar_wait(&produced[slot], (uint32_t)((i / nslots) & 1), s_abort)) break;
                if (i % window == 0 && w > 0 && !tc::mbar_wait(acc_free, (uint32_t)((w - 1) & 1), s_abort)) break;
                tc::fence_after_sync();
                const uint32_t abase = tmem + (uint32_t)a0 + (uint32_t)slot * slot_cols;
                const uint32_t bh = tc::smem_u32(s_b + (2 * slot) * bbuf_bytes);
                const uint32_t bl = tc::smem_u32(s_b + (2 * slot + 1) * bbuf_bytes);
                const bool wstart = (i % window) == 0;
                for (int e = 0; e < nmma; e++) {
                    const TcMma mm = s_mma[e];
                    const uint32_t baddr = ((mm.idesc_flags & 1u) ? bl : bh) + mm.b_off;
                    const uint64_t desc = (uint64_t)(((baddr >> 4) & 0x3FFFu) | ((kLBO >> 4) << 16)) |
                                          ((uint64_t)desc_hi << 32);
                    const uint32_t acc = (wstart && (mm.idesc_flags & 2u)) ? 0u : 1u;
                    tc::mma_ts(tmem + mm.d_col, abase + mm.a_col, desc, mm.idesc_flags & ~3u, acc);
                }
                tc::mma_commit(&mma_done[slot]);
                if (i % window == window - 1 || i == nch - 1) tc::mma_commit(acc_ready);
                if (issued < nch) {
                    const int st = issued % kTcStages;
                    // the stage held chunk issued - kTcStages, released by the producers before produced[]
                    if (!tc::mbar_wait(&empty[st], (uint32_t)(((issued - kTcStages) / kTcStages) & 1), s_abort)) break;
                    tc::mbar_arrive_expect_tx(&full[st], stage_tx);
                    tc::tma_load_2d(s_d + st * stage_bytes, &fmap, 0, (int)((cta.c0 + issued) * nshell), &full[st]);
                    issued++;
                }
            }
            // drain: every MMA issued by this thread, and every TMA load it started
            tc::mma_commit(drain);
            volatile int no_abort = 0;
            tc::mbar_wait(drain, 0, &no_abort);
            for (int st = 0; st < kTcStages && st < issued; st++) {
                const int last = st + kTcStages * ((issued - 1 - st) / kTcStages);
                tc::mbar_wait(&full[st], (uint32_t)((last / kTcStages) & 1), &no_abort);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------- producers
        const int q = warp & 3, h = warp >> 2;  // lane quadrant, 8-cell slice of the chunk
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        const int row = 32 * q + lane;
        short2 rf[kTcMaxMT];
#pragma unroll
        for (int m = 0; m < kTcMaxMT; m++) rf[m] = s_rowf[m * 128 + row];
        for (int i = 0; i < nch; i++) {
            const int st = i % kTcStages, slot = i % nslots, w = i / window;
            if (!tc::mbar_wait_warp(&full[st], (uint32_t)((i / kTcStages) & 1), s_abort)) break;
            if (i >= nslots && !tc::mbar_wait_warp(&mma_done[slot], (uint32_t)((i / nslots - 1) & 1), s_abort)) break;
            const uint8_t* D = s_d + st * stage_bytes;
            // A operand first (the longer job): all loads of this lane's rows, then the products
            float4 xa[kTcMaxMT][2], xb[kTcMaxMT][2];
#pragma unroll
            for (int m = 0; m < kTcMaxMT; m++) {
                if (m < nmt && rf[m].x >= 0) {
                    const float4* r1 = (const float4*)(D + rf[m].x * 128);
                    xa[m][0] = r1[(2 * h) ^ (rf[m].x & 7)];
                    xa[m][1] = r1[(2 * h + 1) ^ (rf[m].x & 7)];
                    if (RA == 2) {
                        const float4* r2 = (const float4*)(D + rf[m].y * 128);
                        xb[m][0] = r2[(2 * h) ^ (rf[m].y & 7)];
                        xb[m][1] = r2[(2 * h + 1) ^ (rf[m].y & 7)];
                    }
                } else {
                    xa[m][0] = xa[m][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                    xb[m][0] = xb[m][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            const uint32_t abase = tmem + lane_base + (uint32_t)a0 + (uint32_t)slot * slot_cols;
#pragma unroll
            for (int m = 0; m < kTcMaxMT; m++) {
                if (m >= nmt) break;
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    const float4 a = xa[m][j];
                    if (RA == 2) {
                        const float4 c = xb[m][j];
                        tc::split2_prod(a.x, c.x, a.y, c.y, hi[2 * j], lo[2 * j]);
                        tc::split2_prod(a.z, c.z, a.w, c.w, hi[2 * j + 1], lo[2 * j + 1]);
                    } else {
                        tc::split2(a.x, a.y, hi[2 * j], lo[2 * j]);
                        tc::split2(a.z, a.w, hi[2 * j + 1], lo[2 * j + 1]);
                    }
                }
                tc::tmem_st4(abase + (uint32_t)(m * 32 + h * 4), hi);
                tc::tmem_st4(abase + (uint32_t)(m * 32 + 16 + h * 4), lo);
            }
            // B operand: (column n, 8-cell group kg) -> one 16-byte core-matrix row of hi and of lo
            uint8_t* Bh = s_b + (2 * slot) * bbuf_bytes;
            uint8_t* Bl = s_b + (2 * slot + 1) * bbuf_bytes;
            for (int it = tid; it < ncol * (kTcChunk / 8); it += kTcProducers) {
                const int kg = it / ncol, n = it - (it / ncol) * ncol;
                const short2 f = s_colf[n];
                uint4 hi, lo;
                if (f.x >= 0) {
                    const float4* r1 = (const float4*)(D + f.x * 128);
                    const float4 x0 = r1[(2 * kg) ^ (f.x & 7)], x1 = r1[(2 * kg + 1) ^ (f.x & 7)];
                    if (CA == 2) {
                        const float4* r2 = (const float4*)(D + f.y * 128);
                        const float4 y0 = r2[(2 * kg) ^ (f.y & 7)], y1 = r2[(2 * kg + 1) ^ (f.y & 7)];
                        tc::split2_prod(x0.x, y0.x, x0.y, y0.y, hi.x, lo.x);
                        tc::split2_prod(x0.z, y0.z, x0.w, y0.w, hi.y, lo.y);
                        tc::split2_prod(x1.x, y1.x, x1.y, y1.y, hi.z, lo.z);
                        tc::split2_prod(x1.z, y1.z, x1.w, y1.w, hi.w, lo.w);
                    } else {
                        tc::split2(x0.x, x0.y, hi.x, lo.x);
                        tc::split2(x0.z, x0.w, hi.y, lo.y);
                        tc::split2(x1.x, x1.y, hi.z, lo.z);
                        tc::split2(x1.z, x1.w, hi.w, lo.w);
                    }
                } else {
                    hi = make_uint4(0u, 0u, 0u, 0u);
                    lo = hi;
                }
                const uint32_t off = (uint32_t)(n / 8) * kSBO + (uint32_t)kg * kLBO + (uint32_t)(n % 8) * 16;
                *(uint4*)(Bh + off) = hi;
                *(uint4*)(Bl + off) = lo;
            }
            tc::fence_proxy_async_smem();
            tc::tmem_st_wait();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(&empty[st]);
                tc::mbar_arrive(&produced[slot]);
            }
            // drain the accumulators at the end of a window
            if (i % window == window - 1 || i == nch - 1) {
                if (!tc::mbar_wait_warp(acc_ready, (uint32_t)(w & 1), s_abort)) break;
                tc::fence_after_sync();
                for (int g = h; g < acc_cols / 16; g += 4) {
                    uint32_t v[16];
                    tc::tmem_ld16(tmem + lane_base + (uint32_t)(g * 16), v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 16; j++) s_acc[(g * 16 + j) * 128 + row] += __uint_as_float(v[j]);
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(acc_free);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    double* out = partial + (size_t)blockIdx.x * (kTcAccMax * 128);
    for (int i = tid; i < acc_cols * 128; i += kTcThreads) out[i] = (double)s_acc[i];
    if (warp == kTcProducers / 32) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
    if (tid == 0 && *s_abort) atomicExch(err, tc::kErrTimeout);
}

// S[b] = sum over the blocks of the bin's group of partial[block][slot]
__global__ void tc_reduce_kernel(const double* __restrict__ partial, const int4* __restrict__ bin_map, int64_t nbins,
                                 double* __restrict__ S) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbins; b += (int64_t)gridDim.x * blockDim.x) {
        const int4 m = bin_map[b];  // first block, block count, slot
        double s = 0.0;
        for (int k = 0; k < m.y; k++) s += partial[(size_t)(m.x + k) * (kTcAccMax * 128) + m.z];
        S[b] = s;
    }
}

// ---------------------------------------------------------------------------------
// self-test GEMM: D[128 x N] = A[128 x 32] * B[N x 32]^T with A written to TMEM
// and B to shared memory exactly as the contraction does (bf16 bit patterns in).
__global__ void __launch_bounds__(128, 1) tc_selftest_kernel(const uint16_t* __restrict__ A,
                                                             const uint16_t* __restrict__ B, int N,
                                                             float* __restrict__ D, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* sb = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bar = (uint64_t*)(sb + 32768);
    uint32_t* s_tmem = (uint32_t*)(bar + 1);
    volatile int* s_abort = (volatile int*)(s_tmem + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_fence_init();
        *s_abort = 0;
    }
    // B in the K-major core-matrix layout
    for (int it = tid; it < N * 4; it += 128) {
        const int kg = it / N, n = it % N;
        uint4 v;
        uint32_t* pv = (uint32_t*)&v;
        for (int j = 0; j < 4; j++)
            pv[j] = (uint32_t)B[n * 32 + 8 * kg + 2 * j] | ((uint32_t)B[n * 32 + 8 * kg + 2 * j + 1] << 16);
        *(uint4*)(sb + (n / 8) * kSBO + kg * kLBO + (n % 8) * 16) = v;
    }
    if (warp == 0) {
        tc::tmem_alloc(s_tmem, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;
    // A: row = tid, 32 K values -> 16 columns at kTcABase
    uint32_t a[16];
    for (int c = 0; c < 16; c++) a[c] = (uint32_t)A[tid * 32 + 2 * c] | ((uint32_t)A[tid * 32 + 2 * c + 1] << 16);
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    tc::tmem_st8(tmem + lane_base + kTcABase, a);
    tc::tmem_st8(tmem + lane_base + kTcABase + 8, a + 8);
    tc::fence_proxy_async_smem();
    tc::tmem_st_wait();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t sbase = tc::smem_u32(sb);
        for (int ks = 0; ks < 2; ks++)
            tc::mma_ts(tmem, tmem + kTcABase + ks * 8, tc::smem_desc(sbase + ks * 2 * kLBO, kLBO, kSBO),
                       tc::idesc_bf16(128, N), ks ? 1u : 0u);
        tc::mma_commit(bar);
    }
    __syncwarp();
    const bool ok = tc::mbar_wait_warp(bar, 0, s_abort);
    tc::fence_after_sync();
    if (ok)
        for (int g = 0; g < N / 16; g++) {
            uint32_t v[16];
            tc::tmem_ld16(tmem + lane_base + g * 16, v);
            tc::tmem_ld_wait();
            for (int j = 0; j < 16; j++) D[tid * N + g * 16 + j] = __uint_as_float(v[j]);
        }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
    if (tid == 0 && *s_abort) atomicExch(err, tc::kErrTimeout);
}

}  // namespace ps

// =====================================================================================
// host side
// =====================================================================================
using namespace ps;

struct TcState {
    CUtensorMap fmap;
    std::vector<TcCta> ctas;
    int ngroups = 0;
    int nshell = 0;
    int stage_bytes = 0, bbuf_bytes = 0, smem_bytes = 0;
    int window = 64;
    int slot_cap = 2, acc_max = 256;
    int ra = 2, ca = 1;
    void *d_ctas = nullptr, *d_groups = nullptr, *d_mtiles = nullptr, *d_runs = nullptr, *d_rowf = nullptr,
         *d_colf = nullptr, *d_binmap = nullptr;
    double* d_partial = nullptr;
    int* d_err = nullptr;
    double executed_flops_per_cell = 0;
};

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

static size_t tc_smem_bytes(int stage_bytes, int bbuf_bytes, int slots, int acc_max) {
    return 1024 + (size_t)kTcStages * stage_bytes + 2 * (size_t)slots * bbuf_bytes + (size_t)acc_max * 128 * 4 +
           kTcMaxMT * 128 * 4 + kTcMaxCols * 4 + kTcMaxMma * sizeof(TcMma) + (2 * kTcStages + 11) * 8 + 64;
}

// Build the groups: rows sorted by column span, 128-row M tiles, 16-column blocks.
poly_status ps_tc_prepare(PsPlan* p) {
    if (p->is_double) return POLY_ERR_UNSUPPORTED;
    TcState* t = new (std::nothrow) TcState();
    if (!t) return POLY_ERR_ALLOC;
    p->tc = t;
    const int n = p->order;
    t->ra = n >= 3 ? 2 : 1;
    t->ca = n - t->ra;
    t->nshell = p->nshell;
    auto rkey = [&](const int32_t* b) { return std::make_pair(b[0], t->ra == 2 ? b[1] : -1); };
    auto ckey = [&](const int32_t* b) { return std::make_pair(b[t->ra], t->ca == 2 ? b[t->ra + 1] : -1); };
    std::map<std::pair<int, int>, std::set<std::pair<int, int>>> rows;
    std::set<std::pair<int, int>> allcols;
    for (int64_t i = 0; i < p->nbins; i++) {
        rows[rkey(&p->bins[i * n])].insert(ckey(&p->bins[i * n]));
        allcols.insert(ckey(&p->bins[i * n]));
    }
    std::map<std::pair<int, int>, int> gcol;
    for (auto& c : allcols) gcol[c] = (int)gcol.size();
    struct Row {
        std::pair<int, int> key;
        std::vector<int> cols;  // global column indices, sorted
    };
    std::vector<Row> rl;
    for (auto& kv : rows) {
        Row r{kv.first, {}};
        for (auto& c : kv.second) r.cols.push_back(gcol[c]);
        std::sort(r.cols.begin(), r.cols.end());
        rl.push_back(r);
    }
    std::stable_sort(rl.begin(), rl.end(), [](const Row& a, const Row& b) {
        return std::make_pair(a.cols.front(), a.cols.back()) < std::make_pair(b.cols.front(), b.cols.back());
    });
    const int nmt_total = (int)((rl.size() + 127) / 128);
    // group consecutive M tiles; a group is valid when its local column list (<= 256)
    // and its accumulator columns (<= 256) fit
    auto mt_cols = [&](int m) {
        std::set<int> s;
        for (size_t r = (size_t)m * 128; r < std::min(rl.size(), (size_t)(m + 1) * 128); r++)
            s.insert(rl[r].cols.begin(), rl[r].cols.end());
        return s;
    };
    struct GroupPlan {
        int m0, m1;
        std::vector<int> local;  // global col indices, sorted, padded later
        int acc;
    };
    auto plan_group = [&](int m0, int m1, GroupPlan& g) -> bool {
        std::set<int> u;
        for (int m = m0; m < m1; m++) {
            auto s = mt_cols(m);
            u.insert(s.begin(), s.end());
        }
        g.m0 = m0;
        g.m1 = m1;
        g.local.assign(u.begin(), u.end());
        if ((int)g.local.size() > kTcMaxCols) return false;
        std::map<int, int> lidx;
        for (size_t i = 0; i < g.local.size(); i++) lidx[g.local[i]] = (int)i;
        g.acc = 0;
        for (int m = m0; m < m1; m++) {
            std::set<int> blocks;
            for (int c : mt_cols(m)) blocks.insert(lidx[c] / 16);
            g.acc += 16 * (int)blocks.size();
        }
        return g.acc <= kTcAccMax && (m1 - m0) <= kTcMaxMT;
    };
    std::vector<GroupPlan> gplans;
    int ngroups = (nmt_total + kTcMaxMT - 1) / kTcMaxMT;
    while (true) {
        gplans.clear();
        bool ok = true;
        for (int g = 0; g < ngroups && ok; g++) {
            const int m0 = (int)((long long)nmt_total * g / ngroups), m1 = (int)((long long)nmt_total * (g + 1) / ngroups);
            GroupPlan gp;
            if (m1 <= m0) continue;
            ok = plan_group(m0, m1, gp);
            gplans.push_back(gp);
        }
        if (ok) break;
        if (ngroups >= nmt_total) return POLY_ERR_UNSUPPORTED;  // a single M tile does not fit
        ngroups++;
    }
    t->ngroups = (int)gplans.size();
    // device tables
    std::vector<TcGroup> groups;
    std::vector<TcMTile> mtiles;
    std::vector<int4> runs;
    std::vector<short2> rowf, colf;
    std::map<std::tuple<int, int, int, int>, std::pair<int, int>> slot_of;  // (row, col) keys -> (group, slot)
    std::vector<std::pair<int, int>> gcol_key(gcol.size());
    for (auto& kv : gcol) gcol_key[kv.second] = kv.first;
    double work_cells = 0;
    std::vector<double> gwork;
    for (int gi = 0; gi < t->ngroups; gi++) {
        const GroupPlan& gp = gplans[gi];
        TcGroup G{};
        G.mt_off = (int)mtiles.size();
        G.nmt = gp.m1 - gp.m0;
        G.col_off = (int)colf.size();
        const int ncol = ((int)gp.local.size() + 15) / 16 * 16;
        G.ncol = ncol;
        std::map<int, int> lidx;
        for (size_t i = 0; i < gp.local.size(); i++) {
            lidx[gp.local[i]] = (int)i;
            auto k = gcol_key[gp.local[i]];
            short2 f;
            f.x = (short)(k.first - 1);
            f.y = (short)(k.second > 0 ? k.second - 1 : -1);
            colf.push_back(f);
        }
        for (int i = (int)gp.local.size(); i < ncol; i++) colf.push_back(make_short2(-1, -1));
        int acc = 0;
        for (int m = gp.m0; m < gp.m1; m++) {
            TcMTile M{};
            M.row_off = (int)rowf.size();
            M.run_off = (int)runs.size();
            const size_t r0 = (size_t)m * 128, r1 = std::min(rl.size(), r0 + 128);
            for (size_t r = r0; r < r0 + 128; r++) {
                short2 f = make_short2(-1, -1);
                if (r < r1) {
                    f.x = (short)(rl[r].key.first - 1);
                    f.y = (short)(rl[r].key.second > 0 ? rl[r].key.second - 1 : -1);
                }
                rowf.push_back(f);
            }
            std::set<int> blocks;
            for (size_t r = r0; r < r1; r++)
                for (int c : rl[r].cols) blocks.insert(lidx[c] / 16);
            // merge consecutive blocks into runs
            std::vector<int> bl(blocks.begin(), blocks.end());
            std::map<int, std::pair<int, int>> block_acc;  // block -> (run n0, acc col of run start)
            for (size_t k = 0; k < bl.size();) {
                size_t e = k;
                while (e + 1 < bl.size() && bl[e + 1] == bl[e] + 1 && (int)(e + 2 - k) * 16 <= 256) e++;
                const int n0 = bl[k] * 16, nn = (int)(e - k + 1) * 16;
                runs.push_back(make_int4(n0, nn, acc, m - gp.m0));
                for (size_t q = k; q <= e; q++) block_acc[bl[q]] = {n0, acc};
                acc += nn;
                k = e + 1;
            }
            M.nrun = (int)runs.size() - M.run_off;
            for (size_t r = r0; r < r1; r++)
                for (int c : rl[r].cols) {
                    const int lc = lidx[c];
                    auto ba = block_acc[lc / 16];
                    const int acc_col = ba.second + (lc - ba.first);
                    auto ck = gcol_key[c];
                    slot_of[{rl[r].key.first, rl[r].key.second, ck.first, ck.second}] = {gi, acc_col * 128 + (int)(r - r0)};
                }
            mtiles.push_back(M);
        }
        G.acc_cols = acc;
        groups.push_back(G);
        gwork.push_back((double)acc);
        work_cells += acc;
        t->executed_flops_per_cell += 3.0 * 2.0 * 128.0 * acc;
    }
    // blocks: split each group's chunks in proportion to its work
    const int64_t ncell = (int64_t)p->N * p->N * p->N;
    const int64_t nchunks = (ncell + kTcChunk - 1) / kTcChunk;
    const int budget = std::max(p->sms, t->ngroups);
    std::vector<int> nsplit(t->ngroups);
    int used = 0;
    for (int g = 0; g < t->ngroups; g++) {
        nsplit[g] = std::max(1, (int)(budget * gwork[g] / work_cells));
        nsplit[g] = (int)std::min<int64_t>(nsplit[g], std::max<int64_t>(1, nchunks / 8));
        used += nsplit[g];
    }
    std::vector<int> first(t->ngroups);
    for (int g = 0; g < t->ngroups; g++) {
        first[g] = (int)t->ctas.size();
        for (int k = 0; k < nsplit[g]; k++) {
            TcCta c{};
            c.group = g;
            c.c0 = nchunks * k / nsplit[g];
            c.c1 = nchunks * (k + 1) / nsplit[g];
            t->ctas.push_back(c);
        }
    }
    std::vector<int4> binmap(p->nbins);
    for (int64_t i = 0; i < p->nbins; i++) {
        auto rk = rkey(&p->bins[i * n]);
        auto ck = ckey(&p->bins[i * n]);
        auto gs = slot_of.at({rk.first, rk.second, ck.first, ck.second});
        binmap[i] = make_int4(first[gs.first], nsplit[gs.first], gs.second, 0);
    }
    auto up = [&](void** d, const void* h, size_t bytes) -> poly_status {
        poly_status s = ps_alloc(p, d, bytes);
        if (s) return s;
        return cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice) ? POLY_ERR_CUDA : POLY_OK;
    };
    poly_status s;
    if ((s = up(&t->d_ctas, t->ctas.data(), t->ctas.size() * sizeof(TcCta))) ||
        (s = up(&t->d_groups, groups.data(), groups.size() * sizeof(TcGroup))) ||
        (s = up(&t->d_mtiles, mtiles.data(), mtiles.size() * sizeof(TcMTile))) ||
        (s = up(&t->d_runs, runs.data(), std::max<size_t>(1, runs.size()) * sizeof(int4))) ||
        (s = up(&t->d_rowf, rowf.data(), rowf.size() * sizeof(short2))) ||
        (s = up(&t->d_colf, colf.data(), colf.size() * sizeof(short2))) ||
        (s = up(&t->d_binmap, binmap.data(), std::max<size_t>(1, binmap.size()) * sizeof(int4))))
        return s;
    for (auto& g : groups)
        if (g.nmt > 0 && (int)runs.size() > 0) {
            int nr = 0;
            for (int m = 0; m < g.nmt; m++) nr += mtiles[g.mt_off + m].nrun;
            if (nr > kTcMaxRuns) return POLY_ERR_UNSUPPORTED;
        }
    if ((s = ps_alloc(p, (void**)&t->d_partial, t->ctas.size() * (size_t)kTcAccMax * 128 * 8))) return s;
    if ((s = ps_alloc(p, (void**)&t->d_err, 16))) return s;
    if (cudaMemset(t->d_err, 0, 16)) return POLY_ERR_CUDA;
    // tensor map over the cell-tiled fields [ncell/32 * nshell rows][32 cells] fp32: one box = one 32-cell
    // chunk of every shell (a contiguous block), 128-byte swizzle
    auto enc = get_encode();
    if (!enc) return POLY_ERR_UNSUPPORTED;
    cuuint64_t gdim[2] = {(cuuint64_t)kTcChunk, (cuuint64_t)(ncell / kTcChunk) * (cuuint64_t)p->nshell};
    cuuint64_t gstride[1] = {(cuuint64_t)kTcChunk * 4};
    cuuint32_t box[2] = {(cuuint32_t)kTcChunk, (cuuint32_t)p->nshell};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&t->fmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->d_fields, gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return POLY_ERR_CUDA;
    t->stage_bytes = (p->nshell * 128 + 1023) / 1024 * 1024;
    int maxcol = 16, maxacc = 16;
    for (auto& g : groups) {
        maxcol = std::max(maxcol, g.ncol);
        maxacc = std::max(maxacc, g.acc_cols);
        int nm = 0;
        for (int m = 0; m < g.nmt; m++) nm += 6 * mtiles[g.mt_off + m].nrun;
        if (nm > kTcMaxMma) return POLY_ERR_UNSUPPORTED;
    }
    t->bbuf_bytes = maxcol * kTcChunk * 2;
    t->acc_max = maxacc;
    t->slot_cap = 4;  // A/B slots: as many as shared memory allows (the kernel also bounds them by TMEM)
    while (t->slot_cap > 2 && tc_smem_bytes(t->stage_bytes, t->bbuf_bytes, t->slot_cap, maxacc) > 227 * 1024)
        t->slot_cap--;
    t->smem_bytes = (int)tc_smem_bytes(t->stage_bytes, t->bbuf_bytes, t->slot_cap, maxacc);
    if (t->smem_bytes > 227 * 1024) return POLY_ERR_UNSUPPORTED;
    const char* w = getenv("POLY_TC_WINDOW");
    if (w && atoi(w) > 0) t->window = atoi(w);
    return POLY_OK;
}

poly_status ps_tc_sums(PsPlan* p, cudaStream_t st) {
    TcState* t = p->tc;
    if (!t) return POLY_ERR_UNSUPPORTED;
    cudaError_t e;
    auto launch = [&](auto kern) -> cudaError_t {
        cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, t->smem_bytes);
        if (e2) return e2;
        kern<<<(unsigned)t->ctas.size(), kTcThreads, t->smem_bytes, st>>>(
            t->fmap, t->nshell, t->stage_bytes, t->bbuf_bytes, t->slot_cap, t->acc_max, t->window, (const TcCta*)t->d_ctas,
            (const TcGroup*)t->d_groups, (const TcMTile*)t->d_mtiles, (const int4*)t->d_runs,
            (const short2*)t->d_rowf, (const short2*)t->d_colf, t->d_partial, t->d_err);
        return cudaGetLastError();
    };
    if (t->ra == 2 && t->ca == 1) e = launch(tc_contract_kernel<2, 1>);
    else if (t->ra == 2 && t->ca == 2) e = launch(tc_contract_kernel<2, 2>);
    else e = launch(tc_contract_kernel<1, 1>);
    if (e) return POLY_ERR_CUDA;
    if (p->timing) cudaEventRecord(p->ev[3], st);
    const int blocks = (int)std::min<int64_t>((p->nbins + 255) / 256, 4096);
    tc_reduce_kernel<<<std::max(1, blocks), 256, 0, st>>>(t->d_partial, (const int4*)t->d_binmap, p->nbins, p->d_S);
    p->launches += 2;
    return cudaGetLastError() ? POLY_ERR_CUDA : POLY_OK;
}

void ps_tc_free(PsPlan* p) {
    delete p->tc;
    p->tc = nullptr;
}

poly_status ps_check_device_error(PsPlan* p) {
    if (!p->tc || !p->tc->d_err) return POLY_OK;
    int v = 0;
    if (cudaMemcpy(&v, p->tc->d_err, sizeof(int), cudaMemcpyDeviceToHost)) return POLY_ERR_CUDA;
    if (v) {
        cudaMemset(p->tc->d_err, 0, sizeof(int));
        return POLY_ERR_TIMEOUT;
    }
    return POLY_OK;
}

double ps_tc_executed_flops(const PsPlan* p) {
    return p->tc ? p->tc->executed_flops_per_cell * (double)p->N * p->N * p->N : 0.0;
}

extern "C" int poly_diag_tc_gemm(const uint16_t* A_host, const uint16_t* B_host, int N, float* D_host) {
    if (N < 16 || N > 256 || N % 16) return 1;
    uint16_t *dA = nullptr, *dB = nullptr;
    float* dD = nullptr;
    int* dErr = nullptr;
    int rc = 0, herr = 0;
    const size_t smem = 1024 + 32768 + 64;
    if (cudaMalloc(&dA, 128 * 32 * 2) || cudaMalloc(&dB, (size_t)N * 32 * 2) || cudaMalloc(&dD, (size_t)128 * N * 4) ||
        cudaMalloc(&dErr, 4))
        rc = 3;
    if (!rc && (cudaMemcpy(dA, A_host, 128 * 32 * 2, cudaMemcpyHostToDevice) ||
                cudaMemcpy(dB, B_host, (size_t)N * 32 * 2, cudaMemcpyHostToDevice) || cudaMemset(dErr, 0, 4) ||
                cudaMemset(dD, 0, (size_t)128 * N * 4)))
        rc = 4;
    if (!rc && cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) rc = 4;
    if (!rc) {
        tc_selftest_kernel<<<1, 128, smem>>>(dA, dB, N, dD, dErr);
        if (cudaGetLastError() || cudaDeviceSynchronize()) rc = 4;
    }
    if (!rc && (cudaMemcpy(D_host, dD, (size_t)128 * N * 4, cudaMemcpyDeviceToHost) ||
                cudaMemcpy(&herr, dErr, 4, cudaMemcpyDeviceToHost)))
        rc = 4;
    if (!rc && herr) rc = 5;
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(dErr);
    return rc;
}
