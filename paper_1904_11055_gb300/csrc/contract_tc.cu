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
// Block layout: producer warps in teams of 8 (three teams where every group has
// three A/B slots, else two) and 4 issuer warps.  The last
// issuer warp when the block has fewer than 4 M tiles (else issuer 0) streams
// 32-cell chunks of all shell fields (one contiguous block of the cell-tiled
// field layout) into shared memory with TMA (128-byte swizzle).
// With T teams, team t produces chunks t, t + T, ..., so that one team's barrier
// waits overlap the other teams' work; chunk i goes to A/B slot i mod nslots (up
// to 4 slots, as many as tensor memory holds next to the accumulators, and at
// least T), so a team reuses a slot only after the MMAs of a chunk no later than its previous one.
// Three teams at 72 registers a thread instead of two at 96 keep more producer warps
// in flight: the products are issue- and latency-bound.
// Producer warp w of a team owns
// TMEM lane quadrant w % 4 and the 16-cell half w / 4 of a chunk: in every M tile
// of the block, each lane forms the 16 products of its row in its half and
// writes their hi and lo parts with one 16-column tcgen05.st (per M tile the A
// slot holds [hi | lo] of cells 0-15, then [hi | lo] of cells 16-31), so the
// work per chunk is proportional to the number of M tiles.  The rows of a warp
// come from 8 consecutive k1 and a few consecutive k2, so its shared-memory reads
// of the factors are bank-conflict-free broadcasts.  The team then writes the
// column factors (B operand) into shared memory in the K-major core-matrix layout.  Issuer warp m issues the MMAs of M tile m (operands in
// registers; one elected lane issues and commits).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <tuple>
#include <array>
#include <cstring>
#include <map>
#include <new>
#include <set>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "plan_internal.h"
#include "tc.cuh"
#include "../../include/polyspec_diag.h"

namespace ps {

constexpr int kTcChunk = 32;         // cells per chunk (K of one pipeline step)
constexpr int kTcStages = 6;         // TMA stages (a multiple of 2 and 3: each team cycles through its own)
constexpr int kTcMaxMT = 4;          // M tiles per block
constexpr int kTcTeamWarps = 8;      // producer warps per team: 4 lane quadrants x 2 pairs of M tiles
constexpr int kTcIssuers = kTcMaxMT;  // one MMA-issuing warp per M tile
// threads of a block with `teams` producer teams (team t takes chunks t, t + teams, ...):
// three teams where every group has three A/B slots, else two
__host__ __device__ constexpr int tc_threads(int teams) { return (teams * kTcTeamWarps + kTcIssuers) * 32; }
constexpr int kTcAccMax = 256;       // accumulator columns per block
constexpr int kTcABase = 256;        // first TMEM column of the A operand in the self-test
constexpr int kTcMaxRunsMt = 4;      // N runs per M tile
constexpr int kTcMaxSlots = 4;       // A/B slots
constexpr int kTcMaxCols = 256;      // local B columns per block
constexpr int kTcRowOctet = 8;       // pair rows of one producer warp come from 8 consecutive k1
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

// Window bookkeeping without divisions: the accumulators are drained after the
// last chunk of each window of `window` chunks and after the block's last chunk.
struct TcWindow {
    int end, index;  // last chunk of the current window, window number
    __device__ TcWindow(int i0, int window) : end((i0 / window + 1) * window - 1), index(i0 / window) {}
    __device__ void advance_to(int i, int window) {
        while (i > end) {
            end += window;
            index++;
        }
    }
};

// One B item: 8 cells of column factor(s) -> hi and lo 16-byte core-matrix rows.
// key1 < 0 marks a padding column (zeros).  With three factors (CA = 3) the first two are
// multiplied in FP32 first.
template <int CA>
__device__ __forceinline__ void tc_b_item(uint32_t D, int key1, int key2, int key3, uint32_t dst_hi,
                                          uint32_t dst_lo) {
    uint32_t h[4] = {0u, 0u, 0u, 0u}, l[4] = {0u, 0u, 0u, 0u};
    if (key1 >= 0) {
        float4 x0, x1;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(x0.x), "=f"(x0.y), "=f"(x0.z), "=f"(x0.w) : "r"(D + (uint32_t)key1));
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(x1.x), "=f"(x1.y), "=f"(x1.z), "=f"(x1.w) : "r"(D + ((uint32_t)key1 ^ 16u)));
        if (CA == 3) {
            float4 z0, z1;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(z0.x), "=f"(z0.y), "=f"(z0.z), "=f"(z0.w) : "r"(D + (uint32_t)key3));
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(z1.x), "=f"(z1.y), "=f"(z1.z), "=f"(z1.w) : "r"(D + ((uint32_t)key3 ^ 16u)));
            x0.x *= z0.x;
            x0.y *= z0.y;
            x0.z *= z0.z;
            x0.w *= z0.w;
            x1.x *= z1.x;
            x1.y *= z1.y;
            x1.z *= z1.z;
            x1.w *= z1.w;
        }
        if (CA >= 2) {
            float4 y0, y1;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(y0.x), "=f"(y0.y), "=f"(y0.z), "=f"(y0.w) : "r"(D + (uint32_t)key2));
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(y1.x), "=f"(y1.y), "=f"(y1.z), "=f"(y1.w) : "r"(D + ((uint32_t)key2 ^ 16u)));
            tc::split2_prod_fast(x0.x, y0.x, x0.y, y0.y, h[0], l[0]);
            tc::split2_prod_fast(x0.z, y0.z, x0.w, y0.w, h[1], l[1]);
            tc::split2_prod_fast(x1.x, y1.x, x1.y, y1.y, h[2], l[2]);
            tc::split2_prod_fast(x1.z, y1.z, x1.w, y1.w, h[3], l[3]);
        } else {
            tc::split2_fast(x0.x, x0.y, h[0], l[0]);
            tc::split2_fast(x0.z, x0.w, h[1], l[1]);
            tc::split2_fast(x1.x, x1.y, h[2], l[2]);
            tc::split2_fast(x1.z, x1.w, h[3], l[3]);
        }
    }
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst_hi), "r"(h[0]), "r"(h[1]), "r"(h[2]), "r"(h[3])
                 : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst_lo), "r"(l[0]), "r"(l[1]), "r"(l[2]), "r"(l[3])
                 : "memory");
}

// Shared-memory byte offset of 16-byte chunk c of staged shell row k (128-byte
// swizzle): k * 128 + ((c ^ (k & 7)) * 16) = row_key(k) ^ (c * 16).
__device__ __forceinline__ uint32_t tc_row_key(int k) { return (uint32_t)(k * 128) ^ (uint32_t)((k & 7) * 16); }

// The 16 products of one row in its 16-cell half of a chunk: v[0..7] = hi, v[8..15] = lo,
// column j of each holding cells 2j, 2j + 1 of the half.  r1, r2 = stage base + the row
// factors' keys with the half already folded in (key ^ 64 half): the stage base is
// 1024-aligned and the swizzle only flips address bits 4-6, so the 16-byte chunk c4 of
// the half lies at r ^ (16 c4), one XOR with an immediate per load.
template <int RA>
__device__ __forceinline__ void tc_row_products(uint32_t r1, uint32_t r2, uint32_t r3, uint32_t* v) {
#pragma unroll
    for (int c4 = 0; c4 < 4; c4++) {
        float4 x, y;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w)
                     : "r"(r1 ^ (uint32_t)(16 * c4)));
        if (RA == 3) {  // rows of three fields: the first and third multiplied in FP32 first
            float4 z;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(z.x), "=f"(z.y), "=f"(z.z), "=f"(z.w)
                         : "r"(r3 ^ (uint32_t)(16 * c4)));
            x.x *= z.x;
            x.y *= z.y;
            x.z *= z.z;
            x.w *= z.w;
        }
        if (RA >= 2) {
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(y.x), "=f"(y.y), "=f"(y.z), "=f"(y.w)
                         : "r"(r2 ^ (uint32_t)(16 * c4)));
            tc::split2_prod_fast(x.x, y.x, x.y, y.y, v[2 * c4], v[8 + 2 * c4]);
            tc::split2_prod_fast(x.z, y.z, x.w, y.w, v[2 * c4 + 1], v[8 + 2 * c4 + 1]);
        } else {
            tc::split2_fast(x.x, x.y, v[2 * c4], v[8 + 2 * c4]);
            tc::split2_fast(x.z, x.w, v[2 * c4 + 1], v[8 + 2 * c4 + 1]);
        }
    }
}

template <int RA, int CA, int TEAMS>
__global__ void __launch_bounds__(tc_threads(TEAMS), 1)
    tc_contract_kernel(const __grid_constant__ CUtensorMap fmap, int nshell, int stage_bytes, int bbuf_bytes,
                       int slot_cap, int acc_max, int window, const TcCta* __restrict__ ctas, const TcGroup* __restrict__ groups,
                       const TcMTile* __restrict__ mtiles, const int4* __restrict__ runs,
                       const short4* __restrict__ rowf, const short4* __restrict__ colf, double* __restrict__ partial,
                       int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* s_d = base;                                        // kTcStages x stage_bytes (1024-aligned)
    uint8_t* s_b = s_d + kTcStages * stage_bytes;               // [slot][hi, lo] x bbuf_bytes
    float* s_acc = (float*)(s_b + 2 * slot_cap * bbuf_bytes);   // [acc_max cols][128 rows]
    short4* s_rowf = (short4*)(s_acc + (size_t)acc_max * 128);  // [kTcMaxMT][128]
    short4* s_colf = s_rowf + kTcMaxMT * 128;                   // [kTcMaxCols]
    uint64_t* bars = (uint64_t*)(s_colf + kTcMaxCols);
    uint64_t* full = bars;                                      // [kTcStages]
    uint64_t* empty = full + kTcStages;                         // [kTcStages]
    uint64_t* produced = empty + kTcStages;                     // [kTcMaxSlots]
    uint64_t* mma_done = produced + kTcMaxSlots;                // [kTcMaxSlots]
    uint64_t* acc_ready = mma_done + kTcMaxSlots;
    uint64_t* acc_free = acc_ready + 1;
    uint64_t* drain = acc_free + 1;
    uint32_t* s_tmem = (uint32_t*)(drain + 1);
    volatile int* s_abort = (volatile int*)(s_tmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TcCta cta = ctas[blockIdx.x];
    const TcGroup grp = groups[cta.group];
    const int nch = (int)(cta.c1 - cta.c0);
    const int nmt = grp.nmt, ncol = grp.ncol, acc_cols = grp.acc_cols;
    constexpr int kTcThreads = tc_threads(TEAMS);
    constexpr int kProdWarps = TEAMS * kTcTeamWarps;
    // TMEM columns: accumulators [0, a0), then the A slots of nmt x 32 columns (hi 16 + lo 16 per M tile)
    const int a0 = (acc_cols + 31) / 32 * 32;
    const uint32_t slot_cols = (uint32_t)(nmt * 32);
    int nslots = (512 - a0) / (int)slot_cols;
    nslots = nslots < slot_cap ? nslots : slot_cap;  // >= 2: a0 <= 256 and nmt <= 4
    // Producer teams at work: at most nslots.  A team reuses a slot after the MMAs of chunk
    // i - nslots; the parity wait on that slot's barrier is unambiguous only if the slot's
    // use before that (chunk i - 2 nslots) is known complete, which the team's own previous
    // wait (chunk i - nteams - nslots, MMAs committed in chunk order) implies when
    // nteams <= nslots.
    const int nteams = nslots < TEAMS ? nslots : TEAMS;

    if (tid == 0) {
        for (int st = 0; st < kTcStages; st++) {
            tc::mbar_init(&full[st], 1);
            tc::mbar_init(&empty[st], kTcTeamWarps);
        }
        for (int b = 0; b < kTcMaxSlots; b++) {
            tc::mbar_init(&produced[b], kTcTeamWarps);  // one team writes a slot per chunk
            tc::mbar_init(&mma_done[b], nmt);  // one commit per issuer
        }
        tc::mbar_init(acc_ready, nmt);
        tc::mbar_init(acc_free, kTcTeamWarps);  // the team that owns a window's last chunk drains it
        tc::mbar_init(drain, nmt);
        tc::mbar_fence_init();
        *s_abort = 0;
    }
    for (int i = tid; i < kTcMaxMT * 128; i += kTcThreads) {
        const int m = i >> 7;
        s_rowf[i] = m < nmt ? rowf[mtiles[grp.mt_off + m].row_off + (i & 127)] : make_short4(0, 0, 0, 0);
    }
    for (int i = tid; i < kTcMaxCols; i += kTcThreads) s_colf[i] = i < ncol ? colf[grp.col_off + i] : make_short4(-1, -1, -1, -1);
    for (int i = tid; i < acc_cols * 128; i += kTcThreads) s_acc[i] = 0.f;
    if (warp == kProdWarps) {
        tc::tmem_alloc(s_tmem, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;
    const uint32_t stage_tx = (uint32_t)nshell * kTcChunk * 4;

    if (warp >= kProdWarps) {
        // ------------------------------------------------------------- MMA issuers and the loads
        const int m = warp - kProdWarps;
        const bool el = tc::elect_one();
        const int pre = kTcStages < nch ? kTcStages : nch;
        int c = pre;  // next chunk to load
        // the TMA loads come from an issuer warp without an M tile when there is one, else from issuer 0
        const int loader = nmt < kTcIssuers ? kTcIssuers - 1 : 0;
        if (m == loader) {
            if (el && nch > 0) {
                tc::prefetch_tensormap(&fmap);
                for (int c0 = 0; c0 < pre; c0++) {
                    tc::mbar_arrive_expect_tx(&full[c0], stage_tx);
                    tc::tma_load_2d(s_d + c0 * stage_bytes, &fmap, 0, (int)((cta.c0 + c0) * nshell), &full[c0]);
                }
            }
            __syncwarp();
        }
        if (m < nmt) {
            uint32_t r_d[kTcMaxRunsMt], r_b[kTcMaxRunsMt], r_id[kTcMaxRunsMt];
            const TcMTile mt = mtiles[grp.mt_off + m];
            const int nrun = mt.nrun;
#pragma unroll
            for (int r = 0; r < kTcMaxRunsMt; r++) {
                const int4 run = r < nrun ? runs[mt.run_off + r] : make_int4(0, 16, 0, 0);  // n0, nn, acc col
                r_d[r] = tmem + (uint32_t)run.z;
                r_b[r] = (uint32_t)(run.x / 8) * kSBO;
                r_id[r] = tc::idesc_bf16(128, run.y);
            }
            // 64-bit descriptor = start address | LBO | (SBO, sm_100 descriptor version) << 32
            const uint64_t desc_k = ((uint64_t)((kSBO >> 4) | (1u << 14)) << 32) | (uint64_t)((kLBO >> 4) << 16);
            TcWindow win(0, window);
            int lst = 0;
            uint32_t lph = 0;  // stage and phase of empty[] that frees the stage for chunk c
            int slot = 0;
            uint32_t ph = 0;  // phase of produced[slot] for chunk i
            for (int i = 0; i < nch; i++) {
                win.advance_to(i, window);
                const bool wstart = i == win.end - window + 1;
                if (!tc::mbar_wait_warp(&produced[slot], ph, s_abort)) break;
                if (wstart && win.index > 0 && !tc::mbar_wait_warp(acc_free, (uint32_t)((win.index - 1) & 1), s_abort))
                    break;
                tc::fence_after_sync();
                if (el) {
                    const uint32_t a = tmem + (uint32_t)a0 + (uint32_t)slot * slot_cols + (uint32_t)(m * 32);
                    const uint32_t bh = tc::smem_u32(s_b + (2 * slot) * bbuf_bytes);
                    const uint32_t bl = tc::smem_u32(s_b + (2 * slot + 1) * bbuf_bytes);
                    const uint32_t first = wstart ? 0u : 1u;
#pragma unroll
                    for (int r = 0; r < kTcMaxRunsMt; r++) {
                        if (r < nrun) {
#pragma unroll
                            for (int ks = 0; ks < kTcChunk / 16; ks++) {
                                const uint32_t bo = r_b[r] + (uint32_t)ks * 2 * kLBO;
                                const uint64_t dh = desc_k | (uint64_t)(((bh + bo) >> 4) & 0x3FFFu);
                                const uint64_t dl = desc_k | (uint64_t)(((bl + bo) >> 4) & 0x3FFFu);
                                const uint32_t ak = a + (uint32_t)(ks * 16);  // hi; lo at + 8
                                tc::mma_ts(r_d[r], ak, dh, r_id[r], ks == 0 ? first : 1u);  // hi x hi
                                tc::mma_ts(r_d[r], ak, dl, r_id[r], 1u);                    // hi x lo
                                tc::mma_ts(r_d[r], ak + 8, dh, r_id[r], 1u);                // lo x hi
                            }
                        }
                    }
                    tc::mma_commit(&mma_done[slot]);
                    if (i == win.end || i == nch - 1) tc::mma_commit(acc_ready);
                }
                __syncwarp();
                if (m == loader && c < nch) {
                    // the stage held chunk c - kTcStages = i, released by its team before produced[]
                    if (!tc::mbar_wait_warp(&empty[lst], lph, s_abort)) break;
                    if (el) {
                        tc::mbar_arrive_expect_tx(&full[lst], stage_tx);
                        tc::tma_load_2d(s_d + lst * stage_bytes, &fmap, 0, (int)((cta.c0 + c) * nshell), &full[lst]);
                    }
                    __syncwarp();
                    c++;
                    if (++lst == kTcStages) {
                        lst = 0;
                        lph ^= 1u;
                    }
                }
                if (++slot == nslots) {
                    slot = 0;
                    ph ^= 1u;
                }
            }
            // every MMA this issuer started completes before the columns are freed
            if (el && nch > 0) tc::mma_commit(drain);
            __syncwarp();
        }
        if (m == loader && m >= nmt) {
            // a warp that only loads: refill each stage once its team has released it
            int lst = 0;
            uint32_t lph = 0;  // stage and phase of empty[] that frees the stage for chunk c
            for (; c < nch; c++) {
                if (!tc::mbar_wait_warp(&empty[lst], lph, s_abort)) break;
                if (el) {
                    tc::mbar_arrive_expect_tx(&full[lst], stage_tx);
                    tc::tma_load_2d(s_d + lst * stage_bytes, &fmap, 0, (int)((cta.c0 + c) * nshell), &full[lst]);
                }
                __syncwarp();
                if (++lst == kTcStages) {
                    lst = 0;
                    lph ^= 1u;
                }
            }
        }
        if (m == loader && el) {
            // every load started (chunks 0 .. c - 1) lands before the block exits
            volatile int no_abort = 0;
            for (int s2 = 0; s2 < kTcStages && s2 < c; s2++) {
                const int last = s2 + kTcStages * ((c - 1 - s2) / kTcStages);
                tc::mbar_wait(&full[s2], (uint32_t)((last / kTcStages) & 1), &no_abort);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------- producers
        const int team = warp / kTcTeamWarps, tw = warp % kTcTeamWarps;
        const int q = tw & 3, half = tw >> 2;  // lane quadrant, 16-cell half of the chunk
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        const int row = 32 * q + lane;
        // this lane's row factors in each M tile (in-range shells)
        uint32_t key1[kTcMaxMT], key2[kTcMaxMT], key3[RA == 3 ? kTcMaxMT : 1];
#pragma unroll
        for (int m = 0; m < kTcMaxMT; m++) {
            const short4 f = s_rowf[m * 128 + row];
            key1[m] = tc_row_key(f.x) ^ (uint32_t)(64 * half);
            key2[m] = tc_row_key(RA >= 2 ? f.y : 0) ^ (uint32_t)(64 * half);
            if (RA == 3) key3[m] = tc_row_key(f.z) ^ (uint32_t)(64 * half);
        }
        const int ttid = tid % (kTcTeamWarps * 32);
        // stages team, team + nteams, ... in turn; slots i mod nslots
        const uint32_t abase0 = tmem + lane_base + (uint32_t)a0 + (uint32_t)(16 * half);
        const uint32_t Bbase = tc::smem_u32(s_b);
        const uint32_t sd0 = tc::smem_u32(s_d);
        // this thread's first B item (column n, 8-cell group kg), fixed for every chunk
        const int nbitems = ncol * (kTcChunk / 8);
        int b_key1 = -1, b_key2 = 0, b_key3 = 0;
        uint32_t b_off = 0;
        if (ttid < nbitems) {
            const int kg = ttid / ncol, n = ttid - kg * ncol;
            const short4 f = s_colf[n];
            if (f.x >= 0) {
                b_key1 = (int)(tc_row_key(f.x) ^ (uint32_t)(2 * kg * 16));
                b_key2 = (int)(tc_row_key(CA >= 2 ? f.y : 0) ^ (uint32_t)(2 * kg * 16));
                b_key3 = (int)(tc_row_key(CA == 3 ? f.z : 0) ^ (uint32_t)(2 * kg * 16));
            }
            b_off = (uint32_t)(n / 8) * kSBO + (uint32_t)kg * kLBO + (uint32_t)(n % 8) * 16;
        }
        int st = team;
        uint32_t ph_full = 0;
        TcWindow win(team, window);
        for (int i = team < nteams ? team : nch; i < nch; i += nteams) {
            if (!tc::mbar_wait_warp(&full[st], ph_full, s_abort)) break;
            const int slot = i % nslots, use = i / nslots;  // slot and its use count
            if (use > 0) {
                // the MMAs of chunk i - nslots have read the slot
                if (!tc::mbar_wait_warp(&mma_done[slot], (uint32_t)((use - 1) & 1), s_abort)) break;
            }
            const uint32_t abase = abase0 + (uint32_t)slot * slot_cols;
            const uint32_t Bh = Bbase + (uint32_t)(2 * slot * bbuf_bytes);
            const uint32_t Bl = Bh + (uint32_t)bbuf_bytes;
            tc::fence_after_sync();
            const uint32_t D = sd0 + (uint32_t)(st * stage_bytes);
            // A operand: this lane's row in each M tile, cells [16 half, 16 half + 16), hi and lo in one
            // 16-column store; the B item (column n, 8-cell group kg -> one 16-byte core-matrix row of
            // hi and of lo) after the first tile, while its stores drain
#pragma unroll
            for (int m = 0; m < kTcMaxMT; m++) {
                if (m < nmt) {
                    uint32_t v[16];
                    tc_row_products<RA>(D + key1[m], D + key2[m], RA == 3 ? D + key3[RA == 3 ? m : 0] : 0u, v);
                    tc::tmem_st16(abase + (uint32_t)(m * 32), v);
                }
                if (m == 0 && ttid < nbitems) tc_b_item<CA>(D, b_key1, b_key2, b_key3, Bh + b_off, Bl + b_off);
            }
            for (int it = ttid + kTcTeamWarps * 32; it < nbitems; it += kTcTeamWarps * 32) {
                const int kg = it / ncol, n = it - kg * ncol;
                const short4 f = s_colf[n];
                const uint32_t off = (uint32_t)(n / 8) * kSBO + (uint32_t)kg * kLBO + (uint32_t)(n % 8) * 16;
                tc_b_item<CA>(D, f.x >= 0 ? (int)(tc_row_key(f.x) ^ (uint32_t)(2 * kg * 16)) : -1,
                              (int)(tc_row_key(CA >= 2 && f.x >= 0 ? f.y : 0) ^ (uint32_t)(2 * kg * 16)),
                              (int)(tc_row_key(CA == 3 && f.x >= 0 ? f.z : 0) ^ (uint32_t)(2 * kg * 16)), Bh + off,
                              Bl + off);
            }
            tc::fence_proxy_async_smem();
            tc::tmem_st_wait();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(&empty[st]);
                tc::mbar_arrive(&produced[slot]);
            }
            st += nteams;
            if (st >= kTcStages) {
                st -= kTcStages;
                ph_full ^= 1u;
            }
            // drain the accumulators after the last chunk of a window
            win.advance_to(i, window);
            if (i == win.end || i == nch - 1) {
                if (!tc::mbar_wait_warp(acc_ready, (uint32_t)(win.index & 1), s_abort)) break;
                tc::fence_after_sync();
                for (int g = half; g < acc_cols / 16; g += 2) {
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
    if (warp == kProdWarps) {
        // every issuer committed its MMAs to `drain`; wait for them before freeing the columns
        volatile int no_abort2 = 0;
        if (nch > 0 && lane == 0) tc::mbar_wait(drain, 0, &no_abort2);
        __syncwarp();
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
    int acc_max = 256, slot_cap = 2;
    int teams = 2;  // producer teams per block
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
           kTcMaxMT * 128 * 8 + kTcMaxCols * 8 + (2 * kTcStages + 2 * kTcMaxSlots + 3) * 8 + 64;
}

// Sorted 16-column blocks of one M tile -> runs (first block, block count), at most
// kTcMaxRunsMt of them: the narrowest gaps are filled (their sums are computed and unused).
static std::vector<std::pair<int, int>> tc_runs(const std::set<int>& blocks) {
    std::vector<std::pair<int, int>> rr;
    for (int b : blocks) {
        if (!rr.empty() && rr.back().first + rr.back().second == b) rr.back().second++;
        else rr.push_back({b, 1});
    }
    while ((int)rr.size() > kTcMaxRunsMt) {
        size_t best = 0;
        int gap = 1 << 30;
        for (size_t k = 0; k + 1 < rr.size(); k++) {
            const int g = rr[k + 1].first - (rr[k].first + rr[k].second);
            if (g < gap) {
                gap = g;
                best = k;
            }
        }
        rr[best].second = rr[best + 1].first + rr[best + 1].second - rr[best].first;
        rr.erase(rr.begin() + (long)best + 1);
    }
    return rr;
}

// Build the groups: 32-row blocks of rows sorted by column span, 128-row M tiles,
// 16-column blocks.
// Host tables of the contraction: groups of M-tile instances, their accumulator
// runs, the row and column factors, the blocks (group, chunk range) and the bin
// map.  Fills t's host fields (ra, ca, nshell, ngroups, ctas, executed flops)
// and h; touches no device.
struct TcTables {
    std::vector<TcGroup> groups;
    std::vector<TcMTile> mtiles;
    std::vector<int4> runs;
    std::vector<short4> rowf, colf;
    std::vector<int4> binmap;
};

static poly_status tc_launch_shape(const PsPlan* p, const std::vector<TcGroup>& groups, TcState* t);

static poly_status tc_build_tables(const PsPlan* p, TcState* t, TcTables& h) {
    const int n = p->order;
    t->ra = n >= 6 ? 3 : (n >= 3 ? 2 : 1);
    t->ca = n - t->ra;
    t->nshell = p->nfield;  // field rows staged per chunk: nshell, or 2 nshell for a multipole plan
    const bool ra2 = t->ra >= 2;
    // a multipole plan's first leg reads the Legendre-weighted field of its shell (slot k1 - 1 + nshell)
    const int shift = p->ell > 0 ? p->nshell : 0;

    const int max_mt = std::max(1, std::min(kTcMaxMT, p->tc_max_mt));  // M tiles per group (tunable)
    using CKey = std::array<int, 3>;  // column factors (shells from 1; -1: none)
    using RKey = std::array<int, 3>;  // row factors (shells from 1; -1: none)
    auto rkey = [&](const int32_t* b) { return RKey{b[0], t->ra >= 2 ? b[1] : -1, t->ra == 3 ? b[2] : -1}; };
    auto ckey = [&](const int32_t* b) {
        return CKey{b[t->ra], t->ca >= 2 ? b[t->ra + 1] : -1, t->ca == 3 ? b[t->ra + 2] : -1};
    };
    std::map<RKey, std::set<CKey>> rows;
    std::set<CKey> allcols;
    for (int64_t i = 0; i < p->nbins; i++) {
        rows[rkey(&p->bins[i * n])].insert(ckey(&p->bins[i * n]));
        allcols.insert(ckey(&p->bins[i * n]));
    }
    std::map<CKey, int> gcol;
    for (auto& c : allcols) gcol[c] = (int)gcol.size();
    // accumulator columns per group: a multipole plan stages twice the rows per chunk, so its groups
    // are held to what still fits shared memory next to the TMA stages and three A/B slots (two if
    // three leave no room)
    int acc_budget = kTcAccMax;
    if (p->ell > 0) {
        const int stage = (p->nfield * 128 + 1023) / 1024 * 1024;
        const int cols = std::min(kTcMaxCols, ((int)allcols.size() + 15) / 16 * 16);
        for (int slots = 3; slots >= 2; slots--) {
            const long room = 227L * 1024 - (long)tc_smem_bytes(stage, cols * kTcChunk * 2, slots, 0);
            acc_budget = (int)std::min<long>(kTcAccMax, std::max<long>(0, room / (128 * 4)) / 16 * 16);
            if (acc_budget >= 64) break;
        }
        if (acc_budget < 16) return POLY_ERR_UNSUPPORTED;
    }
    struct Row {
        bool valid;
        RKey key;                 // shells (from 1) of the row factors; in range also for padding rows
        std::vector<int> cols;    // global column indices, sorted (empty for padding rows)
    };
    // A producer warp takes 32 rows.  Pair rows: the rows of one octet of 8
    // consecutive k1, sorted by (k2, k1) and cut in 32s, so that a warp's rows
    // use at most 8 consecutive k1 and a few consecutive k2 (the factor reads are
    // bank-conflict-free broadcasts).  Single-field rows: 32 consecutive k1.
    // Lanes without a row repeat the block's first row (their accumulator rows are
    // never read).
    const int ns = p->nshell;
    std::map<int, std::vector<std::pair<RKey, const std::set<CKey>*>>> octets;
    for (auto& kv : rows) {
        const int k1 = kv.first[0];
        octets[ra2 ? (k1 - 1) / kTcRowOctet : (k1 - 1) / 32].push_back({kv.first, &kv.second});
    }
    std::vector<std::vector<Row>> blocks;
    for (auto& ov : octets) {
        auto& lst = ov.second;
        std::sort(lst.begin(), lst.end(), [](const auto& x, const auto& y) {
            return std::make_tuple(x.first[1], x.first[2], x.first[0]) < std::make_tuple(y.first[1], y.first[2], y.first[0]);
        });
        for (size_t t = 0; t < lst.size(); t += 32) {
            std::vector<Row> blk(32);
            for (size_t l = 0; l < 32; l++) {
                if (t + l < lst.size()) {
                    Row& r = blk[l];
                    r.valid = true;
                    r.key = lst[t + l].first;
                    for (auto& c : *lst[t + l].second) r.cols.push_back(gcol[c]);
                    std::sort(r.cols.begin(), r.cols.end());
                } else {
                    blk[l] = Row{false, lst[t].first, {}};
                }
            }
            blocks.push_back(std::move(blk));
        }
    }
    (void)ns;
    std::vector<std::pair<std::pair<int, int>, const std::vector<Row>*>> bl;  // (column span, block)
    for (auto& blk : blocks) {
        int lo = 1 << 30, hi = -1;
        for (const Row& r : blk)
            if (r.valid) {
                lo = std::min(lo, r.cols.front());
                hi = std::max(hi, r.cols.back());
            }
        bl.push_back({{lo, hi}, &blk});
    }
    std::stable_sort(bl.begin(), bl.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    std::vector<Row> rl;
    for (auto& b : bl) rl.insert(rl.end(), b.second->begin(), b.second->end());
    while (rl.size() % 128) rl.push_back(Row{false, RKey{1, t->ra >= 2 ? 1 : -1, t->ra == 3 ? 1 : -1}, {}});
    const int nmt_total = (int)(rl.size() / 128);
    auto mt_cols = [&](int m) {
        std::set<int> s;
        for (size_t r = (size_t)m * 128; r < (size_t)(m + 1) * 128; r++) s.insert(rl[r].cols.begin(), rl[r].cols.end());
        return s;
    };
    // Tile instances: an M tile with more than kTcMaxCols columns (the trispectrum's pair
    // columns) is split into instances over ranges of its columns; each instance is placed
    // in a group on its own, and its products are formed again there.
    struct Inst {
        int m;
        std::vector<int> cols;  // global column indices, sorted
    };
    std::vector<Inst> inst;
    for (int m = 0; m < nmt_total; m++) {
        auto sc = mt_cols(m);
        std::vector<int> v(sc.begin(), sc.end());
        const int np = std::max(1, (int)((v.size() + kTcMaxCols - 1) / kTcMaxCols));
        for (int k = 0; k < np; k++)
            inst.push_back(Inst{m, std::vector<int>(v.begin() + (long)(v.size() * k / np),
                                                    v.begin() + (long)(v.size() * (k + 1) / np))});
    }
    const int ninst = (int)inst.size();
    // group consecutive instances; a group is valid when its local column list (<= 256)
    // and its accumulator columns (<= 256) fit
    struct GroupPlan {
        int m0, m1;              // instances [m0, m1)
        std::vector<int> local;  // global col indices, sorted, padded later
        int acc;
    };
    auto plan_group = [&](int m0, int m1, GroupPlan& g) -> bool {
        std::set<int> u;
        for (int i = m0; i < m1; i++) u.insert(inst[i].cols.begin(), inst[i].cols.end());
        g.m0 = m0;
        g.m1 = m1;
        g.local.assign(u.begin(), u.end());
        if ((int)g.local.size() > kTcMaxCols) return false;
        std::map<int, int> lidx;
        for (size_t i = 0; i < g.local.size(); i++) lidx[g.local[i]] = (int)i;
        g.acc = 0;
        for (int i = m0; i < m1; i++) {
            std::set<int> cb;
            for (int c : inst[i].cols) cb.insert(lidx[c] / 16);
            for (auto& rr : tc_runs(cb)) g.acc += 16 * rr.second;
        }
        return g.acc <= acc_budget && (m1 - m0) <= max_mt;
    };
    // groups: the fewest that fit, with the instances spread evenly over them (each group
    // pays a fixed per-chunk cost for loading and synchronisation)
    std::vector<GroupPlan> gplans;
    int ngroups = (ninst + max_mt - 1) / max_mt;
    while (true) {
        gplans.clear();
        bool ok = true;
        for (int g = 0; g < ngroups && ok; g++) {
            const int m0 = (int)((long long)ninst * g / ngroups), m1 = (int)((long long)ninst * (g + 1) / ngroups);
            GroupPlan gp;
            if (m1 <= m0) continue;
            ok = plan_group(m0, m1, gp);
            gplans.push_back(gp);
        }
        if (ok) break;
        if (ngroups >= ninst) return POLY_ERR_UNSUPPORTED;  // a single instance does not fit
        ngroups++;
    }
    t->ngroups = (int)gplans.size();
    // tables
    std::vector<TcGroup>& groups = h.groups;
    std::vector<TcMTile>& mtiles = h.mtiles;
    std::vector<int4>& runs = h.runs;
    std::vector<short4>& rowf = h.rowf;
    std::vector<short4>& colf = h.colf;
    // (row, col) keys -> (group, slot); shells (from 1, or -1 for none) packed one per byte (the keys
    // hold shell numbers, not field slots, so the weighted slots of a multipole plan do not enter them)
    static_assert(kPsMaxShells + 1 < 256, "a shell number + 1 must fit one byte of the packed key");
    if (p->nshell > kPsMaxShells) return POLY_ERR_UNSUPPORTED;
    auto pack = [](const RKey& r, const CKey& c) {
        return (uint64_t)(r[0] + 1) | (uint64_t)(r[1] + 1) << 8 | (uint64_t)(r[2] + 1) << 16 |
               (uint64_t)(c[0] + 1) << 24 | (uint64_t)(c[1] + 1) << 32 | (uint64_t)(c[2] + 1) << 40;
    };
    std::unordered_map<uint64_t, std::pair<int, int>> slot_of;
    slot_of.reserve((size_t)p->nbins * 2);
    std::vector<CKey> gcol_key(gcol.size());
    for (auto& kv : gcol) gcol_key[kv.second] = kv.first;
    double work_cells = 0;
    std::vector<double> gwork;
    for (int gi = 0; gi < t->ngroups; gi++) {
        const GroupPlan& gp = gplans[gi];
        TcGroup G{};
        G.mt_off = (int)mtiles.size();
        G.nmt = gp.m1 - gp.m0;  // instances of M tiles
        G.col_off = (int)colf.size();
        const int ncol = ((int)gp.local.size() + 15) / 16 * 16;
        G.ncol = ncol;
        std::map<int, int> lidx;
        for (size_t i = 0; i < gp.local.size(); i++) {
            lidx[gp.local[i]] = (int)i;
            const CKey& k = gcol_key[gp.local[i]];
            colf.push_back(make_short4((short)(k[0] - 1), (short)(k[1] > 0 ? k[1] - 1 : -1),
                                       (short)(k[2] > 0 ? k[2] - 1 : -1), (short)-1));
        }
        for (int i = (int)gp.local.size(); i < ncol; i++) colf.push_back(make_short4(-1, -1, -1, -1));
        int acc = 0;
        for (int ii = gp.m0; ii < gp.m1; ii++) {
            const Inst& in = inst[ii];
            const int m = in.m;
            TcMTile M{};
            M.row_off = (int)rowf.size();
            M.run_off = (int)runs.size();
            const size_t r0 = (size_t)m * 128, r1 = r0 + 128;
            for (size_t r = r0; r < r1; r++) {
                const RKey& k = rl[r].key;
                rowf.push_back(make_short4((short)(k[0] - 1 + shift), (short)(k[1] > 0 ? k[1] - 1 : -1),
                                           (short)(k[2] > 0 ? k[2] - 1 : -1), (short)-1));
            }
            std::set<int> cb;
            for (int c : in.cols) cb.insert(lidx[c] / 16);
            std::map<int, std::pair<int, int>> block_acc;  // block -> (run n0, acc col of run start)
            for (auto& rr : tc_runs(cb)) {
                const int n0 = rr.first * 16, nn = rr.second * 16;
                runs.push_back(make_int4(n0, nn, acc, ii - gp.m0));
                for (int q = rr.first; q < rr.first + rr.second; q++) block_acc[q] = {n0, acc};
                acc += nn;
            }
            M.nrun = (int)runs.size() - M.run_off;
            for (size_t r = r0; r < r1; r++)
                for (int c : rl[r].cols) {
                    if (!std::binary_search(in.cols.begin(), in.cols.end(), c)) continue;  // another instance's
                    const int lc = lidx[c];
                    auto ba = block_acc[lc / 16];
                    const int acc_col = ba.second + (lc - ba.first);
                    slot_of[pack(rl[r].key, gcol_key[c])] = {gi, acc_col * 128 + (int)(r - r0)};
                }
            mtiles.push_back(M);
        }
        G.acc_cols = acc;
        groups.push_back(G);
        // per-chunk cost in cycles: tensor pipe (3 MMAs x K/16 per 16 accumulator columns) or the
        // producers (a fixed loading and synchronisation cost plus a share per M tile), whichever is longer
        const double wk = std::max(3.0 * acc, 550.0 + 360.0 * G.nmt);
        gwork.push_back(wk);
        work_cells += wk;
        t->executed_flops_per_cell += 3.0 * 2.0 * 128.0 * acc;
    }
    // blocks: split each group's chunks in proportion to its work
    const int64_t ncell = (int64_t)p->N * p->N * p->N;
    const int64_t nchunks = (ncell + kTcChunk - 1) / kTcChunk;
    const int budget = std::max(p->sms * p->tc_cta_mult / 2, t->ngroups);
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
    std::vector<int4>& binmap = h.binmap;
    binmap.resize(p->nbins);
    for (int64_t i = 0; i < p->nbins; i++) {
        auto rk = rkey(&p->bins[i * n]);
        auto ck = ckey(&p->bins[i * n]);
        auto gs = slot_of.at(pack(rk, ck));
        binmap[i] = make_int4(first[gs.first], nsplit[gs.first], gs.second, 0);
    }
    return tc_launch_shape(p, h.groups, t);
}

// Launch shape of the contraction from the groups (host only): TMA stage bytes, B buffer
// bytes, accumulator columns, A/B slot cap, shared memory and the producer team count.
static poly_status tc_launch_shape(const PsPlan* p, const std::vector<TcGroup>& groups, TcState* t) {
    t->stage_bytes = (p->nfield * 128 + 1023) / 1024 * 1024;
    int maxcol = 16, maxacc = 16;
    for (auto& g : groups) {
        maxcol = std::max(maxcol, g.ncol);
        maxacc = std::max(maxacc, g.acc_cols);
    }
    t->bbuf_bytes = maxcol * kTcChunk * 2;
    t->acc_max = maxacc;
    t->slot_cap = kTcMaxSlots;  // B slots: as many as shared memory holds (the kernel also bounds them by TMEM)
    while (t->slot_cap > 2 && tc_smem_bytes(t->stage_bytes, t->bbuf_bytes, t->slot_cap, maxacc) > 227 * 1024)
        t->slot_cap--;
    t->smem_bytes = (int)tc_smem_bytes(t->stage_bytes, t->bbuf_bytes, t->slot_cap, maxacc);
    if (t->smem_bytes > 227 * 1024) return POLY_ERR_UNSUPPORTED;
    // a third producer team where every group has three A/B slots (the kernel's slot count:
    // what tensor memory holds beside the group's accumulators, at most slot_cap)
    int min_slots = t->slot_cap;
    for (auto& g : groups) min_slots = std::min(min_slots, (512 - (g.acc_cols + 31) / 32 * 32) / (g.nmt * 32));
    t->teams = min_slots >= 3 ? 3 : 2;
    return POLY_OK;
}

poly_status ps_tc_prepare(PsPlan* p) {
    if (p->is_double) return POLY_ERR_UNSUPPORTED;
    TcState* t = new (std::nothrow) TcState();
    if (!t) return POLY_ERR_ALLOC;
    p->tc = t;
    TcTables h;
    if (poly_status s0 = tc_build_tables(p, t, h)) return s0;
    const std::vector<TcGroup>& groups = h.groups;
    const int64_t ncell = (int64_t)p->N * p->N * p->N;
    auto up = [&](void** d, const void* src, size_t bytes) -> poly_status {
        poly_status s = ps_alloc(p, d, bytes);
        if (s) return s;
        return cudaMemcpy(*d, src, bytes, cudaMemcpyHostToDevice) ? POLY_ERR_CUDA : POLY_OK;
    };
    poly_status s;
    if ((s = up(&t->d_ctas, t->ctas.data(), t->ctas.size() * sizeof(TcCta))) ||
        (s = up(&t->d_groups, groups.data(), groups.size() * sizeof(TcGroup))) ||
        (s = up(&t->d_mtiles, h.mtiles.data(), h.mtiles.size() * sizeof(TcMTile))) ||
        (s = up(&t->d_runs, h.runs.data(), std::max<size_t>(1, h.runs.size()) * sizeof(int4))) ||
        (s = up(&t->d_rowf, h.rowf.data(), h.rowf.size() * sizeof(short4))) ||
        (s = up(&t->d_colf, h.colf.data(), h.colf.size() * sizeof(short4))) ||
        (s = up(&t->d_binmap, h.binmap.data(), std::max<size_t>(1, h.binmap.size()) * sizeof(int4))))
        return s;
    if ((s = ps_alloc(p, (void**)&t->d_partial, t->ctas.size() * (size_t)kTcAccMax * 128 * 8))) return s;
    if ((s = ps_alloc(p, (void**)&t->d_err, 16))) return s;
    if (cudaMemset(t->d_err, 0, 16)) return POLY_ERR_CUDA;
    // tensor map over the cell-tiled fields [ncell/32 * nfield rows][32 cells] fp32: one box = one 32-cell
    // chunk of every field slot (a contiguous block), 128-byte swizzle
    auto enc = get_encode();
    if (!enc) return POLY_ERR_UNSUPPORTED;
    cuuint64_t gdim[2] = {(cuuint64_t)kTcChunk, (cuuint64_t)(ncell / kTcChunk) * (cuuint64_t)p->nfield};
    cuuint64_t gstride[1] = {(cuuint64_t)kTcChunk * 4};
    cuuint32_t box[2] = {(cuuint32_t)kTcChunk, (cuuint32_t)p->nfield};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&t->fmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->d_fields, gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return POLY_ERR_CUDA;
    // Accumulation window (chunks of 32 cells summed in FP32 in tensor memory before a drain).
    // The tensor-core FP32 accumulation error grows with the window; at 256^3 the largest
    // error over the split-BF16 scale is 1.3e-6 for the bispectrum at 128 chunks (6e-7 at 64;
    // the contraction takes 6.54 ms instead of 6.67), but 1.5e-5 for the trispectrum
    // (products of four fields) at 64 chunks, 5.9e-6 at 16.
    t->window = p->order >= 4 ? 16 : 128;
    const char* w = getenv("POLY_TC_WINDOW");
    if (w && atoi(w) > 0) t->window = atoi(w);
    return POLY_OK;
}

static int diag_tc_tables(int N, int order, const double* edges, int nshell, unsigned flags, int ell, int sms,
                          int max_mt, int cta_mult, int64_t* sizes, int64_t* ctas, int32_t* groups, int32_t* mtiles,
                          int32_t* runs, int16_t* rowf, int16_t* colf, int32_t* binmap) {
    if (!sizes || sms < 1 || max_mt < 1 || cta_mult < 1) return POLY_ERR_ARG;
    PsPlan hp;  // host tables only: no device call, no device memory
    std::vector<short> lines;
    if (poly_status s = ps_plan_host_tables(&hp, N, 1.0, order, nshell, edges, POLY_SPLIT_BF16, flags, ell, lines))
        return s;
    hp.sms = sms;
    hp.tc_max_mt = max_mt;
    hp.tc_cta_mult = cta_mult;
    TcState t;
    TcTables h;
    if (poly_status s = tc_build_tables(&hp, &t, h)) return s;
    const int64_t n[9] = {hp.nbins, (int64_t)t.ctas.size(), (int64_t)h.groups.size(), (int64_t)h.mtiles.size(),
                          (int64_t)h.runs.size(), (int64_t)h.rowf.size(), (int64_t)h.colf.size(), t.teams, t.slot_cap};
    for (int i = 0; i < 9; i++) sizes[i] = n[i];
    for (size_t i = 0; ctas && i < t.ctas.size(); i++) {
        ctas[3 * i] = t.ctas[i].group;
        ctas[3 * i + 1] = t.ctas[i].c0;
        ctas[3 * i + 2] = t.ctas[i].c1;
    }
    for (size_t i = 0; groups && i < h.groups.size(); i++) {
        const TcGroup& g = h.groups[i];
        const int32_t v[5] = {g.mt_off, g.nmt, g.col_off, g.ncol, g.acc_cols};
        std::memcpy(groups + 5 * i, v, sizeof v);
    }
    for (size_t i = 0; mtiles && i < h.mtiles.size(); i++) {
        mtiles[3 * i] = h.mtiles[i].row_off;
        mtiles[3 * i + 1] = h.mtiles[i].run_off;
        mtiles[3 * i + 2] = h.mtiles[i].nrun;
    }
    for (size_t i = 0; runs && i < h.runs.size(); i++) {
        const int32_t v[4] = {h.runs[i].x, h.runs[i].y, h.runs[i].z, h.runs[i].w};
        std::memcpy(runs + 4 * i, v, sizeof v);
    }
    for (size_t i = 0; rowf && i < h.rowf.size(); i++) {
        rowf[3 * i] = h.rowf[i].x;
        rowf[3 * i + 1] = h.rowf[i].y;
        rowf[3 * i + 2] = h.rowf[i].z;
    }
    for (size_t i = 0; colf && i < h.colf.size(); i++) {
        colf[3 * i] = h.colf[i].x;
        colf[3 * i + 1] = h.colf[i].y;
        colf[3 * i + 2] = h.colf[i].z;
    }
    for (size_t i = 0; binmap && i < h.binmap.size(); i++) {
        binmap[3 * i] = h.binmap[i].x;
        binmap[3 * i + 1] = h.binmap[i].y;
        binmap[3 * i + 2] = h.binmap[i].z;
    }
    return POLY_OK;
}

extern "C" int poly_diag_tc_tables(int N, int order, const double* edges, int nshell, unsigned flags, int ell,
                                   int sms, int max_mt, int cta_mult, int64_t* sizes, int64_t* ctas, int32_t* groups,
                                   int32_t* mtiles, int32_t* runs, int16_t* rowf, int16_t* colf, int32_t* binmap) {
    try {
        return diag_tc_tables(N, order, edges, nshell, flags, ell, sms, max_mt, cta_mult, sizes, ctas, groups, mtiles,
                              runs, rowf, colf, binmap);
    } catch (const std::bad_alloc&) {
        return POLY_ERR_ALLOC;
    }
}

poly_status ps_tc_sums(PsPlan* p, cudaStream_t st) {
    TcState* t = p->tc;
    if (!t) return POLY_ERR_UNSUPPORTED;
    cudaError_t e;
    auto launch = [&](auto kern, int threads) -> cudaError_t {
        cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, t->smem_bytes);
        if (e2) return e2;
        kern<<<(unsigned)t->ctas.size(), threads, t->smem_bytes, st>>>(
            t->fmap, t->nshell, t->stage_bytes, t->bbuf_bytes, t->slot_cap, t->acc_max, t->window, (const TcCta*)t->d_ctas,
            (const TcGroup*)t->d_groups, (const TcMTile*)t->d_mtiles, (const int4*)t->d_runs,
            (const short4*)t->d_rowf, (const short4*)t->d_colf, t->d_partial, t->d_err);
        return cudaGetLastError();
    };
    auto launch_teams = [&](auto k2, auto k3) { return t->teams == 3 ? launch(k3, tc_threads(3)) : launch(k2, tc_threads(2)); };
    if (t->ra == 2 && t->ca == 1) e = launch_teams(tc_contract_kernel<2, 1, 2>, tc_contract_kernel<2, 1, 3>);
    else if (t->ra == 2 && t->ca == 2) e = launch_teams(tc_contract_kernel<2, 2, 2>, tc_contract_kernel<2, 2, 3>);
    else if (t->ra == 2 && t->ca == 3) e = launch_teams(tc_contract_kernel<2, 3, 2>, tc_contract_kernel<2, 3, 3>);
    else if (t->ra == 3 && t->ca == 3) e = launch_teams(tc_contract_kernel<3, 3, 2>, tc_contract_kernel<3, 3, 3>);
    else e = launch_teams(tc_contract_kernel<1, 1, 2>, tc_contract_kernel<1, 1, 3>);
    if (e) return POLY_ERR_CUDA;
    if (p->timing) cudaEventRecord(p->ev[3], st);
    const int blocks = (int)std::min<int64_t>((p->nbins + 255) / 256, 4096);
    tc_reduce_kernel<<<std::max(1, blocks), 256, 0, st>>>(t->d_partial, (const int4*)t->d_binmap, p->nbins, p->d_S);
    p->launches += 2;
    return cudaGetLastError() ? POLY_ERR_CUDA : POLY_OK;
}

void ps_tc_free(PsPlan* p) {
    if (TcState* t = p->tc) {
        for (void* d : {t->d_ctas, t->d_groups, t->d_mtiles, t->d_runs, t->d_rowf, t->d_colf, t->d_binmap,
                        (void*)t->d_partial, (void*)t->d_err})
            ps_free(p, d);
    }
    delete p->tc;
    p->tc = nullptr;
}

poly_status ps_check_device_error(PsPlan* p) {
    if (ps_adj_device_error(p)) return POLY_ERR_TIMEOUT;
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
