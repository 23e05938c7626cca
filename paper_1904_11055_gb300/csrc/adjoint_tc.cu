// Tensor-core form of the adjoint's per-cell contraction for the bispectrum
// (n = 3, split-BF16 plans):
//   G_m(x) = sum_{(i, j)} W_m[i][j] D_i(x) D_j(x)
//          = sum_j D_j(x) T_{m,j}(x),   T_{m,j}(x) = sum_i W_m[i][j] D_i(x),
// where W_m[i][j] = w_e for the entry e = (m, i, j) of the adjoint (i <= j:
// the other two shells of a bin that contains m; w_e = sum g_b / count_b).
// T is a GEMM over the shells: M = 128 cells (TMEM lanes), K = the shells
// (A = D^T, split into bf16 hi + lo and written to TMEM), N = the (m, j)
// columns (B = W^T, hi + lo, resident in shared memory in the K-major
// core-matrix layout).  hi.hi + hi.lo + lo.hi products accumulate in FP32 in
// TMEM over the (few) K steps; the epilogue reduces each row against the cell's
// own D_j: G_m(x) = sum over m's columns of D_j(x) T[x][(m, j)].
//
// Columns come in chunks of 16: chunk (m, jb) holds j = 16 jb .. 16 jb + 15
// (columns of j's that m has no entry for carry zero weights), so within a
// chunk j is a fixed offset and the epilogue reads the 16 D_j of its cell at
// fixed shared-memory offsets.  A chunk is kept only where m has an entry.
//
// A group of m's holds their chunks in at most (512 - K) / 2 columns.  A block
// owns a pair of groups (members 0 and 1, each with its own half of TMEM next
// to A) and a range of 128-cell tiles; both members use the same A.  A tile's
// fields are four contiguous blocks of the cell-tiled layout; one thread of the
// MMA warp brings them into shared memory with bulk copies, two tiles ahead,
// rows padded with zeros up to K.  Eight cell warps (two per TMEM lane
// quadrant) write A and run the epilogues, each over one half of a member's
// m's; the MMA warp issues the MMAs.  Per tile: member 1's MMAs run while the
// cell warps reduce member 0; then the cell warps write the next tile's A, and
// the next tile's member-0 MMAs run while they reduce member 1.
#include <cuda.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "plan_internal.h"
#include "tc.cuh"

namespace ps {

constexpr int kAtCells = 128;                       // cells per tile (TMEM lanes)
constexpr int kAtCellWarps = 8;                     // two per lane quadrant
constexpr int kAtThreads = 32 * kAtCellWarps + 32;  // + the MMA warp
constexpr int kAtMaxRuns = 2;                       // N runs of <= 256 columns per group
constexpr int kAtMaxK = 128;                        // padded shell count (K) at most
constexpr int kAtChunk = 16;                        // columns per chunk (one j block)
constexpr int kAtDBufs = 3;                         // field tiles in flight (t in its epilogue, t + 1, t + 2)

struct AtGroup {
    int chunk_off, nchunk;    // chunks [chunk_off, chunk_off + nchunk) of the chunk table
    int hsplit;               // chunks [0, hsplit) hold the first half of the m's, [hsplit, nchunk) the rest
    int b_off;                // byte offset of the group's B (hi) in the B arrays
    int kmask[kAtMaxRuns];    // per run: bit k set when K block k (16 shells) has a nonzero weight
};

// B position of each entry: byte offset within the B arrays (-1: the entry has no column)
__global__ void at_scatter_kernel(const float* __restrict__ w, const int* __restrict__ pos, int nent,
                                  uint16_t* __restrict__ bhi, uint16_t* __restrict__ blo) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nent; e += gridDim.x * blockDim.x) {
        const int p = pos[e];
        if (p < 0) continue;
        const float v = w[e];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        bhi[p / 2] = *reinterpret_cast<const uint16_t*>(&h);
        blo[p / 2] = *reinterpret_cast<const uint16_t*>(&l);
    }
}

// chunk[c]: bits 0-7 jb, bits 8-15 m, bit 16: last chunk of its m.
// D: cell-tiled fields, [cell / 32][nshell][cell % 32]; ncell a multiple of 32.
// A block takes the pair of groups (2 pr, 2 pr + 1) (the second may be absent); acap: TMEM columns of one
// accumulator buffer (member b at column b * acap; A at 512 - kp).
__global__ void __launch_bounds__(kAtThreads, 1)
    at_contract_kernel(const float* __restrict__ D, int nshell, int kp, int acap, int64_t ntile, int64_t ncell,
                       const AtGroup* __restrict__ groups, int ngroups, int ranges, const int* __restrict__ chunks,
                       const uint8_t* __restrict__ bhi_g, const uint8_t* __restrict__ blo_g, float* __restrict__ G,
                       int* __restrict__ err) {
    // every pointer below is smem_raw plus an offset, so that the compiler keeps shared-memory loads
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int npairs = (ngroups + 1) / 2;
    const int pr = blockIdx.x % npairs, range = blockIdx.x / npairs;
    AtGroup gm[2];
    gm[0] = groups[2 * pr];
    if (2 * pr + 1 < ngroups) gm[1] = groups[2 * pr + 1];
    else gm[1] = AtGroup{0, 0, 0, 0, {0, 0}};
    const uint32_t sbo = (uint32_t)kp * 16u;  // bytes per 8 columns of B (kp/8 core matrices of 128 B)
    const int ncol0 = gm[0].nchunk * kAtChunk, ncol1 = gm[1].nchunk * kAtChunk;
    const int bbytes0 = ncol0 / 8 * (int)sbo, bbytes1 = ncol1 / 8 * (int)sbo;
    const int dfloats = kAtCells * kp;        // one tile of fields, [4][kp][32]
    uint8_t* s_b = smem_raw;                  // member 0: hi, lo; member 1: hi, lo ([ncol/8][kp/8] core matrices)
    float* s_d = reinterpret_cast<float*>(smem_raw + 2 * (bbytes0 + bbytes1));  // kAtDBufs tiles
    int* s_chunk = reinterpret_cast<int*>(s_d + kAtDBufs * dfloats);           // member 0's, then member 1's
    const int nch_all = gm[0].nchunk + gm[1].nchunk;
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_chunk + ((nch_all + 1) & ~1));
    uint64_t* a_ready = bars;        // A of the next tile written (8 cell warps)
    uint64_t* acc_full = bars + 1;   // [2] the MMAs of member b completed
    uint64_t* acc_free = bars + 3;   // [2] the epilogue read member b's accumulators (8 cell warps)
    uint64_t* drain = bars + 5;
    uint64_t* d_full = bars + 6;     // [kAtDBufs] a tile's fields landed
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 6 + kAtDBufs);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // B of both members, the chunk tables, and the zero rows [nshell, kp) of every field buffer
    for (int i = tid; i < bbytes0 / 16; i += kAtThreads) {
        reinterpret_cast<uint4*>(s_b)[i] = reinterpret_cast<const uint4*>(bhi_g + gm[0].b_off)[i];
        reinterpret_cast<uint4*>(s_b + bbytes0)[i] = reinterpret_cast<const uint4*>(blo_g + gm[0].b_off)[i];
    }
    for (int i = tid; i < bbytes1 / 16; i += kAtThreads) {
        reinterpret_cast<uint4*>(s_b + 2 * bbytes0)[i] = reinterpret_cast<const uint4*>(bhi_g + gm[1].b_off)[i];
        reinterpret_cast<uint4*>(s_b + 2 * bbytes0 + bbytes1)[i] = reinterpret_cast<const uint4*>(blo_g + gm[1].b_off)[i];
    }
    for (int c = tid; c < gm[0].nchunk; c += kAtThreads) s_chunk[c] = chunks[gm[0].chunk_off + c];
    for (int c = tid; c < gm[1].nchunk; c += kAtThreads) s_chunk[gm[0].nchunk + c] = chunks[gm[1].chunk_off + c];
    const int npad = (kp - nshell) * 32;
    for (int i = tid; i < 4 * kAtDBufs * npad; i += kAtThreads) {
        const int blk = i / npad, r = i - blk * npad;  // blk: buffer * 4 + quadrant
        s_d[(blk >> 2) * dfloats + (blk & 3) * kp * 32 + nshell * 32 + r] = 0.f;
    }
    if (tid == 0) {
        tc::mbar_init(a_ready, kAtCellWarps);
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(acc_full + b, 1);
            tc::mbar_init(acc_free + b, kAtCellWarps);
        }
        tc::mbar_init(drain, 1);
        for (int b = 0; b < kAtDBufs; b++) tc::mbar_init(d_full + b, 1);
        tc::mbar_fence_init();
        *s_abort = 0;
    }
    if (warp == kAtCellWarps) {
        tc::tmem_alloc(s_tmem, 512);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *s_tmem;
    const uint32_t a0 = 512u - (uint32_t)kp;  // A: hi at [a0, a0 + kp/2), lo at [a0 + kp/2, 512)
    const int64_t t0 = ntile * range / ranges, t1 = ntile * (range + 1) / ranges;

    if (warp == kAtCellWarps) {
        // ------------------------------------------------------ field copies, MMA issue
        const bool el = tc::elect_one();
        int64_t last[kAtDBufs];  // last tile copied into each buffer
        for (int b = 0; b < kAtDBufs; b++) last[b] = -1;
        auto load_tile = [&](int64_t t) {
            const int b = (int)((t - t0) % kAtDBufs);
            const int64_t c0 = t * kAtCells;
            const int nq = (int)((ncell - c0 < kAtCells ? ncell - c0 : kAtCells) / 32);
            const uint32_t qbytes = (uint32_t)nshell * 32u * 4u;
            tc::mbar_arrive_expect_tx(d_full + b, (uint32_t)nq * qbytes);
            for (int q = 0; q < nq; q++)
                tc::bulk_load(s_d + b * dfloats + q * kp * 32, D + (size_t)(c0 + 32 * q) * nshell, qbytes, d_full + b);
            last[b] = t;
        };
        if (el)
            for (int64_t t = t0; t < t1 && t < t0 + kAtDBufs; t++) load_tile(t);
        const uint64_t desc_k = ((uint64_t)(((sbo >> 4) & 0x3FFFu) | (1u << 14)) << 32) | (uint64_t)((128u >> 4) << 16);
        for (int64_t t = t0; t < t1; t++) {
            const int64_t k = t - t0;
            if (!tc::mbar_wait_warp(a_ready, (uint32_t)(k & 1), s_abort)) break;
            bool ok = true;
            for (int b = 0; b < 2 && ok; b++) {
                // the epilogue of member b for tile t - 1 has read its accumulators
                if (k > 0 && !tc::mbar_wait_warp(acc_free + b, (uint32_t)((k - 1) & 1), s_abort)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                if (el) {
                    // tile t - 1 is fully reduced: its field buffer takes tile t - 1 + kAtDBufs
                    if (b == 1 && k > 0 && t - 1 + kAtDBufs < t1) load_tile(t - 1 + kAtDBufs);
                    const int ncol = b ? ncol1 : ncol0;
                    if (ncol > 0) {
                        const uint32_t bh = tc::smem_u32(s_b + (b ? 2 * bbytes0 : 0));
                        const uint32_t bl = bh + (uint32_t)(b ? bbytes1 : bbytes0);
                        const uint32_t idesc = tc::idesc_bf16(128, ncol);  // ncol <= acap <= 256: one MMA run
                        uint32_t acc = 0u;
                        for (int ks = 0; ks < kp / 16; ks++) {
                            if (!((gm[b].kmask[0] >> ks) & 1)) continue;
                            const uint32_t bo = (uint32_t)ks * 256u;
                            const uint64_t dh = desc_k | (uint64_t)(((bh + bo) >> 4) & 0x3FFFu);
                            const uint64_t dl = desc_k | (uint64_t)(((bl + bo) >> 4) & 0x3FFFu);
                            const uint32_t ah = tmem + a0 + (uint32_t)(ks * 8), al = ah + (uint32_t)(kp / 2);
                            const uint32_t d = tmem + (uint32_t)(b * acap);
                            tc::mma_ts(d, ah, dh, idesc, acc);  // hi x hi
                            tc::mma_ts(d, ah, dl, idesc, 1u);   // hi x lo
                            tc::mma_ts(d, al, dh, idesc, 1u);   // lo x hi
                            acc = 1u;
                        }
                    }
                    tc::mma_commit(acc_full + b);  // also for an absent member: it arrives once the MMAs so far finish
                }
                __syncwarp();
            }
            if (!ok) break;
        }
        // every MMA and copy issued completes before the block frees its columns and exits
        if (el) {
            tc::mma_commit(drain);
            volatile int no_abort = 0;
            tc::mbar_wait(drain, 0, &no_abort);
            for (int b = 0; b < kAtDBufs; b++)
                if (last[b] >= 0) {
                    no_abort = 0;
                    tc::mbar_wait(d_full + b, (uint32_t)(((last[b] - t0) / kAtDBufs) & 1), &no_abort);
                }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------ cells: A, epilogue
        const int q = warp & 3, h = warp >> 2;  // lane quadrant, half of each member's m's
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        // A of tile t (hi/lo pairs of shells, 32 shells per store pair; the two halves take alternate blocks)
        auto build_a = [&](int64_t t) -> bool {
            const int64_t k = t - t0;
            const int b = (int)(k % kAtDBufs);
            if (!tc::mbar_wait_warp(d_full + b, (uint32_t)((k / kAtDBufs) & 1), s_abort)) return false;
            const float* sd = s_d + b * dfloats + q * kp * 32 + lane;
            for (int k0 = 32 * h; k0 < kp; k0 += 64) {
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int i = 0; i < 16; i++) tc::split2_fast(sd[32 * (k0 + 2 * i)], sd[32 * (k0 + 2 * i + 1)], hi[i], lo[i]);
                tc::tmem_st16(tmem + lane_base + a0 + (uint32_t)(k0 / 2), hi);
                tc::tmem_st16(tmem + lane_base + a0 + (uint32_t)(kp / 2 + k0 / 2), lo);
            }
            tc::tmem_st_wait();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(a_ready);
            return true;
        };
        // G_m(x) = sum over m's chunks (m, jb) of sum_i D_{16 jb + i}(x) T[x][(m, 16 jb + i)], member b
        auto epilogue = [&](int b, const float* sd, int64_t cell) {
            const int base_c = b ? gm[0].nchunk : 0;
            const int c_begin = h ? gm[b].hsplit : 0, c_end = h ? gm[b].nchunk : gm[b].hsplit;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int c = c_begin; c < c_end; c++) {
                const int cd = s_chunk[base_c + c];
                uint32_t v[16];
                tc::tmem_ld16(tmem + lane_base + (uint32_t)(b * acap + c * kAtChunk), v);
                const float* dj = sd + 32 * kAtChunk * (cd & 255);
                float x[16];
#pragma unroll
                for (int i = 0; i < 16; i++) x[i] = dj[32 * i];
                tc::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; i++) acc[i & 3] = fmaf(x[i], __uint_as_float(v[i]), acc[i & 3]);
                if (cd & (1 << 16)) {
                    if (cell < ncell) G[(size_t)((cd >> 8) & 255) * ncell + cell] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
                    acc[0] = acc[1] = acc[2] = acc[3] = 0.f;
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(acc_free + b);
        };
        bool ok = t0 >= t1 || build_a(t0);
        for (int64_t t = t0; t < t1 && ok; t++) {
            const int64_t k = t - t0;
            const float* sd = s_d + (int)(k % kAtDBufs) * dfloats + q * kp * 32 + lane;
            const int64_t cell = t * kAtCells + 32 * q + lane;
            // member 0 (its MMAs are done; member 1's run meanwhile)
            if (!tc::mbar_wait_warp(acc_full, (uint32_t)(k & 1), s_abort)) break;
            tc::fence_after_sync();
            epilogue(0, sd, cell);
            // every MMA of tile t is done with A: write the next tile's, then reduce member 1 while
            // the next tile's member-0 MMAs run
            if (!tc::mbar_wait_warp(acc_full + 1, (uint32_t)(k & 1), s_abort)) break;
            tc::fence_after_sync();
            if (t + 1 < t1 && !build_a(t + 1)) break;
            epilogue(1, sd, cell);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kAtCellWarps) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
    if (tid == 0 && *s_abort) atomicExch(err, tc::kErrTimeout);
}

}  // namespace ps

using namespace ps;

struct AtState {
    std::vector<AtGroup> groups;
    std::vector<int> empty_m;  // shells with no entry: G_m = 0
    int kp = 0, acap = 0, ranges = 1, max_nchunk = 0;
    size_t smem = 0;
    void *d_groups = nullptr, *d_chunks = nullptr, *d_pos = nullptr, *d_bhi = nullptr, *d_blo = nullptr;
    int* d_err = nullptr;
    int nent = 0;
};

// shared memory of a block whose pair of groups has nc0 and nc1 chunks
static size_t at_smem_bytes(int nc0, int nc1, int kp) {
    const size_t ncol = (size_t)(nc0 + nc1) * kAtChunk;
    return 2 * ncol / 8 * kp * 16 + kAtDBufs * (size_t)kAtCells * kp * 4 + (size_t)(nc0 + nc1 + 1) * 4 +
           8 * (8 + kAtDBufs) + 16;
}

// Host tables of the tensor-core adjoint: the groups of m's with their chunks
// (m, j block) and the B position of every entry.  Fills S's host fields and
// chunks, pos and b_total (bytes of one B array); touches no device.
// ent: the adjoint's entries in order (m ascending), each (m, f1, f2) with f1 <= f2.
static poly_status at_build_tables(const PsPlan* p, const std::vector<int>& ent_m, const std::vector<short4>& ent,
                                   AtState* S, std::vector<int>& chunks, std::vector<int>& pos, size_t& b_total) {
    const int64_t ncell = (int64_t)p->N * p->N * p->N;
    const int ns = p->nshell;
    S->kp = (ns + 31) / 32 * 32;  // the A stores write 16 columns (32 shells) of hi and of lo at a time
    const int kp = S->kp;
    // chunks: (m, jb) for each j block that holds a j of one of m's entries (j = f2)
    std::vector<std::vector<int>> mjb(ns);
    for (size_t e = 0; e < ent.size(); e++) mjb[ent_m[e]].push_back(ent[e].y / kAtChunk);
    for (int m = 0; m < ns; m++) {
        auto& v = mjb[m];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        if (v.empty()) S->empty_m.push_back(m);
    }
    // groups of consecutive m's within TMEM (512 - kp columns) and the block's shared memory, split into
    // two halves of about equal chunk counts
    // two accumulator buffers next to A: acap columns each, one MMA run of at most 256
    S->acap = std::min(256, (512 - kp) / 2 / 32 * 32);  // each buffer starts on a 32-column boundary
    const int chunk_cap = S->acap / kAtChunk;
    // a group fits when two groups of its size fit one block (the blocks take pairs of groups)
    auto fits = [&](int nchunk) { return nchunk <= chunk_cap && at_smem_bytes(nchunk, nchunk, kp) <= 227 * 1024; };
    std::map<std::pair<int, int>, std::pair<int, int>> chpos;  // (m, jb) -> (group, chunk)
    b_total = 0;
    for (int m = 0; m < ns;) {
        int nch = 0, m1 = m;
        while (m1 < ns && fits(nch + (int)mjb[m1].size())) nch += (int)mjb[m1++].size();
        if (m1 == m) return POLY_ERR_UNSUPPORTED;  // one shell's chunks do not fit
        int split = m1, best = nch, pre = 0;
        for (int ms = m; ms <= m1; ms++) {
            const int worst = std::max(pre, nch - pre);
            if (worst < best) {
                best = worst;
                split = ms;
            }
            if (ms < m1) pre += (int)mjb[ms].size();
        }
        AtGroup G{};
        G.chunk_off = (int)chunks.size();
        const int gi = (int)S->groups.size();
        int c = 0;
        for (int mm = m; mm < m1; mm++) {
            if (mm == split) G.hsplit = c;
            for (size_t q = 0; q < mjb[mm].size(); q++) {
                chpos[{mm, mjb[mm][q]}] = {gi, c++};
                chunks.push_back(mjb[mm][q] | (mm << 8) | (q + 1 == mjb[mm].size() ? (1 << 16) : 0));
            }
        }
        if (split == m1) G.hsplit = c;
        G.nchunk = c;
        G.b_off = (int)b_total;
        b_total += (size_t)c * kAtChunk / 8 * kp * 16;
        S->groups.push_back(G);
        S->max_nchunk = std::max(S->max_nchunk, c);
        m = m1;
    }
    // B positions of the entries (column 16 chunk + j % 16, row k = f1) and the nonzero K blocks of each run
    pos.assign(ent.size(), -1);
    for (size_t e = 0; e < ent.size(); e++) {
        const int j = ent[e].y, k = ent[e].x;
        const auto gp = chpos.at({ent_m[e], j / kAtChunk});
        AtGroup& G = S->groups[gp.first];
        const int n = gp.second * kAtChunk + j % kAtChunk;
        pos[e] = G.b_off + (n / 8) * kp * 16 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
        G.kmask[n / 256] |= 1 << (k / 16);
    }
    S->nent = (int)ent.size();
    // at least half the SM's shared memory: one block per SM, so no block waits in tcgen05.alloc for another
    S->smem = std::max<size_t>(at_smem_bytes(S->max_nchunk, S->max_nchunk, kp), 116 * 1024);
    const int64_t ntile = (ncell + kAtCells - 1) / kAtCells;
    const int npairs = ((int)S->groups.size() + 1) / 2;
    S->ranges = (int)std::max<int64_t>(1, std::min<int64_t>(ntile, (2 * p->sms + npairs - 1) / npairs));
    return POLY_OK;
}

poly_status ps_at_prepare(PsPlan* p, const std::vector<int>& ent_m, const std::vector<short4>& ent, AtState** out) {
    *out = nullptr;
    const int64_t ncell = (int64_t)p->N * p->N * p->N;
    if (p->order != 3 || p->prec != POLY_SPLIT_BF16 || p->nshell > kAtMaxK || ncell % 32) return POLY_ERR_UNSUPPORTED;
    AtState* S = new (std::nothrow) AtState();
    if (!S) return POLY_ERR_ALLOC;
    std::vector<int> chunks, pos;
    size_t b_total = 0;
    if (poly_status s0 = at_build_tables(p, ent_m, ent, S, chunks, pos, b_total)) {
        delete S;
        return s0;
    }
    auto up = [&](void** d, const void* h, size_t bytes) -> poly_status {
        poly_status s = ps_alloc(p, d, bytes);
        if (s) return s;
        return cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice) ? POLY_ERR_CUDA : POLY_OK;
    };
    poly_status s;
    if ((s = up(&S->d_groups, S->groups.data(), S->groups.size() * sizeof(AtGroup))) ||
        (s = up(&S->d_chunks, chunks.data(), chunks.size() * 4)) ||
        (s = up(&S->d_pos, pos.data(), std::max<size_t>(1, pos.size()) * 4)) ||
        (s = ps_alloc(p, &S->d_bhi, std::max<size_t>(16, b_total))) ||
        (s = ps_alloc(p, &S->d_blo, std::max<size_t>(16, b_total))) || (s = ps_alloc(p, (void**)&S->d_err, 16))) {
        delete S;
        return s;
    }
    if (cudaMemset(S->d_bhi, 0, std::max<size_t>(16, b_total)) || cudaMemset(S->d_blo, 0, std::max<size_t>(16, b_total)) ||
        cudaMemset(S->d_err, 0, 16)) {
        delete S;
        return POLY_ERR_CUDA;
    }
    *out = S;
    return POLY_OK;
}

static int diag_adj_tables(int N, int order, const double* edges, int nshell, unsigned flags, int prec, int sms,
                           int64_t* sizes, int32_t* moff, int16_t* ent, int32_t* eoff, int32_t* ebins,
                           int32_t* at_groups, int32_t* at_chunks, int32_t* at_pos) {
    if (!sizes || sms < 1) return POLY_ERR_ARG;
    if (order > 4) return POLY_ERR_UNSUPPORTED;  // as poly_backward
    PsPlan hp;  // host tables only: no device call, no device memory
    std::vector<short> lines;
    if (poly_status s = ps_plan_host_tables(&hp, N, 1.0, order, nshell, edges, (poly_precision)prec, flags, 0, lines))
        return s;
    hp.sms = sms;
    std::vector<int> mo, eo, eb;
    std::vector<short4> en;
    ps_adj_entries(&hp, mo, en, eo, eb);
    AtState S;
    std::vector<int> chunks, pos;
    size_t b_total = 0;
    bool at = order == 3 && prec == POLY_SPLIT_BF16 && nshell <= kAtMaxK && ((int64_t)N * N * N) % 32 == 0;
    if (at) {
        std::vector<int> ent_m(en.size());
        for (int m = 0; m < nshell; m++)
            for (int e = mo[m]; e < mo[m + 1]; e++) ent_m[e] = m;
        const poly_status s = at_build_tables(&hp, ent_m, en, &S, chunks, pos, b_total);
        if (s && s != POLY_ERR_UNSUPPORTED) return s;
        at = !s;
    }
    const int64_t n[10] = {(int64_t)en.size(), (int64_t)eb.size(), at ? (int64_t)S.groups.size() : 0,
                           at ? (int64_t)chunks.size() : 0, S.kp, S.acap, (int64_t)b_total, S.ranges,
                           (int64_t)S.empty_m.size(), S.max_nchunk};
    for (int i = 0; i < 10; i++) sizes[i] = n[i];
    if (moff) std::copy(mo.begin(), mo.end(), moff);
    for (size_t i = 0; ent && i < en.size(); i++) {
        ent[3 * i] = en[i].x;
        ent[3 * i + 1] = en[i].y;
        ent[3 * i + 2] = en[i].z;
    }
    if (eoff) std::copy(eo.begin(), eo.end(), eoff);
    if (ebins) std::copy(eb.begin(), eb.end(), ebins);
    if (!at) return POLY_OK;
    for (size_t g = 0; at_groups && g < S.groups.size(); g++) {
        const AtGroup& G = S.groups[g];
        const int32_t v[6] = {G.chunk_off, G.nchunk, G.hsplit, G.b_off, G.kmask[0], G.kmask[1]};
        std::copy(v, v + 6, at_groups + 6 * g);
    }
    if (at_chunks) std::copy(chunks.begin(), chunks.end(), at_chunks);
    if (at_pos) std::copy(pos.begin(), pos.end(), at_pos);
    return POLY_OK;
}

extern "C" int poly_diag_adj_tables(int N, int order, const double* edges, int nshell, unsigned flags, int prec,
                                    int sms, int64_t* sizes, int32_t* moff, int16_t* ent, int32_t* eoff,
                                    int32_t* ebins, int32_t* at_groups, int32_t* at_chunks, int32_t* at_pos) {
    try {
        return diag_adj_tables(N, order, edges, nshell, flags, prec, sms, sizes, moff, ent, eoff, ebins, at_groups,
                               at_chunks, at_pos);
    } catch (const std::bad_alloc&) {
        return POLY_ERR_ALLOC;
    }
}

// G[m][x] for all m from the plan's fields and the entry weights w (FP32, entry order).
cudaError_t ps_at_contract(PsPlan* p, AtState* S, const float* w, cudaStream_t st) {
    const int nb = std::max(1, std::min(1024, (S->nent + 255) / 256));
    at_scatter_kernel<<<nb, 256, 0, st>>>(w, (const int*)S->d_pos, S->nent, (uint16_t*)S->d_bhi, (uint16_t*)S->d_blo);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    if ((e = cudaFuncSetAttribute(at_contract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S->smem)))
        return e;
    const int64_t ncell = (int64_t)p->N * p->N * p->N;
    for (int m : S->empty_m)
        if ((e = cudaMemsetAsync((float*)p->d_G + (size_t)m * ncell, 0, (size_t)ncell * 4, st))) return e;
    const int64_t ntile = (ncell + kAtCells - 1) / kAtCells;
    const unsigned nblk = (unsigned)(((S->groups.size() + 1) / 2) * (size_t)S->ranges);
    at_contract_kernel<<<nblk, kAtThreads, S->smem, st>>>((const float*)p->d_fields, p->nshell, S->kp, S->acap, ntile, ncell,
                                                          (const AtGroup*)S->d_groups, (int)S->groups.size(), S->ranges,
                                                          (const int*)S->d_chunks, (const uint8_t*)S->d_bhi,
                                                          (const uint8_t*)S->d_blo, (float*)p->d_G, S->d_err);
    return cudaGetLastError();
}

int ps_at_error(AtState* S) {
    int v = 0;
    if (!S || !S->d_err || cudaMemcpy(&v, S->d_err, 4, cudaMemcpyDeviceToHost)) return 0;
    if (v) cudaMemset(S->d_err, 0, 4);
    return v;
}

void ps_at_free(AtState* S) { delete S; }
