// Host side of the polyspectrum library: plan construction (shell tables, bin
// enumeration, contraction tiles, exact counts) and the C ABI of polyspec.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <stdexcept>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/polyspec.h"
#include "kernels.h"
#include "plan_internal.h"
#include "../../include/polyspec_diag.h"

namespace {

thread_local std::string g_last_error;
int g_fail_alloc_after = 0;

poly_status set_error(poly_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

poly_status cuda_error(cudaError_t e, const char* where) {
    return set_error(POLY_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PS_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);   \
    } while (0)

#define PS_TRY(call)                          \
    do {                                      \
        poly_status s_ = (call);              \
        if (s_ != POLY_OK) return s_;         \
    } while (0)

// Runs f, turning a C++ exception from host containers into a status: no
// exception crosses the C ABI.
template <typename F>
static poly_status guarded(F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return set_error(POLY_ERR_ALLOC, "host allocation failed");
    } catch (const std::exception& ex) {
        return set_error(POLY_ERR_ARG, ex.what());
    }
}

// ---- counts cache (per process) -----------------------------------------
struct CountKey {
    int N, order;
    unsigned rule;
    std::vector<double> edges;
    bool operator<(const CountKey& o) const {
        return std::tie(N, order, rule, edges) < std::tie(o.N, o.order, o.rule, o.edges);
    }
};
std::mutex g_count_mu;
std::map<CountKey, std::vector<int64_t>> g_count_cache;

}  // namespace

void ps_set_last_error(const std::string& msg) { g_last_error = msg; }

// ---------------------------------------------------------------------------
// allocation helper with the failure-injection hook
// ---------------------------------------------------------------------------
poly_status ps_alloc(PsPlan* p, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (g_fail_alloc_after > 0 && --g_fail_alloc_after == 0)
        return set_error(POLY_ERR_ALLOC, "injected allocation failure");
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return set_error(POLY_ERR_ALLOC, std::string("cudaMalloc(") + std::to_string(bytes) + "): " +
                                             cudaGetErrorString(e));
    }
    p->allocations.push_back(*ptr);
    p->allocation_bytes.push_back(bytes);
    return POLY_OK;
}

void ps_free(PsPlan* p, void* ptr) {
    if (!ptr) return;
    auto it = std::find(p->allocations.begin(), p->allocations.end(), ptr);
    if (it != p->allocations.end()) {
        cudaFree(ptr);
        p->allocation_bytes.erase(p->allocation_bytes.begin() + (it - p->allocations.begin()));
        p->allocations.erase(it);
    }
}

template <typename V>
static poly_status upload(PsPlan* p, void** dptr, const std::vector<V>& h) {
    PS_TRY(ps_alloc(p, dptr, h.size() * sizeof(V)));
    if (!h.empty()) PS_CUDA(cudaMemcpy(*dptr, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
    return POLY_OK;
}

// ---------------------------------------------------------------------------
// bins: k_1 >= ... >= k_n (1-based), row-major with k_n fastest, polygon rule
// ---------------------------------------------------------------------------
void enumerate_bins(int nshell, const std::vector<double>& edges, int order, bool all_sorted,
                           std::vector<int32_t>& out) {
    std::vector<double> c(nshell);
    for (int s = 0; s < nshell; s++) c[s] = 0.5 * (edges[s] + edges[s + 1]);
    std::vector<int> k(order, 1);
    // iterate in lexicographic order of (k_1, ..., k_n) with k_1 >= k_2 >= ...
    std::vector<int> cur(order);
    std::function<void(int)> rec = [&](int d) {
        if (d == order) {
            double rest = 0;
            for (int t = 1; t < order; t++) rest += c[cur[t] - 1];
            if (all_sorted || c[cur[0] - 1] <= rest + 1e-9 * c[cur[0] - 1])
                for (int t = 0; t < order; t++) out.push_back(cur[t]);
            return;
        }
        const int hi = d == 0 ? nshell : cur[d - 1];
        for (int v = 1; v <= hi; v++) {
            cur[d] = v;
            rec(d + 1);
        }
    };
    rec(0);
}

// ---------------------------------------------------------------------------
// shell line tables: per shell, the (ky, kz >= 0) lines crossing it and the
// |kx| run [a, b] on each line.  |q|^2 = rho2 + kx^2 grows with |kx|, so the
// shell's kx on a line form one run: a is the first |kx| with |q|^2 >= e_s^2,
// b the last (<= K) with |q|^2 < e_{s+1}^2, found from a square root and then
// settled by the exact comparisons e_s^2 <= |q|^2 < e_{s+1}^2 in double, |q|^2
// converted exactly (q = 0 is in no shell).
// ---------------------------------------------------------------------------
void build_lines(const PsPlan* p, const double* e, int s, std::vector<short>& lines) {
    const int K = p->K;
    const double lo2 = e[s] * e[s], hi2 = e[s + 1] * e[s + 1];
    for (int ky = -K; ky <= K; ky++)
        for (int kz = 0; kz <= K; kz++) {
            const long long rho2 = (long long)ky * ky + (long long)kz * kz;
            auto q2 = [&](long long kx) { return (double)(rho2 + kx * kx); };
            long long a = lo2 > (double)rho2 ? (long long)std::sqrt(lo2 - (double)rho2) : 0;
            if (a > K + 1) a = K + 1;
            while (a > 0 && q2(a - 1) >= lo2) a--;
            while (a <= K && q2(a) < lo2) a++;
            if (a == 0 && rho2 == 0) a = 1;
            long long b = hi2 > (double)rho2 ? (long long)std::sqrt(hi2 - (double)rho2) : -1;
            if (b > K) b = K;
            while (b >= 0 && q2(b) >= hi2) b--;
            while (b < K && q2(b + 1) < hi2) b++;
            if (a <= b) {
                lines.push_back((short)ky);
                lines.push_back((short)kz);
                lines.push_back((short)a);
                lines.push_back((short)b);
            }
        }
}

// ---------------------------------------------------------------------------
// CUDA-core contraction tiles: rows = products of the first ra shells of a
// bin, cols = products of the rest (ra = 1, 2, 2, 2, 3 for n = 2..6); rows
// grouped 64 at a time after sorting by their column span, each group's column
// union cut into chunks of 64.
// ---------------------------------------------------------------------------
void build_cc_tiles(PsPlan* p, CcTiles& t, int first_shift) {
    using Key = std::array<int, 3>;  // 1-based field slots, -1 padded
    const int n = p->order;
    const int ra = n <= 2 ? 1 : (n <= 5 ? 2 : 3), ca = n - ra;
    auto key = [](const int32_t* b, int cnt) {
        Key k{-1, -1, -1};
        for (int i = 0; i < cnt; i++) k[i] = b[i];
        return k;
    };
    // first_shift > 0: the bin's first leg reads the weighted field slot k1 + first_shift (multipoles)
    auto rkey = [&](const int32_t* b) {
        Key k = key(b, ra);
        k[0] += first_shift;
        return k;
    };
    auto ckey = [&](const int32_t* b) { return key(b + ra, ca); };
    std::map<Key, std::vector<Key>> rows;  // row -> col keys
    for (int64_t i = 0; i < p->nbins; i++) rows[rkey(&p->bins[i * n])].push_back(ckey(&p->bins[i * n]));
    struct RowInfo {
        Key key;
        std::vector<Key> cols;
    };
    std::vector<RowInfo> ri;
    for (auto& kv : rows) {
        auto cols = kv.second;
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
        ri.push_back({kv.first, cols});
    }
    std::stable_sort(ri.begin(), ri.end(), [](const RowInfo& a, const RowInfo& b) {
        return std::make_pair(a.cols.front(), a.cols.back()) < std::make_pair(b.cols.front(), b.cols.back());
    });
    // (row key, col key) -> slot; the six slots (from 1, or -1; at most 2 * kPsMaxShells) packed 10 bits each
    static_assert(2 * kPsMaxShells + 1 < 1024, "a field slot + 1 must fit 10 bits of the packed key");
    if (p->nshell > kPsMaxShells) throw std::length_error("build_cc_tiles: more shells than the packed keys hold");
    auto pack = [](const Key& r, const Key& c) {
        uint64_t v = 0;
        for (int i = 0; i < 3; i++) v = v << 10 | (uint64_t)(r[i] + 1);
        for (int i = 0; i < 3; i++) v = v << 10 | (uint64_t)(c[i] + 1);
        return v;
    };
    std::unordered_map<uint64_t, int64_t> slot_of;
    slot_of.reserve((size_t)p->nbins * 2);
    for (size_t g = 0; g < ri.size(); g += kCcTM) {
        const size_t g1 = std::min(ri.size(), g + kCcTM);
        std::vector<Key> cu;
        for (size_t r = g; r < g1; r++) cu.insert(cu.end(), ri[r].cols.begin(), ri[r].cols.end());
        std::sort(cu.begin(), cu.end());
        cu.erase(std::unique(cu.begin(), cu.end()), cu.end());
        for (size_t c0 = 0; c0 < cu.size(); c0 += kCcTN) {
            const size_t c1 = std::min(cu.size(), c0 + kCcTN);
            PsTile tile{};
            tile.row_off = (int)t.rowf.size();
            tile.nrow = (int)(g1 - g);
            tile.col_off = (int)t.colf.size();
            tile.ncol = (int)(c1 - c0);
            tile.field_off = (int)t.field_ids.size();
            std::map<int, int> local;  // shell (0-based) -> local field index
            auto loc = [&](int shell1) -> short {
                if (shell1 < 0) return -1;
                auto it = local.find(shell1 - 1);
                if (it != local.end()) return (short)it->second;
                int id = (int)local.size();
                local[shell1 - 1] = id;
                t.field_ids.push_back(shell1 - 1);
                return (short)id;
            };
            auto factors = [&](const Key& k) {  // in order: local ids follow first appearance, row by row
                const short a = loc(k[0]);
                const short b = loc(k[1]);
                const short c = loc(k[2]);
                return make_short4(a, b, c, -1);
            };
            for (size_t r = g; r < g1; r++) t.rowf.push_back(factors(ri[r].key));
            std::map<Key, int> cidx;
            for (size_t c = c0; c < c1; c++) {
                t.colf.push_back(factors(cu[c]));
                cidx[cu[c]] = (int)(c - c0);
            }
            tile.nfield = (int)local.size();
            const int tid = (int)t.tiles.size();
            for (size_t r = g; r < g1; r++)
                for (auto& ck : ri[r].cols) {
                    auto it = cidx.find(ck);
                    if (it == cidx.end()) continue;
                    const int rr = (int)(r - g), cc = it->second;
                    tile.region_mask |= 1u << ((rr / 32) * 4 + cc / 16);
                    slot_of[pack(ri[r].key, ck)] = (int64_t)tid * (kCcTM * kCcTN) + rr * kCcTN + cc;
                }
            t.tiles.push_back(tile);
        }
    }
    t.slot.resize(p->nbins);
    for (int64_t i = 0; i < p->nbins; i++) t.slot[i] = slot_of.at(pack(rkey(&p->bins[i * n]), ckey(&p->bins[i * n])));
}

static int choose_splits(int ntiles, int64_t nchunks, int sms) {
    int want = std::max(1, (4 * sms + ntiles - 1) / ntiles);
    int64_t maxs = std::max<int64_t>(1, nchunks / 16);
    return (int)std::min<int64_t>(want, maxs);
}

// ---------------------------------------------------------------------------
// exact counts: FP64 counting fields on the symmetry wedge
//   0 <= x <= y <= z <= floor(N/2), weight = orbit size under coordinate
//   permutations and sign flips (x_c -> N - x_c); sum_wedge w prod iota = sum_x prod iota.
// The counting fields are invariant under those 48 symmetries of the cube
// because the shells are spheres.  Even N.
// ---------------------------------------------------------------------------
static void count_wedge(int N, std::vector<int32_t>& widx, std::vector<double>& wgt) {
    const int h = N / 2;
    for (int x = 0; x <= h; x++)
        for (int y = x; y <= h; y++)
            for (int z = y; z <= h; z++) {
                int perms = (x == y && y == z) ? 1 : (x == y || y == z) ? 3 : 6;
                double w = perms;
                for (int v : {x, y, z}) w *= (v == 0 || 2 * v == N) ? 1.0 : 2.0;
                widx.push_back((int32_t)(((int64_t)x * N + y) * N + z));
                wgt.push_back(w);
            }
}

// Bins whose closures may wrap around the grid: a closed polygon q_1 + ... + q_n = 0
// (mod N) can differ from an exact closure only where some component sum reaches
// +-N, which needs sum_t K_t >= N with K_t the largest component of a mode of shell
// b_t (the largest kz of the shell's lines: the shells are symmetric under axis
// permutations).  Bins below that bound count exact closures only.
static void bin_wraps(const PsPlan* p, uint8_t* out) {
    for (int64_t b = 0; b < p->nbins; b++) {
        int64_t k = 0;
        for (int t = 0; t < p->order; t++) k += p->shell_kz[p->bins[b * p->order + t] - 1];
        out[b] = k >= p->N ? 1 : 0;
    }
}

// Exact counts from integer closure maps (counts_exact.cu), for plans whose closures cannot wrap:
// legs split into A (the first max(1, n - 3)) and B (the rest); per distinct group, the product of
// its full-grid FP64 counting fields is forward transformed on the cube |p_c| <= K' = |A| K and
// rounded to its integer closure map; count_b = sum_p G_A(p) G_B(p) in 64-bit integers.
static poly_status exact_counts(PsPlan* p, cudaStream_t st, std::vector<int64_t>& counts) {
    const int N = p->N, n = p->order, K = p->K;
    const int a = std::max(1, n - 3);
    const int Kp = a * K;
    if (p->flags & POLY_ALLOW_ALIAS) return set_error(POLY_ERR_COUNT, "exact counts need closures that cannot wrap");
    if (2 * Kp + 1 > N) return set_error(POLY_ERR_COUNT, "exact counts: the first legs' sums exceed the grid");
    std::map<std::array<int, 3>, int> gid;
    std::vector<std::array<int, 3>> groups;
    std::vector<int2> which((size_t)p->nbins);
    auto group_of = [&](const int32_t* k, int cnt) {
        std::array<int, 3> g{-1, -1, -1};
        for (int i = 0; i < cnt; i++) g[i] = k[i] - 1;
        auto it = gid.find(g);
        if (it != gid.end()) return it->second;
        const int id = (int)groups.size();
        gid[g] = id;
        groups.push_back(g);
        return id;
    };
    for (int64_t b = 0; b < p->nbins; b++) {
        const int32_t* k = &p->bins[b * n];
        which[b] = make_int2(group_of(k, a), group_of(k + a, n - a));
    }
    const size_t n3 = (size_t)N * N * N;
    const size_t mapsz = (size_t)(2 * Kp + 1) * (2 * Kp + 1) * (Kp + 1);
    std::vector<void*> tmp;
    auto talloc = [&](void** ptr, size_t bytes) -> poly_status {
        cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(POLY_ERR_ALLOC, "exact counts workspace allocation failed");
        }
        tmp.push_back(*ptr);
        return POLY_OK;
    };
    const int sb = std::min(8, p->nshell);
    const bool spill_inv = ps_plane_needs_spill(N, K, 1) == 1, spill_fwd = ps_plane_needs_spill(N, Kp, 1) == 1;
    const size_t spill_elems = std::max(spill_inv ? ps_spill_elems(N, K, N * sb, 1) : 0,
                                        spill_fwd ? ps_spill_elems(N, Kp, N, 1) : 0);
    void *d_iota = nullptr, *d_prod = nullptr, *d_W = nullptr, *d_fh = nullptr, *d_spill = nullptr, *d_maps = nullptr,
         *d_which = nullptr, *d_out = nullptr, *d_err = nullptr;
    poly_status rc = POLY_OK;
    cudaError_t e = cudaSuccess;
    do {
        if ((rc = talloc(&d_iota, (size_t)p->nshell * n3 * 8)) || (rc = talloc(&d_prod, n3 * 8)) ||
            (rc = talloc(&d_W, (size_t)N * (2 * Kp + 1) * (Kp + 1) * 16)) || (rc = talloc(&d_fh, mapsz * 16)) ||
            (spill_elems && (rc = talloc(&d_spill, spill_elems * 16))) ||
            (rc = talloc(&d_maps, groups.size() * mapsz * 8)) || (rc = talloc(&d_which, which.size() * sizeof(int2))) ||
            (rc = talloc(&d_out, which.size() * 8)) || (rc = talloc(&d_err, 4)))
            break;
        if ((e = cudaMemsetAsync(d_err, 0, 4, st)) ||
            (e = cudaMemcpyAsync(d_which, which.data(), which.size() * sizeof(int2), cudaMemcpyHostToDevice, st))) {
            rc = cuda_error(e, "exact counts upload");
            break;
        }
        // full-grid FP64 counting fields, natural layout
        for (int s0 = 0; s0 < p->nshell && !rc; s0 += sb) {
            const int ns = std::min(sb, p->nshell - s0);
            if ((e = ps_inverse(N, 1, 1, nullptr, p->d_lines, p->d_line_off, s0, ns, K, 0, N, p->d_tw_inv,
                                (double*)d_iota + (size_t)s0 * n3, n3, d_spill, nullptr, 0, 0, st)))
                rc = cuda_error(e, "exact counts: counting fields");
        }
        for (size_t g = 0; g < groups.size() && !rc; g++) {
            const auto& G = groups[g];
            if ((e = ps_prod_fields((const double*)d_iota, n3, G[0], G[1], G[2], (double*)d_prod, st)) ||
                (e = ps_forward(N, 1, d_prod, Kp, p->d_tw_fwd, d_W, d_fh, d_spill, st)) ||
                (e = ps_round_map(d_fh, mapsz, 1.0 / (double)n3, (long long*)d_maps + g * mapsz, (int*)d_err, st)))
                rc = cuda_error(e, "exact counts: closure maps");
        }
        if (rc) break;
        if ((e = ps_dot_maps((const long long*)d_maps, mapsz, (const int2*)d_which, (int)p->nbins, Kp,
                             (unsigned long long*)d_out, st))) {
            rc = cuda_error(e, "exact counts: sums");
            break;
        }
        std::vector<unsigned long long> c(which.size());
        int err = 0;
        if ((e = cudaMemcpyAsync(c.data(), d_out, c.size() * 8, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaMemcpyAsync(&err, d_err, 4, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st))) {
            rc = cuda_error(e, "exact counts readback");
            break;
        }
        if (err) {
            rc = set_error(POLY_ERR_COUNT, "exact counts: a closure map is not an integer");
            break;
        }
        counts.assign(c.begin(), c.end());
    } while (0);
    for (void* q : tmp) cudaFree(q);
    return rc;
}

static poly_status compute_counts(PsPlan* p, cudaStream_t st) {
    CountKey key{p->N, p->order, p->flags & POLY_BINS_ALL_SORTED, p->edges};
    {
        std::lock_guard<std::mutex> lk(g_count_mu);
        auto it = g_count_cache.find(key);
        if (it != g_count_cache.end()) {
            p->counts = it->second;
            return POLY_OK;
        }
    }
    const int N = p->N, h = N / 2;
    std::vector<int32_t> widx;
    std::vector<double> wgt;
    count_wedge(N, widx, wgt);
    const int64_t nw = (int64_t)widx.size();
    // device buffers (freed at the end of this function)
    std::vector<void*> tmp;
    auto talloc = [&](void** ptr, size_t bytes) -> poly_status {
        cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(POLY_ERR_ALLOC, "counts workspace allocation failed");
        }
        tmp.push_back(*ptr);
        return POLY_OK;
    };
    auto cleanup = [&]() {
        for (void* q : tmp) cudaFree(q);
    };
    poly_status rc = POLY_OK;
    void *d_widx = nullptr, *d_wgt = nullptr, *d_iota = nullptr, *d_planes = nullptr, *d_spill = nullptr,
         *d_part = nullptr, *d_S = nullptr;
    const int sb = std::min(8, p->nshell);  // shells per inverse batch
    const size_t plane_elems = (size_t)(h + 1) * N * N;
    const bool spill = ps_plane_needs_spill(N, p->K, 1) == 1;
    const CcTiles& t = p->cc;
    const int64_t nchunks = (nw + ps_cc_chunk(1) - 1) / ps_cc_chunk(1);
    const int nsplit = choose_splits((int)t.tiles.size(), nchunks, p->sms);
    const int64_t cps = (nchunks + nsplit - 1) / nsplit;
    const int64_t slot_stride = (int64_t)t.tiles.size() * kCcTM * kCcTN;
    do {
        if ((rc = talloc(&d_widx, widx.size() * 4))) break;
        if ((rc = talloc(&d_wgt, wgt.size() * 8))) break;
        if ((rc = talloc(&d_iota, (size_t)p->nshell * nw * 8))) break;
        if ((rc = talloc(&d_planes, (size_t)sb * plane_elems * 8))) break;
        if (spill && (rc = talloc(&d_spill, ps_spill_elems(N, p->K, (h + 1) * sb, 1) * 16))) break;
        if ((rc = talloc(&d_part, (size_t)nsplit * slot_stride * 8))) break;
        if ((rc = talloc(&d_S, (size_t)std::max<int64_t>(1, p->nbins) * 8))) break;
        cudaError_t e;
        if ((e = cudaMemcpyAsync(d_widx, widx.data(), widx.size() * 4, cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(d_wgt, wgt.data(), wgt.size() * 8, cudaMemcpyHostToDevice, st))) {
            rc = cuda_error(e, "counts upload");
            break;
        }
        for (int s0 = 0; s0 < p->nshell && !rc; s0 += sb) {
            const int ns = std::min(sb, p->nshell - s0);
            if ((e = ps_inverse(N, 1, 1, nullptr, p->d_lines, p->d_line_off, s0, ns, p->K, 0, h + 1, p->d_tw_inv,
                                d_planes, plane_elems, d_spill, nullptr, 0, 0, st))) {
                rc = cuda_error(e, "counting fields");
                break;
            }
            if ((e = ps_gather_cells(1, d_planes, plane_elems, ns, (const int32_t*)d_widx, nw,
                                     (double*)d_iota + (size_t)s0 * nw, nw, st))) {
                rc = cuda_error(e, "wedge gather");
                break;
            }
        }
        if (rc) break;
        if ((e = ps_contract_cc(1, 1, 0, p->order >= 5 ? 3 : 2, d_iota, (size_t)nw, 0, nw, d_wgt, (const PsTile*)p->d_cc_tiles,
                                (int)t.tiles.size(), (const int*)p->d_cc_field_ids, (const short4*)p->d_cc_rowf,
                                (const short4*)p->d_cc_colf, nsplit, cps, (double*)d_part, st)) ||
            (e = ps_reduce_slots((double*)d_part, nsplit, slot_stride, (const int64_t*)p->d_cc_slot, p->nbins,
                                 (double*)d_S, st))) {
            rc = cuda_error(e, "count contraction");
            break;
        }
        std::vector<double> S(p->nbins);
        if ((e = cudaMemcpyAsync(S.data(), d_S, p->nbins * 8, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            rc = cuda_error(e, "count readback");
            break;
        }
        const double n3 = (double)N * N * N;
        p->counts.resize(p->nbins);
        // The FP64 sum lands next to the integer count; rounding is exact while its error is
        // below 0.5.  The largest deviation seen is ~1e-3 (256^3, n = 4, counts ~1e11); a
        // deviation above 0.05 means the FP64 sum can no longer be trusted to round correctly,
        // and the plan's counts come from the integer closure maps instead.
        for (int64_t b = 0; b < p->nbins; b++) {
            const double v = S[b] / n3, r = std::nearbyint(v);
            if (std::fabs(v - r) > 0.05 || r < 0) {
                char msg[160];
                snprintf(msg, sizeof msg, "polygon count of bin %lld is not an integer: %.6f", (long long)b, v);
                rc = set_error(POLY_ERR_COUNT, msg);
                break;
            }
            p->counts[b] = (int64_t)r;
        }
    } while (0);
    cleanup();
    const char* force = getenv("POLY_COUNTS_EXACT");  // "1": always take the closure-map route (tests)
    if (rc == POLY_ERR_COUNT || (rc == POLY_OK && force && force[0] == '1')) rc = exact_counts(p, st, p->counts);
    if (rc == POLY_OK) {
        std::lock_guard<std::mutex> lk(g_count_mu);
        g_count_cache[key] = p->counts;
    }
    return rc;
}

// ---------------------------------------------------------------------------
// plan lifetime
// ---------------------------------------------------------------------------
static void free_plan(PsPlan* p) {
    if (!p) return;
    ps_batched_forget(p);
    int cur = -1;
    cudaGetDevice(&cur);
    if (p->device >= 0 && cur != p->device) cudaSetDevice(p->device);
    ps_tc_free(p);   // each frees its own buffers through ps_free, which drops them from the list
    ps_adj_free(p);
    for (void* q : p->allocations) cudaFree(q);
    p->allocations.clear();
    p->allocation_bytes.clear();
    for (auto& e : p->ev)
        if (e) cudaEventDestroy(e);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
}

constexpr int64_t kMaxSortedTuples = int64_t(1) << 26;  // host tables of about a GB at order 6

// The host part of plan creation: argument checks, the bins, the shell line tables
// (slot nshell holds the union of all shells, used by the adjoint) and the
// CUDA-core contraction tiles over the plain fields.  Touches no device.
poly_status ps_plan_host_tables(PsPlan* p, int N, double L, int order, int nshell, const double* edges,
                               poly_precision prec, unsigned flags, int ell, std::vector<short>& lines) {
    if (!edges || nshell < 1 || nshell > kPsMaxShells) return set_error(POLY_ERR_ARG, "nshell must be in [1, 128]");
    if (ell < 0 || ell > 8 || (ell & 1)) return set_error(POLY_ERR_ARG, "ell must be even, in [0, 8]");
    if (order < 2 || order > 6) return set_error(POLY_ERR_UNSUPPORTED, "order must be in [2, 6]");

    if (!(L > 0) || !std::isfinite(L)) return set_error(POLY_ERR_ARG, "L must be positive");
    if (flags & ~(POLY_BINS_ALL_SORTED | POLY_ALLOW_ALIAS)) return set_error(POLY_ERR_ARG, "unknown flag");
    if (!ps_supported_n(N)) return set_error(POLY_ERR_UNSUPPORTED, "grid size N not in the supported set");
    if (prec == POLY_TF32X3) return set_error(POLY_ERR_UNSUPPORTED, "POLY_TF32X3 is not implemented");
    if (prec != POLY_FP32 && prec != POLY_SPLIT_BF16 && prec != POLY_FP64)
        return set_error(POLY_ERR_ARG, "unknown precision");
    for (int s = 0; s <= nshell; s++)
        if (!std::isfinite(edges[s])) return set_error(POLY_ERR_ARG, "edges must be finite");
    if (edges[0] < 0) return set_error(POLY_ERR_ARG, "edges must be non-negative");
    for (int s = 0; s < nshell; s++)
        if (!(edges[s + 1] > edges[s])) return set_error(POLY_ERR_ARG, "edges must increase strictly");
    p->N = N;
    p->L = L;
    p->order = order;
    p->ell = ell;
    p->nfield = ell > 0 ? 2 * nshell : nshell;
    p->nshell = nshell;
    p->edges.assign(edges, edges + nshell + 1);
    p->prec = prec;
    p->flags = flags;
    p->is_double = prec == POLY_FP64;
    const double emax2 = edges[nshell] * edges[nshell];
    int K = 0;
    while ((double)((long long)(K + 1) * (K + 1)) < emax2) K++;
    p->K = K;
    if (2 * K + 1 > N) return set_error(POLY_ERR_ARG, "outer shell edge exceeds the Nyquist frequency");
    if ((long long)order * K >= N && !(flags & POLY_ALLOW_ALIAS))
        return set_error(POLY_ERR_ALIAS, "n * K >= N: polygon closures would wrap around the grid");

    // the enumeration walks every sorted tuple: C(nshell + order - 1, order) of them
    double tuples = 1.0;
    for (int i = 0; i < order; i++) tuples = tuples * (nshell + i) / (i + 1);
    if (tuples > (double)kMaxSortedTuples)
        return set_error(POLY_ERR_UNSUPPORTED, "too many bins: more than 2^26 sorted shell tuples");
    enumerate_bins(nshell, p->edges, order, (flags & POLY_BINS_ALL_SORTED) != 0, p->bins);
    p->nbins = (int64_t)p->bins.size() / order;

    // shell line tables
    std::vector<int> off{0};
    for (int s = 0; s < nshell; s++) {
        build_lines(p, p->edges.data(), s, lines);
        int kzm = 0;
        for (size_t l = off.back(); l < lines.size() / 4; l++) kzm = std::max(kzm, (int)lines[4 * l + 1]);
        p->shell_kz.push_back(kzm);
        off.push_back((int)(lines.size() / 4));
    }
    {
        const double ue[2] = {p->edges[0], p->edges[nshell]};
        build_lines(p, ue, 0, lines);
        off.push_back((int)(lines.size() / 4));
    }
    p->line_off = off;
    for (int s = 0; s <= nshell; s++) p->max_lines = std::max(p->max_lines, off[s + 1] - off[s]);
    build_cc_tiles(p, p->cc, 0);
    return POLY_OK;
}

static poly_status create_plan(PsPlan* p, int N, double L, int order, int nshell, const double* edges,
                               poly_precision prec, unsigned flags, int ell) {
    std::vector<short> lines;
    PS_TRY(ps_plan_host_tables(p, N, L, order, nshell, edges, prec, flags, ell, lines));
    const int K = p->K;
    const std::vector<int>& off = p->line_off;

    PS_CUDA(cudaGetDevice(&p->device));
    cudaDeviceProp prop;
    PS_CUDA(cudaGetDeviceProperties(&prop, p->device));
    p->sms = prop.multiProcessorCount;
    if (prec == POLY_SPLIT_BF16 && !(prop.major == 10 && prop.minor == 3))
        return set_error(POLY_ERR_UNSUPPORTED, "POLY_SPLIT_BF16 needs an sm_103 device");
    cudaStream_t st = nullptr;

    // twiddles e^{-/+ 2 pi i m / N}, FP64 on the host
    std::vector<double> twf(2 * N), twi(2 * N);
    for (int m = 0; m < N; m++) {
        const double a = 2.0 * 3.14159265358979323846 * (double)m / (double)N;
        twf[2 * m] = std::cos(a);
        twf[2 * m + 1] = -std::sin(a);
        twi[2 * m] = std::cos(a);
        twi[2 * m + 1] = std::sin(a);
    }
    PS_TRY(upload(p, &p->d_tw_fwd, twf));
    PS_TRY(upload(p, &p->d_tw_inv, twi));

    PS_TRY(upload(p, &p->d_lines, lines));
    PS_TRY(upload(p, (void**)&p->d_line_off, off));
    PS_TRY(upload(p, (void**)&p->d_shell_kz, p->shell_kz));

    // contraction tiles (CUDA-core path; the counts use them too)
    PS_TRY(upload(p, &p->d_cc_tiles, p->cc.tiles));
    PS_TRY(upload(p, &p->d_cc_field_ids, p->cc.field_ids));
    PS_TRY(upload(p, &p->d_cc_rowf, p->cc.rowf));
    PS_TRY(upload(p, &p->d_cc_colf, p->cc.colf));
    PS_TRY(upload(p, &p->d_cc_slot, p->cc.slot));

    // workspace
    const size_t n3 = (size_t)N * N * N;
    const size_t es = p->is_double ? 8 : 4;
    const size_t nl = (size_t)(2 * K + 1) * (K + 1);
    PS_TRY(ps_alloc(p, &p->d_W, (size_t)N * nl * 2 * es));
    PS_TRY(ps_alloc(p, &p->d_fhat, nl * (2 * K + 1) * 2 * es));
    PS_TRY(ps_alloc(p, &p->d_fields, (size_t)p->nfield * n3 * es));
    if (ell > 0) PS_TRY(ps_alloc(p, &p->d_fhat_w, nl * (2 * K + 1) * 2 * es));
    {   // x-pass output, indexed by the global line offset: every line of every shell and of
        // the union of the shells (used by the adjoint), at every x
        const size_t lines_all = (size_t)off[nshell + 1];
        PS_TRY(ps_alloc(p, &p->d_xpre, lines_all * N * 2 * es));
        p->xpre_lines = lines_all;
    }
    if (ps_plane_needs_spill(N, K, p->is_double) == 1)
        PS_TRY(ps_alloc(p, &p->d_spill, ps_spill_elems(N, K, N * nshell, p->is_double) * 2 * es));
    const int64_t chunk = ps_cc_chunk(p->is_double);
    const int64_t nchunks = ((int64_t)n3 + chunk - 1) / chunk;
    p->cc_nsplit = choose_splits((int)p->cc.tiles.size(), nchunks, p->sms);
    p->cc_cps = (nchunks + p->cc_nsplit - 1) / p->cc_nsplit;
    p->cc_slot_stride = (int64_t)p->cc.tiles.size() * kCcTM * kCcTN;
    PS_TRY(ps_alloc(p, (void**)&p->d_partial, (size_t)p->cc_nsplit * p->cc_slot_stride * 8));
    PS_TRY(ps_alloc(p, (void**)&p->d_S, (size_t)std::max<int64_t>(1, p->nbins) * 8));
    PS_TRY(ps_alloc(p, (void**)&p->d_counts, (size_t)std::max<int64_t>(1, p->nbins) * 8));
    PS_TRY(ps_alloc(p, &p->d_in_stage, n3 * es));
    PS_TRY(ps_alloc(p, (void**)&p->d_out_stage, (size_t)std::max<int64_t>(1, p->nbins) * 8));
    if (prec == POLY_SPLIT_BF16) PS_TRY(ps_tc_prepare(p));

    // exact counts (plan time, cached)
    PS_TRY(compute_counts(p, st));
    PS_CUDA(cudaMemcpy(p->d_counts, p->counts.data(), p->nbins * 8, cudaMemcpyHostToDevice));
    if (ell > 0) {
        // the counts used the plain tiles; the estimate's first leg reads the weighted fields
        for (void* d : {p->d_cc_tiles, p->d_cc_field_ids, p->d_cc_rowf, p->d_cc_colf, p->d_cc_slot}) ps_free(p, d);
        p->cc = CcTiles();
        build_cc_tiles(p, p->cc, nshell);
        PS_TRY(upload(p, &p->d_cc_tiles, p->cc.tiles));
        PS_TRY(upload(p, &p->d_cc_field_ids, p->cc.field_ids));
        PS_TRY(upload(p, &p->d_cc_rowf, p->cc.rowf));
        PS_TRY(upload(p, &p->d_cc_colf, p->cc.colf));
        PS_TRY(upload(p, &p->d_cc_slot, p->cc.slot));
        if ((int64_t)p->cc.tiles.size() * kCcTM * kCcTN != p->cc_slot_stride)
            return set_error(POLY_ERR_ARG, "multipole tiles differ in shape from the plain ones");
    }
    PS_CUDA(cudaDeviceSynchronize());
    return POLY_OK;
}

// ---------------------------------------------------------------------------
// pipeline pieces used by estimate / backward / batched
// ---------------------------------------------------------------------------
bool ps_xpre_fits(const PsPlan* p, int s0, int ns) {
    return s0 >= 0 && s0 + ns <= p->nshell + 1 && (size_t)p->line_off[s0 + ns] <= p->xpre_lines;
}

static void mark(PsPlan* p, int i, cudaStream_t st) {
    if (p->timing) cudaEventRecord(p->ev[i], st);
}

poly_status ps_fields(PsPlan* p, const void* delta, cudaStream_t st) {
    cudaError_t e;
    mark(p, 0, st);
    if ((e = ps_forward(p->N, p->is_double, delta, p->K, p->d_tw_fwd, p->d_W, p->d_fhat, p->d_spill, st)))
        return cuda_error(e, "forward transform");
    p->launches += 2;
    mark(p, 1, st);
    if (!ps_xpre_fits(p, 0, p->nshell)) return set_error(POLY_ERR_ARG, "x-pass buffer too small");
    if (p->is_double)
        e = ps_inverse(p->N, 1, 0, p->d_fhat, p->d_lines, p->d_line_off, 0, p->nshell, p->K, 0, p->N, p->d_tw_inv,
                       p->d_fields, (size_t)p->N * p->N * p->N, p->d_spill, p->d_xpre, p->max_lines, p->nfield, st);
    else
        e = ps_inverse_ranged_f32(p->N, p->d_fhat, p->d_lines, p->d_line_off, 0, p->nshell, p->K, p->d_tw_inv,
                                  p->d_fields, (size_t)p->N * p->N * p->N, p->d_xpre, p->max_lines, p->nfield,
                                  p->shell_kz.data(), p->d_shell_kz, st);
    if (e) return cuda_error(e, "shell fields");
    p->launches += 2;  // x pass + plane kernel
    if (p->ell > 0) {
        // multipoles: the Legendre-weighted spectrum through the same inverse, into slots nshell .. 2 nshell - 1
        // (the cell-tiled layout puts slot s of a 32-cell block at s * 32, so the base moves by nshell * 32)
        const size_t es = p->is_double ? 8 : 4;
        void* out_w = (char*)p->d_fields + (size_t)p->nshell * 32 * es;
        if ((e = ps_legendre_weight(p->is_double, p->d_fhat, p->K, p->ell, p->d_fhat_w, st)))
            return cuda_error(e, "multipole weights");
        if (p->is_double)
            e = ps_inverse(p->N, 1, 0, p->d_fhat_w, p->d_lines, p->d_line_off, 0, p->nshell, p->K, 0, p->N,
                           p->d_tw_inv, out_w, (size_t)p->N * p->N * p->N, p->d_spill, p->d_xpre, p->max_lines,
                           p->nfield, st);
        else
            e = ps_inverse_ranged_f32(p->N, p->d_fhat_w, p->d_lines, p->d_line_off, 0, p->nshell, p->K, p->d_tw_inv,
                                      out_w, (size_t)p->N * p->N * p->N, p->d_xpre, p->max_lines, p->nfield,
                                      p->shell_kz.data(), p->d_shell_kz, st);
        if (e) return cuda_error(e, "weighted shell fields");
        p->launches += 3;
    }
    mark(p, 2, st);
    return POLY_OK;
}

poly_status ps_sums(PsPlan* p, bool absval, cudaStream_t st) {
    cudaError_t e;
    if (p->prec == POLY_SPLIT_BF16 && !absval) return ps_tc_sums(p, st);
    const size_t n3 = (size_t)p->N * p->N * p->N;
    if ((e = ps_contract_cc(p->is_double, 0, absval ? 1 : 0, p->order >= 5 ? 3 : 2, p->d_fields, n3, p->nfield, (int64_t)n3, nullptr,
                            (const PsTile*)p->d_cc_tiles, (int)p->cc.tiles.size(), (const int*)p->d_cc_field_ids,
                            (const short4*)p->d_cc_rowf, (const short4*)p->d_cc_colf, p->cc_nsplit, p->cc_cps,
                            p->d_partial, st)))
        return cuda_error(e, "contraction");
    if (!absval) mark(p, 3, st);
    if ((e = ps_reduce_slots(p->d_partial, p->cc_nsplit, p->cc_slot_stride, (const int64_t*)p->d_cc_slot, p->nbins,
                             p->d_S, st)))
        return cuda_error(e, "contraction");
    p->launches += 2;
    return POLY_OK;
}

double ps_norm(const PsPlan* p) {  // c_n, times 2 ell + 1 for a multipole plan
    const double n3 = (double)p->N * p->N * p->N;
    return (2.0 * p->ell + 1.0) * std::pow(p->L * p->L * p->L, p->order - 1) / std::pow(n3, p->order);
}

poly_status ps_estimate_impl(PsPlan* p, const void* delta, double* out, double* scale, cudaStream_t st) {
    PS_TRY(ps_fields(p, delta, st));
    PS_TRY(ps_sums(p, false, st));
    const double n3 = (double)p->N * p->N * p->N;
    cudaError_t e;
    if ((e = ps_normalise(p->d_S, p->d_counts, p->nbins, ps_norm(p), n3, out, st)))
        return cuda_error(e, "normalise");
    p->launches += 1;
    mark(p, 4, st);
    if (p->timing) p->ev_recorded = true;
    if (scale) {
        PS_TRY(ps_sums(p, true, st));
        if ((e = ps_normalise(p->d_S, p->d_counts, p->nbins, 1.0, n3, scale, st))) return cuda_error(e, "scale");
        p->launches += 1;
    }
    return POLY_OK;
}

// B_disc of every bin (order-4 plans): forward transform, shell powers, per-bin Wick pairings
static poly_status ps_disconnected_impl(PsPlan* p, const void* delta, double* out, double* power, cudaStream_t st) {
    // each buffer is recorded only once it is complete, so a failure here is retried on the next call
    if (!p->d_bins) {
        void* d = nullptr;
        PS_TRY(upload(p, &d, p->bins));
        p->d_bins = (int32_t*)d;
    }
    if (!p->d_shell_power) {
        void* d = nullptr;
        PS_TRY(ps_alloc(p, &d, (size_t)p->nshell * sizeof(double)));
        p->d_shell_power = (double*)d;
    }
    cudaError_t e;
    if ((e = ps_forward(p->N, p->is_double, delta, p->K, p->d_tw_fwd, p->d_W, p->d_fhat, p->d_spill, st)))
        return cuda_error(e, "forward transform");
    const double n3 = (double)p->N * p->N * p->N;
    if ((e = ps_disconnected(p->is_double, p->d_fhat, p->d_lines, p->d_line_off, p->nshell, p->K, p->d_bins,
                             p->d_counts, p->nbins, ps_norm(p), n3, p->d_shell_power, out, st)))
        return cuda_error(e, "disconnected part");
    p->launches += 4;
    if (power && (e = cudaMemcpyAsync(power, p->d_shell_power, (size_t)p->nshell * sizeof(double),
                                      cudaMemcpyDeviceToDevice, st)))
        return cuda_error(e, "shell power copy");
    return POLY_OK;
}

static poly_status enter(poly_plan p, int* prev) {
    if (!p) return set_error(POLY_ERR_ARG, "NULL plan");
    *prev = -1;
    cudaGetDevice(prev);
    if (*prev != p->device) {
        cudaError_t e = cudaSetDevice(p->device);
        if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    }
    return POLY_OK;
}

static void leave(poly_plan p, int prev) {
    if (prev >= 0 && prev != p->device) cudaSetDevice(prev);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

poly_status poly_plan_create(poly_plan* out, int N, double L, int order, int nshell, const double* edges,
                             poly_precision prec, unsigned flags) {
    return poly_plan_create_multipole(out, N, L, order, nshell, edges, prec, flags, 0);
}

poly_status poly_plan_create_multipole(poly_plan* out, int N, double L, int order, int nshell, const double* edges,
                                       poly_precision prec, unsigned flags, int ell) {
    if (!out) return set_error(POLY_ERR_ARG, "NULL output pointer");
    *out = nullptr;
    g_last_error.clear();
    PsPlan* p = new (std::nothrow) PsPlan();
    if (!p) return set_error(POLY_ERR_ALLOC, "host allocation failed");
    poly_status s;
    try {
        s = create_plan(p, N, L, order, nshell, edges, prec, flags, ell);
    } catch (const std::bad_alloc&) {
        s = set_error(POLY_ERR_ALLOC, "host allocation failed");
    } catch (const std::exception& ex) {
        s = set_error(POLY_ERR_ARG, ex.what());
    }
    if (s != POLY_OK) {
        free_plan(p);
        return s;
    }
    *out = p;
    return POLY_OK;
}

poly_status poly_plan_nbins(poly_plan p, int64_t* nbins) {
    if (!p || !nbins) return set_error(POLY_ERR_ARG, "NULL argument");
    *nbins = p->nbins;
    return POLY_OK;
}

poly_status poly_plan_bins(poly_plan p, int32_t* idx) {
    if (!p || !idx) return set_error(POLY_ERR_ARG, "NULL argument");
    std::memcpy(idx, p->bins.data(), p->bins.size() * sizeof(int32_t));
    return POLY_OK;
}

poly_status poly_plan_counts(poly_plan p, int64_t* counts) {
    if (!p || !counts) return set_error(POLY_ERR_ARG, "NULL argument");
    std::memcpy(counts, p->counts.data(), p->counts.size() * sizeof(int64_t));
    return POLY_OK;
}

poly_status poly_plan_device_bytes(poly_plan p, int64_t* bytes) {
    if (!p || !bytes) return set_error(POLY_ERR_ARG, "NULL argument");
    int64_t sum = 0;
    for (size_t b : p->allocation_bytes) sum += (int64_t)b;
    *bytes = sum;
    return POLY_OK;
}

poly_status poly_plan_bin_wraps(poly_plan p, uint8_t* wraps) {
    if (!p || !wraps) return set_error(POLY_ERR_ARG, "NULL argument");
    bin_wraps(p, wraps);
    return POLY_OK;
}

poly_status poly_estimate(poly_plan p, const void* delta_x, double* out, double* scale_or_null, void* stream) {
    if (!p || !delta_x || !out) return set_error(POLY_ERR_ARG, "NULL argument");
    if ((const void*)out == delta_x || (const void*)scale_or_null == delta_x || out == scale_or_null)
        return set_error(POLY_ERR_ARG, "output aliases an input");
    int prev;
    PS_TRY(enter(p, &prev));
    poly_status s = ps_estimate_impl(p, delta_x, out, scale_or_null, (cudaStream_t)stream);
    leave(p, prev);
    return s;
}

poly_status poly_trispectrum_disconnected(poly_plan p, const void* delta_x, double* out, double* shell_power_or_null,
                                          void* stream) {
    if (!p || !delta_x || !out) return set_error(POLY_ERR_ARG, "NULL argument");
    if (p->order != 4 || p->ell != 0)
        return set_error(POLY_ERR_UNSUPPORTED, "the disconnected part is defined for order-4 monopole plans");
    if ((const void*)out == delta_x || (const void*)shell_power_or_null == delta_x ||
        (const void*)shell_power_or_null == (const void*)out)
        return set_error(POLY_ERR_ARG, "output aliases an input");
    int prev;
    PS_TRY(enter(p, &prev));
    poly_status s = guarded([&] { return ps_disconnected_impl(p, delta_x, out, shell_power_or_null, (cudaStream_t)stream); });
    leave(p, prev);
    return s;
}

poly_status poly_trispectrum_full(poly_plan p, const void* delta_x, const int32_t* k, int ndiag, const double* dedges,
                                  double* T_out, int64_t* counts_out, double* scale_or_null, void* stream) {
    if (!p) return set_error(POLY_ERR_ARG, "NULL plan");
    int prev;
    PS_TRY(enter(p, &prev));
    poly_status s = guarded([&] {
        return ps_trispectrum_full_impl(p, delta_x, k, ndiag, dedges, T_out, counts_out, scale_or_null,
                                        (cudaStream_t)stream);
    });
    leave(p, prev);
    return s;
}

static int poly_diag_fields_impl(void* plan, const void* delta_x, void* fields_host, void* stream) {
    PsPlan* p = (PsPlan*)plan;
    if (!p || !delta_x || !fields_host) return set_error(POLY_ERR_ARG, "NULL argument");
    const size_t n3 = (size_t)p->N * p->N * p->N, es = p->is_double ? 8 : 4, nf = (size_t)p->nfield;
    std::vector<unsigned char> tiled(nf * n3 * es);  // before enter(): a failed allocation leaves the device as it was
    int prev;
    PS_TRY(enter(p, &prev));
    cudaStream_t st = (cudaStream_t)stream;
    poly_status s = ps_fields(p, delta_x, st);
    cudaError_t e;
    if (!s && (e = cudaStreamSynchronize(st))) s = cuda_error(e, "stream synchronise");
    if (!s) {
        if ((e = cudaMemcpy(tiled.data(), p->d_fields, tiled.size(), cudaMemcpyDeviceToHost)))
            s = cuda_error(e, "device to host copy");
    }
    if (!s) {  // cell-tiled [cell / 32][slot][cell % 32] -> natural [slot][cell]
        unsigned char* out = (unsigned char*)fields_host;
        for (size_t f = 0; f < nf; f++)
            for (size_t cell = 0; cell < n3; cell++)
                std::memcpy(out + (f * n3 + cell) * es, tiled.data() + ((cell >> 5) * nf * 32 + f * 32 + (cell & 31)) * es, es);
    }
    leave(p, prev);
    return s;
}

int poly_diag_fields(void* plan, const void* delta_x, void* fields_host, void* stream) {
    try {
        return poly_diag_fields_impl(plan, delta_x, fields_host, stream);
    } catch (const std::bad_alloc&) {
        return set_error(POLY_ERR_ALLOC, "host allocation failed");
    } catch (const std::exception& ex) {
        return set_error(POLY_ERR_ARG, ex.what());
    }
}

static int poly_diag_count_wedge_impl(int N, int64_t* ncell, int32_t* cells, double* weights) {
    if (!ncell || N < 2 || (N & 1)) return set_error(POLY_ERR_ARG, "N must be even");
    std::vector<int32_t> widx;
    std::vector<double> wgt;
    count_wedge(N, widx, wgt);
    *ncell = (int64_t)widx.size();
    if (cells) std::memcpy(cells, widx.data(), widx.size() * sizeof(int32_t));
    if (weights) std::memcpy(weights, wgt.data(), wgt.size() * sizeof(double));
    return POLY_OK;
}

int poly_diag_count_wedge(int N, int64_t* ncell, int32_t* cells, double* weights) {
    try {
        return poly_diag_count_wedge_impl(N, ncell, cells, weights);
    } catch (const std::bad_alloc&) {
        return set_error(POLY_ERR_ALLOC, "host allocation failed");
    } catch (const std::exception& ex) {
        return set_error(POLY_ERR_ARG, ex.what());
    }
}

static int poly_diag_host_tables_impl(int N, int order, const double* edges, int nshell, unsigned flags, int ell,
                                      int64_t* sizes, int32_t* bins, int32_t* tiles, int32_t* field_ids,
                                      int16_t* rowf, int16_t* colf, int64_t* slot, int16_t* lines,
                                      int32_t* line_off) {
    if (!sizes) return set_error(POLY_ERR_ARG, "NULL sizes");
    PsPlan h;  // host tables only: no device call, no device memory
    std::vector<short> ln;
    PS_TRY(ps_plan_host_tables(&h, N, 1.0, order, nshell, edges, POLY_FP64, flags, ell, ln));
    if (ell > 0) {  // as poly_plan_create_multipole leaves them: the first leg on the weighted slots
        h.cc = CcTiles();
        build_cc_tiles(&h, h.cc, nshell);
    }
    const int64_t n[7] = {h.nbins, (int64_t)h.cc.tiles.size(), (int64_t)h.cc.field_ids.size(),
                          (int64_t)h.cc.rowf.size(), (int64_t)h.cc.colf.size(), (int64_t)ln.size() / 4,
                          (int64_t)h.line_off.size()};
    for (int i = 0; i < 7; i++) sizes[i] = n[i];
    if (bins) std::memcpy(bins, h.bins.data(), h.bins.size() * sizeof(int32_t));
    if (tiles) std::memcpy(tiles, h.cc.tiles.data(), h.cc.tiles.size() * sizeof(PsTile));
    if (field_ids) std::memcpy(field_ids, h.cc.field_ids.data(), h.cc.field_ids.size() * sizeof(int32_t));
    if (rowf) std::memcpy(rowf, h.cc.rowf.data(), h.cc.rowf.size() * sizeof(short4));
    if (colf) std::memcpy(colf, h.cc.colf.data(), h.cc.colf.size() * sizeof(short4));
    if (slot) std::memcpy(slot, h.cc.slot.data(), h.cc.slot.size() * sizeof(int64_t));
    if (lines) std::memcpy(lines, ln.data(), ln.size() * sizeof(short));
    if (line_off) std::memcpy(line_off, h.line_off.data(), h.line_off.size() * sizeof(int32_t));
    return POLY_OK;
}

static int poly_diag_bin_wraps_impl(int N, int order, const double* edges, int nshell, unsigned flags,
                                    int64_t* nbins, uint8_t* wraps) {
    if (!nbins) return set_error(POLY_ERR_ARG, "NULL nbins");
    PsPlan h;  // host tables only: no device call, no device memory
    std::vector<short> ln;
    PS_TRY(ps_plan_host_tables(&h, N, 1.0, order, nshell, edges, POLY_FP64, flags, 0, ln));
    *nbins = h.nbins;
    if (wraps) bin_wraps(&h, wraps);
    return POLY_OK;
}

int poly_diag_bin_wraps(int N, int order, const double* edges, int nshell, unsigned flags, int64_t* nbins,
                        uint8_t* wraps) {
    try {
        return poly_diag_bin_wraps_impl(N, order, edges, nshell, flags, nbins, wraps);
    } catch (const std::bad_alloc&) {
        return set_error(POLY_ERR_ALLOC, "host allocation failed");
    } catch (const std::exception& ex) {
        return set_error(POLY_ERR_ARG, ex.what());
    }
}

int poly_diag_host_tables(int N, int order, const double* edges, int nshell, unsigned flags, int ell,
                          int64_t* sizes, int32_t* bins, int32_t* tiles, int32_t* field_ids, int16_t* rowf,
                          int16_t* colf, int64_t* slot, int16_t* lines, int32_t* line_off) {
    try {
        return poly_diag_host_tables_impl(N, order, edges, nshell, flags, ell, sizes, bins, tiles, field_ids, rowf, colf,
                                          slot, lines, line_off);
    } catch (const std::bad_alloc&) {
        return set_error(POLY_ERR_ALLOC, "host allocation failed");
    } catch (const std::exception& ex) {
        return set_error(POLY_ERR_ARG, ex.what());
    }
}

poly_status poly_estimate_host(poly_plan p, const void* delta_x_host, double* out_host, void* stream) {
    if (!p || !delta_x_host || !out_host) return set_error(POLY_ERR_ARG, "NULL argument");
    int prev;
    PS_TRY(enter(p, &prev));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)p->N * p->N * p->N * (p->is_double ? 8 : 4);
    poly_status s = POLY_OK;
    cudaError_t e = cudaMemcpyAsync(p->d_in_stage, delta_x_host, bytes, cudaMemcpyHostToDevice, st);
    if (e) s = cuda_error(e, "host to device copy");
    if (!s) s = ps_estimate_impl(p, p->d_in_stage, p->d_out_stage, nullptr, st);
    if (!s && (e = cudaMemcpyAsync(out_host, p->d_out_stage, p->nbins * 8, cudaMemcpyDeviceToHost, st)))
        s = cuda_error(e, "device to host copy");
    if (!s && (e = cudaStreamSynchronize(st))) s = cuda_error(e, "stream synchronise");
    if (!s) s = ps_check_device_error(p);
    leave(p, prev);
    return s;
}

poly_status poly_backward(poly_plan p, const void* delta_x, const double* dL_dB, void* dL_ddelta, void* stream) {
    if (!p || !delta_x || !dL_dB || !dL_ddelta) return set_error(POLY_ERR_ARG, "NULL argument");
    if (dL_ddelta == delta_x || dL_ddelta == (const void*)dL_dB) return set_error(POLY_ERR_ARG, "output aliases an input");
    int prev;
    PS_TRY(enter(p, &prev));
    poly_status s = guarded([&] { return ps_backward_impl(p, delta_x, dL_dB, dL_ddelta, (cudaStream_t)stream); });
    leave(p, prev);
    return s;
}

poly_status poly_estimate_batched(const poly_plan* plans, const void* const* fields, double* const* outs, int count,
                                  void* stream) {
    if (count < 0 || (count > 0 && (!plans || !fields || !outs))) return set_error(POLY_ERR_ARG, "bad batch");
    for (int i = 0; i < count; i++)
        if (!plans[i] || !fields[i] || !outs[i]) return set_error(POLY_ERR_ARG, "NULL entry in batch");
    return guarded([&] { return ps_batched_impl(plans, fields, outs, count, (cudaStream_t)stream); });
}

poly_status poly_plan_sync(poly_plan p, void* stream) {
    int prev;
    if (!p) return set_error(POLY_ERR_ARG, "NULL plan");
    prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->device) cudaSetDevice(p->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    poly_status s = e ? cuda_error(e, "stream synchronise") : ps_check_device_error(p);
    leave(p, prev);
    return s;
}

void poly_plan_destroy(poly_plan p) { free_plan(p); }

poly_status poly_plan_set_timing(poly_plan p, int enable) {
    if (!p) return set_error(POLY_ERR_ARG, "NULL plan");
    if (enable && !p->ev[0]) {
        int prev;
        PS_TRY(enter(p, &prev));
        for (auto& e : p->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r) {
                leave(p, prev);
                return cuda_error(r, "cudaEventCreate");
            }
        }
        leave(p, prev);
    }
    p->timing = enable != 0;
    p->ev_recorded = false;
    return POLY_OK;
}

// ---------------------------------------------------------------------------
// tunable shape of the tensor-core contraction
// ---------------------------------------------------------------------------
static poly_status apply_tc_config(PsPlan* p, int max_mt, int cta_mult) {
    const int old_mt = p->tc_max_mt, old_mult = p->tc_cta_mult;
    p->tc_max_mt = max_mt;
    p->tc_cta_mult = cta_mult;
    ps_batched_forget(p);  // cached graphs hold the old tables
    ps_tc_free(p);
    const poly_status s = guarded([&] { return ps_tc_prepare(p); });
    if (s) {  // a shape that does not fit: rebuild the previous one, so the plan stays usable
        ps_tc_free(p);
        p->tc_max_mt = old_mt;
        p->tc_cta_mult = old_mult;
        if (guarded([&] { return ps_tc_prepare(p); })) ps_tc_free(p);  // then ps_tc_sums reports UNSUPPORTED
    }
    return s;
}

static bool decode_config(int config, int* max_mt, int* cta_mult) {
    *max_mt = config & 15;
    *cta_mult = (config >> 4) & 15;
    return *max_mt >= 1 && *max_mt <= 4 && (*cta_mult == 1 || *cta_mult == 2 || *cta_mult == 4 || *cta_mult == 6 ||
                                            *cta_mult == 8) &&
           (config >> 8) == 0;
}

poly_status poly_plan_tune(poly_plan p, const void* delta_x, int* config_out, double* ms_out, void* stream) {
    if (!p || !delta_x || !config_out || !ms_out) return set_error(POLY_ERR_ARG, "NULL argument");
    *config_out = 0;
    *ms_out = 0;
    if (p->prec != POLY_SPLIT_BF16) return POLY_OK;  // only the tensor-core contraction has a tunable shape
    int prev;
    PS_TRY(enter(p, &prev));
    cudaStream_t st = (cudaStream_t)stream;
    const bool timing = p->timing;
    p->timing = false;
    const int old_mt = p->tc_max_mt, old_mult = p->tc_cta_mult;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    poly_status s = ps_fields(p, delta_x, st);
    if (!s && (cudaEventCreate(&e0) || cudaEventCreate(&e1))) s = set_error(POLY_ERR_CUDA, "cudaEventCreate");
    float best = -1.f;
    int best_mt = old_mt, best_mult = old_mult;
    for (int mt = 2; mt <= 4 && !s; mt++)
        for (int mult : {1, 2, 4, 6, 8}) {  // CTA budget of 1/2 to 4 waves
            if (s) break;
            poly_status a = apply_tc_config(p, mt, mult);
            if (a == POLY_ERR_UNSUPPORTED) continue;  // this grouping does not fit
            if (a) {
                s = a;
                break;
            }
            cudaError_t e = cudaSuccess;
            if ((s = ps_tc_sums(p, st))) break;  // warm-up
            if ((e = cudaEventRecord(e0, st))) s = cuda_error(e, "cudaEventRecord");
            for (int r = 0; r < 3 && !s; r++) s = ps_tc_sums(p, st);
            if (!s && (e = cudaEventRecord(e1, st))) s = cuda_error(e, "cudaEventRecord");
            if (!s && (e = cudaEventSynchronize(e1))) s = cuda_error(e, "cudaEventSynchronize");
            if (!s) s = ps_check_device_error(p);
            float ms = 0.f;
            if (!s) cudaEventElapsedTime(&ms, e0, e1);
            if (!s && (best < 0 || ms < best)) {
                best = ms;
                best_mt = mt;
                best_mult = mult;
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    poly_status a = apply_tc_config(p, s ? old_mt : best_mt, s ? old_mult : best_mult);
    if (!s) s = a;
    p->timing = timing;
    if (!s) {
        *config_out = best_mt | (best_mult << 4);
        *ms_out = best / 3.0;
    }
    leave(p, prev);
    return s;
}

poly_status poly_plan_set_config(poly_plan p, int config) {
    if (!p) return set_error(POLY_ERR_ARG, "NULL plan");
    if (config == 0) return POLY_OK;
    int mt, mult;
    if (!decode_config(config, &mt, &mult)) return set_error(POLY_ERR_ARG, "not a configuration from poly_plan_tune");
    if (p->prec != POLY_SPLIT_BF16) return POLY_OK;
    if (mt == p->tc_max_mt && mult == p->tc_cta_mult) return POLY_OK;
    int prev;
    PS_TRY(enter(p, &prev));
    poly_status s = apply_tc_config(p, mt, mult);
    leave(p, prev);
    return s;
}

poly_status poly_plan_stats(poly_plan p, poly_stats* out) {
    if (!p || !out) return set_error(POLY_ERR_ARG, "NULL argument");
    std::memset(out, 0, sizeof *out);
    out->launches = p->launches;
    {
        const double n3 = (double)p->N * p->N * p->N;
        double f = 0;
        if (p->prec == POLY_SPLIT_BF16) f = ps_tc_executed_flops(p);
        else
            for (const auto& t : p->cc.tiles) f += 2.0 * 512.0 * __builtin_popcount(t.region_mask) * n3;
        out->contract_flops = f;
    }
    if (!p->ev_recorded) return POLY_OK;
    int prev;
    PS_TRY(enter(p, &prev));
    float ms[4] = {0, 0, 0, 0};
    cudaError_t e = cudaEventSynchronize(p->ev[4]);
    for (int i = 0; i < 4 && !e; i++) e = cudaEventElapsedTime(&ms[i], p->ev[i], p->ev[i + 1]);
    leave(p, prev);
    if (e) return cuda_error(e, "stage events");
    out->ms_forward = ms[0];
    out->ms_fields = ms[1];
    out->ms_contract = ms[2];
    out->ms_reduce = ms[3];
    return POLY_OK;
}

const char* poly_status_string(poly_status s) {
    switch (s) {
        case POLY_OK: return "ok";
        case POLY_ERR_ARG: return "invalid argument";
        case POLY_ERR_ALIAS: return "grid too small: polygon closures alias (n*K >= N)";
        case POLY_ERR_ALLOC: return "allocation failed";
        case POLY_ERR_CUDA: return "CUDA error";
        case POLY_ERR_TIMEOUT: return "device wait timed out";
        case POLY_ERR_UNSUPPORTED: return "unsupported configuration";
        case POLY_ERR_COUNT: return "non-integral polygon count";
    }
    return "unknown status";
}

const char* poly_last_error(void) { return g_last_error.c_str(); }

void poly_debug_fail_alloc_after(int n) { g_fail_alloc_after = n > 0 ? n : 0; }

}  // extern "C"
