// Bispectrum of a small field without allocating device memory.
//
// Some callers cannot call cudaMalloc when they need an estimate: code that
// runs after a memory budget has been fixed and must not allocate any more, or
// code inside a framework whose device allocator belongs to someone else.
// poly_estimate_noalloc serves them: it runs the same kernels as poly_estimate,
// with every intermediate (twiddles, shell tables, spectrum, shell fields,
// contraction partials, sums, counts) placed in one static device array that
// belongs to this library.
//
// Each call builds its host tables (twiddles, shell line tables, contraction
// tiles) in ordinary pageable host memory and copies them, and the counts, into
// the array with cudaMemcpyAsync.  Copies from pageable memory are staged
// through the driver, so a call can wait for its stream before it returns; it
// is not a zero-latency call.
//
// The array costs kNoAllocBytes on every GPU that loads the library, until the
// process exits.  Its device address is looked up once per device, on the first
// call made with that device current (so make that first call before any stream
// capture).  All calls share the array: two calls whose work overlaps on the
// GPU (different streams, or different host threads) race on it.  Each call
// overwrites every region it reads before reading it, so nothing depends on
// what an earlier call left behind.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/polyspec.h"
#include "kernels.h"
#include "plan_internal.h"

namespace {
constexpr size_t kNoAllocBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

poly_status fail(poly_status s, const std::string& msg) {
    ps_set_last_error(msg);  // reported by poly_last_error()
    return s;
}
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the static array for the current device (looked up once per device).
static poly_status scratch_for_current_device(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(POLY_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(POLY_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(POLY_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return POLY_OK;
}

namespace {
struct Carve {  // 256-byte aligned sub-ranges of the static array
    size_t used = 0;
    size_t take(size_t bytes) {
        const size_t off = used;
        used += (bytes + 255) / 256 * 256;
        return off;
    }
};
}  // namespace

static poly_status estimate_noalloc(int N, double L, int nshell, const double* edges, const float* delta_x,
                                    const int64_t* counts, double* out, void* stream) {
    if (!edges || !delta_x || !counts || !out) return fail(POLY_ERR_ARG, "NULL argument");
    if (nshell < 1 || nshell > 128) return fail(POLY_ERR_ARG, "nshell must be in [1, 128]");
    if (!(L > 0) || !std::isfinite(L)) return fail(POLY_ERR_ARG, "L must be positive");
    if (!ps_supported_n(N)) return fail(POLY_ERR_UNSUPPORTED, "grid size N not in the supported set");
    for (int s = 0; s <= nshell; s++)
        if (!std::isfinite(edges[s]) || edges[s] < 0 || (s < nshell && !(edges[s + 1] > edges[s])))
            return fail(POLY_ERR_ARG, "edges must be finite, non-negative and strictly increasing");
    const int order = 3;
    PsPlan hp;  // host-side tables only; owns no device memory
    hp.N = N;
    hp.L = L;
    hp.order = order;
    hp.nshell = nshell;
    hp.edges.assign(edges, edges + nshell + 1);
    const double emax2 = edges[nshell] * edges[nshell];
    int K = 0;
    while ((double)((long long)(K + 1) * (K + 1)) < emax2) K++;
    hp.K = K;
    if (2 * K + 1 > N) return fail(POLY_ERR_ARG, "outer shell edge exceeds the Nyquist frequency");
    if ((long long)order * K >= N) return fail(POLY_ERR_ALIAS, "3 * K >= N: triangle closures would wrap around");
    if (ps_plane_needs_spill(N, K, 0) != 0) return fail(POLY_ERR_UNSUPPORTED, "grid too large for this entry point");
    enumerate_bins(nshell, hp.edges, order, false, hp.bins);
    hp.nbins = (int64_t)hp.bins.size() / order;
    std::vector<short> lines;
    std::vector<int> line_off{0};
    for (int s = 0; s < nshell; s++) {
        build_lines(&hp, hp.edges.data(), s, lines);
        line_off.push_back((int)(lines.size() / 4));
    }
    build_cc_tiles(&hp, hp.cc);
    const int ntiles = (int)hp.cc.tiles.size();
    const int64_t n3 = (int64_t)N * N * N;
    const int64_t chunk = ps_cc_chunk(0);
    const int64_t nchunks = (n3 + chunk - 1) / chunk;
    const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(64, nchunks / 16));
    const int64_t cps = (nchunks + nsplit - 1) / nsplit;
    const int64_t slot_stride = (int64_t)ntiles * kCcTM * kCcTN;
    const size_t nl = (size_t)(2 * K + 1) * (K + 1);

    // layout of the static array
    Carve c;
    const size_t o_twf = c.take((size_t)N * 16), o_twi = c.take((size_t)N * 16);
    const size_t o_lines = c.take(lines.size() * sizeof(short)), o_loff = c.take(line_off.size() * sizeof(int));
    const size_t o_W = c.take((size_t)N * nl * 8), o_fhat = c.take(nl * (2 * K + 1) * 8);
    const size_t o_fields = c.take((size_t)nshell * n3 * 4);
    const size_t o_tiles = c.take(hp.cc.tiles.size() * sizeof(PsTile));
    const size_t o_fid = c.take(hp.cc.field_ids.size() * sizeof(int));
    const size_t o_rowf = c.take(hp.cc.rowf.size() * sizeof(short4)), o_colf = c.take(hp.cc.colf.size() * sizeof(short4));
    const size_t o_slot = c.take(hp.cc.slot.size() * sizeof(int64_t));
    const size_t o_part = c.take((size_t)nsplit * slot_stride * 8);
    const size_t o_S = c.take((size_t)hp.nbins * 8), o_cnt = c.take((size_t)hp.nbins * 8);
    if (c.used > kNoAllocBytes)
        return fail(POLY_ERR_UNSUPPORTED, "this problem needs " + std::to_string(c.used >> 20) +
                                              " MiB of scratch; the static array holds 32 MiB");

    void* base = nullptr;
    poly_status st0 = scratch_for_current_device(&base);
    if (st0) return st0;
    unsigned char* B = (unsigned char*)base;
    cudaStream_t st = (cudaStream_t)stream;

    std::vector<double> twf(2 * N), twi(2 * N);
    for (int m = 0; m < N; m++) {
        const double a = 2.0 * 3.14159265358979323846 * (double)m / (double)N;
        twf[2 * m] = std::cos(a);
        twf[2 * m + 1] = -std::sin(a);
        twi[2 * m] = std::cos(a);
        twi[2 * m + 1] = std::sin(a);
    }
    struct Copy {
        size_t off;
        const void* src;
        size_t bytes;
    } copies[] = {{o_twf, twf.data(), twf.size() * 8},
                  {o_twi, twi.data(), twi.size() * 8},
                  {o_lines, lines.data(), lines.size() * sizeof(short)},
                  {o_loff, line_off.data(), line_off.size() * sizeof(int)},
                  {o_tiles, hp.cc.tiles.data(), hp.cc.tiles.size() * sizeof(PsTile)},
                  {o_fid, hp.cc.field_ids.data(), hp.cc.field_ids.size() * sizeof(int)},
                  {o_rowf, hp.cc.rowf.data(), hp.cc.rowf.size() * sizeof(short4)},
                  {o_colf, hp.cc.colf.data(), hp.cc.colf.size() * sizeof(short4)},
                  {o_slot, hp.cc.slot.data(), hp.cc.slot.size() * sizeof(int64_t)},
                  {o_cnt, counts, (size_t)hp.nbins * 8}};
    for (const Copy& cp : copies)
        if (cp.bytes) {
            cudaError_t e = cudaMemcpyAsync(B + cp.off, cp.src, cp.bytes, cudaMemcpyHostToDevice, st);
            if (e) return fail(POLY_ERR_CUDA, std::string("copy into scratch: ") + cudaGetErrorString(e));
        }
    cudaError_t e;
    if ((e = ps_forward(N, 0, delta_x, K, B + o_twf, B + o_W, B + o_fhat, nullptr, st)) ||
        (e = ps_inverse(N, 0, 0, B + o_fhat, B + o_lines, (const int*)(B + o_loff), 0, nshell, K, 0, N, B + o_twi,
                        B + o_fields, (size_t)n3, nullptr, nullptr, 0, nshell, st)) ||
        (e = ps_contract_cc(0, 0, 0, 2, B + o_fields, (size_t)n3, nshell, n3, nullptr, (const PsTile*)(B + o_tiles), ntiles,
                            (const int*)(B + o_fid), (const short4*)(B + o_rowf), (const short4*)(B + o_colf), nsplit,
                            cps, (double*)(B + o_part), st)) ||
        (e = ps_reduce_slots((const double*)(B + o_part), nsplit, slot_stride, (const int64_t*)(B + o_slot), hp.nbins,
                             (double*)(B + o_S), st)))
        return fail(POLY_ERR_CUDA, std::string("estimate kernels: ") + cudaGetErrorString(e));
    const double n3d = (double)n3;
    const double norm = std::pow(L * L * L, order - 1) / std::pow(n3d, order);
    if ((e = ps_normalise((const double*)(B + o_S), (const int64_t*)(B + o_cnt), hp.nbins, norm, n3d, out, st)))
        return fail(POLY_ERR_CUDA, std::string("normalise: ") + cudaGetErrorString(e));
    return POLY_OK;
}

extern "C" poly_status poly_estimate_noalloc(int N, double L, int nshell, const double* edges, const float* delta_x,
                                             const int64_t* counts, double* out, void* stream) {
    try {  // the host tables are std::vectors: no C++ exception crosses the C ABI
        return estimate_noalloc(N, L, nshell, edges, delta_x, counts, out, stream);
    } catch (const std::bad_alloc&) {
        return fail(POLY_ERR_ALLOC, "host allocation failed");
    } catch (const std::exception& ex) {
        return fail(POLY_ERR_ARG, ex.what());
    }
}
