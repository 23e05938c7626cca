// Adjoint of the estimator for a loss L = sum_b g_b B_b (g = dL/dB):
//   B_b = c_n S_b / (N^3 count_b),  S_b = sum_x prod_t D_{b_t}(x),  c_n = V^{n-1}/N^{3n}
//   G_m(x) = dL/dD_m(x) = sum_b g_b c_n/(N^3 count_b) sum_{t: b_t = m} prod_{u != t} D_{b_u}(x)
//   D_m = inverse(mask_m forward(delta))  =>  dL/d delta(y) = sum_q [mask_{m(q)}(q) Ghat_{m(q)}(q)] e^{+i q.y}
// (the shell kernels are real and even, and the shells are disjoint).
//
// The contraction runs over "entries" e = (m, other factors) with weight
// w_e = sum over the (bin, position) pairs that produce e of g_b / count_b; the
// constant c_n / N^3 is applied when the transformed G_m are gathered.
#include <algorithm>
#include <array>
#include <map>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "plan_internal.h"

namespace ps {

constexpr int kAdjChunk = 64;  // cells per block
constexpr int kAdjThreads = 256;

// w_e = sum_{k in [off[e], off[e+1])} g[bin[k]] / count[bin[k]]
template <typename T>
__global__ void adj_weights_kernel(const double* __restrict__ g, const int64_t* __restrict__ counts,
                                   const int* __restrict__ off, const int* __restrict__ bins, int nent,
                                   T* __restrict__ w) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nent; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = off[e]; k < off[e + 1]; k++) {
            const int b = bins[k];
            if (counts[b] > 0) s += g[b] / (double)counts[b];
        }
        w[e] = (T)s;
    }
}

// G[m][x] = sum_{e of m} w_e prod_{f in factors(e)} D[f][x]; one warp per output shell at a time.
template <typename T>
__global__ void __launch_bounds__(kAdjThreads) adj_g_kernel(const T* __restrict__ D, int nshell, int64_t ncell,
                                                             const int* __restrict__ m_off,
                                                             const short4* __restrict__ ent, const T* __restrict__ w,
                                                             T* __restrict__ G) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s_d = reinterpret_cast<T*>(smem_raw);  // [nshell][kAdjChunk]
    const int64_t x0 = (int64_t)blockIdx.x * kAdjChunk;
    for (int i = threadIdx.x; i < nshell * kAdjChunk; i += blockDim.x) {  // D is cell-tiled over nshell shells
        const int s = i / kAdjChunk, x = i - s * kAdjChunk;
        const int64_t cell = x0 + x;
        s_d[i] = cell < ncell ? D[(size_t)(cell >> 5) * nshell * 32 + (size_t)s * 32 + (cell & 31)] : (T)0;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int m = warp; m < nshell; m += kAdjThreads / 32) {
        T g0 = 0, g1 = 0;
        for (int e = m_off[m]; e < m_off[m + 1]; e++) {
            const short4 f = ent[e];
            const T we = w[e];
            T p0 = we * s_d[f.x * kAdjChunk + lane], p1 = we * s_d[f.x * kAdjChunk + lane + 32];
            if (f.y >= 0) {
                p0 *= s_d[f.y * kAdjChunk + lane];
                p1 *= s_d[f.y * kAdjChunk + lane + 32];
            }
            if (f.z >= 0) {
                p0 *= s_d[f.z * kAdjChunk + lane];
                p1 *= s_d[f.z * kAdjChunk + lane + 32];
            }
            g0 += p0;
            g1 += p1;
        }
        if (x0 + lane < ncell) G[(size_t)m * ncell + x0 + lane] = g0;
        if (x0 + lane + 32 < ncell) G[(size_t)m * ncell + x0 + lane + 32] = g1;
    }
}

// H[line][kx] = scale * F[line][kx] for the modes of one shell (its line runs)
template <typename T>
__global__ void shell_gather_kernel(const Cx<T>* __restrict__ F, const short4* __restrict__ lines, int lb, int le,
                                    int K, T scale, Cx<T>* __restrict__ H) {
    const int nk = 2 * K + 1;
    for (int li = lb + blockIdx.x * blockDim.y + threadIdx.y; li < le; li += gridDim.x * blockDim.y) {
        const short4 L = lines[li];
        const size_t base = ((size_t)(L.x + K) * (K + 1) + L.y) * nk + K;
        const int len = L.w - L.z + 1;            // kx in [a, b]
        const int an = L.z > 0 ? L.z : 1;
        const int len2 = L.w >= an ? L.w - an + 1 : 0;  // kx in [-b, -max(a, 1)]
        for (int t = threadIdx.x; t < len + len2; t += blockDim.x) {
            const int kx = t < len ? L.z + t : -(an + (t - len));
            const Cx<T> v = F[base + kx];
            H[base + kx] = cx<T>(v.re * scale, v.im * scale);
        }
    }
}

}  // namespace ps

using namespace ps;

// host -------------------------------------------------------------------------------
struct AtState;  // adjoint_tc.cu
poly_status ps_at_prepare(PsPlan* p, const std::vector<int>& ent_m, const std::vector<short4>& ent, AtState** out);
cudaError_t ps_at_contract(PsPlan* p, AtState* S, const float* w, cudaStream_t st);
int ps_at_error(AtState* S);
void ps_at_free(AtState* S);

struct AdjTables {
    int nent = 0;
    void* d_Wall = nullptr;      // batched forward transforms of the G_m: intermediates and spectra, or NULL
    void* d_fhat_all = nullptr;
    AtState* at = nullptr;  // tensor-core form of the per-cell contraction (bispectrum, split-BF16)
    void *d_moff = nullptr, *d_ent = nullptr, *d_eoff = nullptr, *d_ebins = nullptr, *d_w = nullptr;
    std::vector<int> line_off;  // host copy of the plan's line offsets
};

// The adjoint's entries: one per (m, sorted other shells) that some bin holds,
// grouped by m (moff), each listing its bins once per position of m in the bin
// (eoff / ebins).  Host only.
void ps_adj_entries(const PsPlan* p, std::vector<int>& moff, std::vector<short4>& ent, std::vector<int>& eoff,
                    std::vector<int>& ebins) {
    const int n = p->order;  // 2 .. 4
    // one record per (bin, position t of m in it): key (m, the other shells sorted, -1 padded), bin; sorted
    // stably by key, so each entry's bins keep the (bin, position) order they were produced in
    struct Rec {
        std::array<int, 4> key;
        int bin;
    };
    std::vector<Rec> recs;
    recs.reserve((size_t)p->nbins * n);
    for (int64_t b = 0; b < p->nbins; b++) {
        const int32_t* k = &p->bins[b * n];
        for (int t = 0; t < n; t++) {
            Rec r{{k[t] - 1, -1, -1, -1}, (int)b};
            int c = 1;
            for (int u = 0; u < n; u++)
                if (u != t) r.key[c++] = k[u] - 1;
            std::sort(r.key.begin() + 1, r.key.begin() + n);
            recs.push_back(r);
        }
    }
    std::stable_sort(recs.begin(), recs.end(), [](const Rec& x, const Rec& y) { return x.key < y.key; });
    moff.assign(p->nshell + 1, 0);
    eoff.assign(1, 0);
    ebins.clear();
    ent.clear();
    for (size_t i = 0; i < recs.size();) {  // key order: grouped by m ascending
        const std::array<int, 4>& key = recs[i].key;
        size_t j = i;
        while (j < recs.size() && recs[j].key == key) ebins.push_back(recs[j++].bin);
        moff[key[0] + 1]++;
        short4 f;
        f.x = (short)key[1];
        f.y = (short)key[2];
        f.z = (short)key[3];
        f.w = 0;
        ent.push_back(f);
        eoff.push_back((int)ebins.size());
        i = j;
    }
    for (int m = 0; m < p->nshell; m++) moff[m + 1] += moff[m];
}

static poly_status adj_prepare(PsPlan* p, AdjTables& A) {
    const int n = p->order;
    std::vector<int> moff, eoff, ebins;
    std::vector<short4> ent;
    ps_adj_entries(p, moff, ent, eoff, ebins);
    A.nent = (int)ent.size();
    if (n == 3 && p->prec == POLY_SPLIT_BF16) {
        std::vector<int> ent_m(ent.size());
        for (int m = 0; m < p->nshell; m++)
            for (int e = moff[m]; e < moff[m + 1]; e++) ent_m[e] = m;
        poly_status s = ps_at_prepare(p, ent_m, ent, &A.at);
        if (s && s != POLY_ERR_UNSUPPORTED) return s;  // unsupported: the CUDA-core kernel below serves
    }
    const size_t es = p->is_double ? 8 : 4;
    auto up = [&](void** d, const void* h, size_t bytes) -> poly_status {
        poly_status s = ps_alloc(p, d, bytes);
        if (s) return s;
        return cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice) ? POLY_ERR_CUDA : POLY_OK;
    };
    poly_status s;
    if ((s = up(&A.d_moff, moff.data(), moff.size() * 4)) || (s = up(&A.d_ent, ent.data(), ent.size() * 8)) ||
        (s = up(&A.d_eoff, eoff.data(), eoff.size() * 4)) ||
        (s = up(&A.d_ebins, ebins.data(), std::max<size_t>(1, ebins.size()) * 4)))
        return s;
    if ((s = ps_alloc(p, &A.d_w, std::max(1, A.nent) * es))) return s;
    A.line_off.resize(p->nshell + 2);
    if (cudaMemcpy(A.line_off.data(), p->d_line_off, (p->nshell + 2) * sizeof(int), cudaMemcpyDeviceToHost))
        return POLY_ERR_CUDA;
    const size_t n3 = (size_t)p->N * p->N * p->N;
    const size_t nl = (size_t)(2 * p->K + 1) * (p->K + 1) * (2 * p->K + 1);
    if ((s = ps_alloc(p, &p->d_G, (size_t)p->nshell * n3 * es))) return s;
    if ((s = ps_alloc(p, &p->d_ghat, nl * 2 * es))) return s;
    // the G_m's forward transforms in one batch when their planes fit shared memory (no spill buffer)
    if (ps_plane_needs_spill(p->N, p->K, p->is_double) == 0) {
        const size_t wsz = (size_t)p->N * (2 * p->K + 1) * (p->K + 1);
        if ((s = ps_alloc(p, &A.d_Wall, (size_t)p->nshell * wsz * 2 * es)) ||
            (s = ps_alloc(p, &A.d_fhat_all, (size_t)p->nshell * nl * 2 * es)))
            return s;
    }
    return POLY_OK;
}

poly_status ps_backward_impl(PsPlan* p, const void* delta, const double* dL_dB, void* dL_ddelta, cudaStream_t st) {
    if (p->order > 4 || p->ell != 0) {
        ps_set_last_error("poly_backward supports monopole plans of orders 2 to 4");
        return POLY_ERR_UNSUPPORTED;
    }
    if (!p->adj) {
        AdjTables* A = new (std::nothrow) AdjTables();
        if (!A) return POLY_ERR_ALLOC;
        poly_status s = adj_prepare(p, *A);
        if (s) {  // the tables' device buffers stay on the plan's list until it is destroyed
            ps_at_free(A->at);
            delete A;
            return s;
        }
        p->adj = A;
    }
    AdjTables& A = *p->adj;
    poly_status s = ps_fields(p, delta, st);
    if (s) return s;
    const int64_t ncell = (int64_t)p->N * p->N * p->N;
    const int dbl = p->is_double;
    cudaError_t e;
    const int wb = std::max(1, std::min(4096, (A.nent + 255) / 256));
    if (dbl)
        adj_weights_kernel<double><<<wb, 256, 0, st>>>(dL_dB, p->d_counts, (const int*)A.d_eoff, (const int*)A.d_ebins,
                                                       A.nent, (double*)A.d_w);
    else
        adj_weights_kernel<float><<<wb, 256, 0, st>>>(dL_dB, p->d_counts, (const int*)A.d_eoff, (const int*)A.d_ebins,
                                                      A.nent, (float*)A.d_w);
    const unsigned gblocks = (unsigned)((ncell + kAdjChunk - 1) / kAdjChunk);
    const size_t smem = (size_t)p->nshell * kAdjChunk * (dbl ? 8 : 4);
    if (A.at) {
        if ((e = ps_at_contract(p, A.at, (const float*)A.d_w, st))) return POLY_ERR_CUDA;
    } else if (dbl) {
        cudaFuncSetAttribute(adj_g_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        adj_g_kernel<double><<<gblocks, kAdjThreads, smem, st>>>((const double*)p->d_fields, p->nshell, ncell,
                                                                  (const int*)A.d_moff, (const short4*)A.d_ent,
                                                                  (const double*)A.d_w, (double*)p->d_G);
    } else {
        cudaFuncSetAttribute(adj_g_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        adj_g_kernel<float><<<gblocks, kAdjThreads, smem, st>>>((const float*)p->d_fields, p->nshell, ncell,
                                                                 (const int*)A.d_moff, (const short4*)A.d_ent,
                                                                 (const float*)A.d_w, (float*)p->d_G);
    }
    if ((e = cudaGetLastError())) return POLY_ERR_CUDA;
    p->launches += A.at ? 3 : 2;
    // H = c_n / N^3 * sum_m mask_m forward(G_m)
    const size_t nl = (size_t)(2 * p->K + 1) * (p->K + 1) * (2 * p->K + 1);
    const size_t es = dbl ? 8 : 4;
    if ((e = cudaMemsetAsync(p->d_ghat, 0, nl * 2 * es, st))) return POLY_ERR_CUDA;
    const double scale = ps_norm(p) / (double)ncell;
    // forward transforms of all G_m: one batched launch pair when the per-field outputs fit (A.d_Wall), else
    // one field at a time through the plan's workspace
    const size_t wsz = (size_t)p->N * (2 * p->K + 1) * (p->K + 1);
    const bool batched = A.d_Wall != nullptr;
    if (batched) {
        if ((e = ps_forward_batched(p->N, dbl, p->d_G, p->nshell, p->K, p->d_tw_fwd, A.d_Wall, A.d_fhat_all, nullptr,
                                    st)))
            return POLY_ERR_CUDA;
        p->launches += 2;
    }
    for (int m = 0; m < p->nshell; m++) {
        const void* Gm = (const char*)p->d_G + (size_t)m * ncell * es;
        const void* Fm = batched ? (const void*)((const char*)A.d_fhat_all + (size_t)m * nl * 2 * es) : p->d_fhat;
        if (!batched) {
            if ((e = ps_forward(p->N, dbl, Gm, p->K, p->d_tw_fwd, p->d_W, p->d_fhat, p->d_spill, st)))
                return POLY_ERR_CUDA;
            p->launches += 2;
        }
        const int lb = A.line_off[m], le = A.line_off[m + 1];
        if (le > lb) {
            dim3 blk(32, 8);
            const unsigned nb = (unsigned)std::min(1024, (le - lb + 7) / 8);
            if (dbl)
                shell_gather_kernel<double><<<nb, blk, 0, st>>>((const Cx<double>*)Fm, (const short4*)p->d_lines,
                                                               lb, le, p->K, scale, (Cx<double>*)p->d_ghat);
            else
                shell_gather_kernel<float><<<nb, blk, 0, st>>>((const Cx<float>*)Fm, (const short4*)p->d_lines,
                                                              lb, le, p->K, (float)scale, (Cx<float>*)p->d_ghat);
            if ((e = cudaGetLastError())) return POLY_ERR_CUDA;
        }
        p->launches += 1;
    }
    (void)wsz;
    // one inverse transform over the union of the shells
    if (!ps_xpre_fits(p, p->nshell, 1)) return POLY_ERR_ARG;
    if ((e = ps_inverse(p->N, dbl, 0, p->d_ghat, p->d_lines, p->d_line_off, p->nshell, 1, p->K, 0, p->N, p->d_tw_inv,
                        dL_ddelta, (size_t)ncell, p->d_spill, p->d_xpre, p->max_lines, 0, st)))
        return POLY_ERR_CUDA;
    p->launches += 2;
    return POLY_OK;
}

void ps_adj_free(PsPlan* p) {
    if (p->adj) ps_at_free(p->adj->at);
    delete p->adj;
    p->adj = nullptr;
}

int ps_adj_device_error(PsPlan* p) { return p->adj && p->adj->at ? ps_at_error(p->adj->at) : 0; }
