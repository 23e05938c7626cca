// Forward R2C transform pruned to the analysis cube, and the fused shell
// gather + C2R inverse transform that produces the shell fields
//   D_s(x) = sum_{q in S_s} F(q) e^{+2 pi i q.x / N}        (Eq. Bkfast, App. A)
// with F = dhat for the density and F = 1 for the counting fields iota_s (Eq. Vn).
//
// Spectrum layout ("line-major", kz >= 0 half of a real field's spectrum):
//   fhat[((ky + K) * (K + 1) + kz) * (2K + 1) + (kx + K)],  |kx|, |ky|, kz <= K,
// where K is the largest integer wavevector component inside the outermost shell.
// Real fields are [x][y][z] with z fastest.
#pragma once
#include <algorithm>
#include <cstdio>

#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"

namespace ps {

constexpr int kPlaneThreads = 256;
constexpr int kPlaneWarps = kPlaneThreads / 32;
constexpr int kXLines = 32;  // lines per block in the x pass

template <typename T>
PS_DEV void load_twiddles(Cx<T>* s_tw, const Cx<double>* g_tw, int n) {
    for (int m = threadIdx.x; m < n; m += blockDim.x) s_tw[m] = cx<T>((T)g_tw[m].re, (T)g_tw[m].im);
}

// ------------------------------------------------------------------------
// forward, step 1: per x plane, R2C along z (rows in pairs), keep kz <= K,
// then DFT along y, keep |ky| <= K:  W[x][(ky+K)(K+1) + kz]
// ------------------------------------------------------------------------
template <typename T>
struct RowPairReader {  // Z(z) = delta(x, y1, z) + i delta(x, y2, z)
    const T* plane;
    int y0, ny;
    int n;
    PS_DEV Cx<T> read(int l, int pos) const {
        int y1 = y0 + 2 * l, y2 = y1 + 1;
        T a = plane[(size_t)y1 * n + pos];
        T b = y2 < ny ? plane[(size_t)y2 * n + pos] : (T)0;
        return cx<T>(a, b);
    }
};

template <typename T, int N, bool SPILL>
__global__ void __launch_bounds__(kPlaneThreads) fwd_plane_kernel(const T* __restrict__ delta, int K,
                                                                  const Cx<double>* __restrict__ g_tw,
                                                                  Cx<T>* __restrict__ W, Cx<T>* __restrict__ spill) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ls = line_stride<T>(N);
    constexpr int LPW = fft_lpw(N);
    Cx<T>* s_tw = reinterpret_cast<Cx<T>*>(smem_raw);
    Cx<T>* s_z = s_tw + N;                              // per-warp row buffers
    Cx<T>* s_t = s_z + (size_t)kPlaneWarps * LPW * ls;  // (K+1) lines of ls
    const int x = blockIdx.x;
    // blockIdx.y: the field of a batch (fields N^3 apart, their W outputs N (2K+1)(K+1) apart)
    delta += (size_t)blockIdx.y * N * N * N;
    W += (size_t)blockIdx.y * N * (2 * K + 1) * (K + 1);
    Cx<T>* Tb = SPILL ? spill + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (K + 1) * ls : s_t;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    load_twiddles(s_tw, g_tw, N);
    __syncthreads();

    const T* plane = delta + (size_t)x * N * N;
    SmemLines<T> zb{s_z + (size_t)warp * LPW * ls, ls};
    const int npairs = (N + 1) / 2;
    for (int p0 = warp * LPW; p0 < npairs; p0 += kPlaneWarps * LPW) {
        const int nl = min(LPW, npairs - p0);
        RowPairReader<T> rd{plane, 2 * p0, N, N};
        warp_fft<T, N, -1>(zb, nl, s_tw, lane, rd, zb);
        // separate the two real rows: X1 = (Z(k) + conj Z(-k))/2, X2 = (Z(k) - conj Z(-k))/(2i)
        for (int e = lane; e < nl * (K + 1); e += 32) {
            const int l = e / (K + 1), kz = e - (e / (K + 1)) * (K + 1);
            Cx<T> zk = zb.read(l, kz), zm = zb.read(l, (N - kz) % N);
            const int y1 = 2 * (p0 + l), y2 = y1 + 1;
            Tb[(size_t)kz * ls + pad_idx<T>(y1)] = cx<T>((T)0.5 * (zk.re + zm.re), (T)0.5 * (zk.im - zm.im));
            if (y2 < N)
                Tb[(size_t)kz * ls + pad_idx<T>(y2)] = cx<T>((T)0.5 * (zk.im + zm.im), (T)-0.5 * (zk.re - zm.re));
        }
        __syncwarp();
    }
    __syncthreads();
    // DFT along y of the K+1 kz columns
    for (int g = warp * LPW; g <= K; g += kPlaneWarps * LPW) {
        SmemLines<T> tb{Tb + (size_t)g * ls, ls};
        warp_fft_inplace<T, N, -1>(tb, min(LPW, K + 1 - g), s_tw, lane);
    }
    __syncthreads();
    const int nl = (2 * K + 1) * (K + 1);
    Cx<T>* Wx = W + (size_t)x * nl;
    for (int e = threadIdx.x; e < nl; e += blockDim.x) {
        const int kyi = e / (K + 1), kz = e - kyi * (K + 1);
        const int ky = kyi - K;
        Wx[e] = Tb[(size_t)kz * ls + pad_idx<T>((ky + N) % N)];
    }
}

// ------------------------------------------------------------------------
// forward, step 2: DFT along x of each (ky, kz) line, keep |kx| <= K
// ------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(kPlaneThreads) fwd_xlines_kernel(const Cx<T>* __restrict__ W, int K,
                                                                   const Cx<double>* __restrict__ g_tw,
                                                                   Cx<T>* __restrict__ fhat) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ls = line_stride<T>(N);
    constexpr int LPW = fft_lpw(N);
    Cx<T>* s_tw = reinterpret_cast<Cx<T>*>(smem_raw);
    Cx<T>* s_x = s_tw + N;
    const int nl = (2 * K + 1) * (K + 1);
    const int l0 = blockIdx.x * kXLines;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // blockIdx.y: the field of a batch
    W += (size_t)blockIdx.y * N * nl;
    fhat += (size_t)blockIdx.y * nl * (2 * K + 1);
    load_twiddles(s_tw, g_tw, N);
    for (int e = threadIdx.x; e < N * kXLines; e += blockDim.x) {
        const int x = e / kXLines, l = e - (e / kXLines) * kXLines;
        s_x[(size_t)l * ls + pad_idx<T>(x)] = (l0 + l < nl) ? W[(size_t)x * nl + l0 + l] : cx<T>(0, 0);
    }
    __syncthreads();
    const int nk = 2 * K + 1;
    for (int g = warp * LPW; g < kXLines; g += kPlaneWarps * LPW) {
        SmemLines<T> xb{s_x + (size_t)g * ls, ls};
        const int cnt = min(LPW, kXLines - g);
        warp_fft_inplace<T, N, -1>(xb, cnt, s_tw, lane);
        for (int e = lane; e < cnt * nk; e += 32) {
            const int l = e / nk, kxi = e - (e / nk) * nk;
            if (l0 + g + l < nl) fhat[(size_t)(l0 + g + l) * nk + kxi] = xb.read(l, (kxi - K + N) % N);
        }
    }
}

// ------------------------------------------------------------------------
// inverse, x pass: for every (shell, line) the masked 1-D inverse transform
// along x, T[s][x][l] = sum_{kx in the line's runs} F(kx, ky, kz) e^{+2 pi i kx x / N},
// stored so that a plane's lines are contiguous: T[line_off[s] * N + x * nl_s + l].
// 32 lines per block.  A warp takes one line at a time and its lanes 32
// consecutive x, so every lane of the warp runs the same kx loop; results pass
// through a [32 x][32 lines] shared tile so that the stores stay coalesced.
template <typename T, int N>
__global__ void __launch_bounds__(256) xpass_kernel(const Cx<T>* __restrict__ fhat, const short4* __restrict__ lines,
                                                    const int* __restrict__ line_off, int s0, int K,
                                                    const Cx<double>* __restrict__ g_tw, Cx<T>* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T>* s_tw = reinterpret_cast<Cx<T>*>(smem_raw);
    const int nk = 2 * K + 1;
    Cx<T>* s_f = s_tw + N;         // [32][nk]: the block's lines, kx in [-K, K]
    Cx<T>* s_o = s_f + 32 * nk;    // [32 x][33]
    short4* s_l = reinterpret_cast<short4*>(s_o + 32 * 33);
    const int s = s0 + blockIdx.y;
    const int lb = line_off[s], nls = line_off[s + 1] - lb;
    const int l0 = blockIdx.x * 32;
    if (l0 >= nls) return;
    const int nl = min(32, nls - l0);
    load_twiddles(s_tw, g_tw, N);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < nl) s_l[threadIdx.x] = lines[lb + l0 + threadIdx.x];
    // stage the run entries of the block's lines (one warp per line)
    for (int l = warp; l < nl; l += 8) {
        const short4 L = lines[lb + l0 + l];
        const Cx<T>* Fl = fhat + ((size_t)(L.x + K) * (K + 1) + L.y) * nk + K;
        const int an = L.z > 0 ? L.z : 1;
        for (int kx = L.z + lane; kx <= L.w; kx += 32) s_f[l * nk + K + kx] = Fl[kx];
        for (int kx = an + lane; kx <= L.w; kx += 32) s_f[l * nk + K - kx] = Fl[-kx];
    }
    __syncthreads();
    Cx<T>* o = out + (size_t)lb * N + l0;
    for (int x0 = 0; x0 < N; x0 += 32) {
        const int x = x0 + lane;
        for (int l = warp; l < nl; l += 8) {
            const short4 L = s_l[l];
            const int a = L.z, b = L.w, an = a > 0 ? a : 1;
            const Cx<T>* f = s_f + l * nk + K;
            T sr = 0, si = 0;
            if (x < N) {
                int m = (a * x) % N;
                for (int kx = a; kx <= b; kx++) {
                    const Cx<T> w = s_tw[m], v = f[kx];
                    sr += v.re * w.re - v.im * w.im;
                    si += v.re * w.im + v.im * w.re;
                    m += x;
                    if (m >= N) m -= N;
                }
                m = ((N - an) * x) % N;  // -an x mod N
                for (int kx = an; kx <= b; kx++) {
                    const Cx<T> w = s_tw[m], v = f[-kx];
                    sr += v.re * w.re - v.im * w.im;
                    si += v.re * w.im + v.im * w.re;
                    m -= x;
                    if (m < 0) m += N;
                }
            }
            s_o[lane * 33 + l] = cx<T>(sr, si);
        }
        __syncthreads();
        for (int xi = warp; xi < 32 && x0 + xi < N; xi += 8)
            if (lane < nl) o[(size_t)(x0 + xi) * nls + lane] = s_o[xi * 33 + lane];
        __syncthreads();
    }
}

template <typename T, int N>
static size_t xpass_smem_n(int K) {
    return ((size_t)N + 32 * (size_t)(2 * K + 1) + 32 * 33) * sizeof(Cx<T>) + 32 * sizeof(short4);
}

// ------------------------------------------------------------------------
// inverse: per (shell, x plane): gather the shell's modes along x,
//   G(ky, kz) = sum_{kx in shell} F(kx, ky, kz) e^{+2 pi i kx x / N},
// DFT along y, then the real transform along z from the kz >= 0 half,
//   D(x, y, z) = Re sum_{kz >= 0} w(kz) H(y, kz) e^{2 pi i kz z / N},  w(0)=1, w(>0)=2,
// done two rows at a time as one complex transform of the Hermitian-extended rows.
// ------------------------------------------------------------------------
template <typename T>
struct HalfPairReader {  // Z(kz) built from rows y1, y2 of Hb (kz lines)
    const Cx<T>* Hb;
    int ls, K, n, y0;
    PS_DEV Cx<T> read(int l, int pos) const {
        const int y1 = y0 + 2 * l, y2 = y1 + 1;
        const bool has2 = y2 < n;
        if (pos == 0) {
            Cx<T> h1 = Hb[pad_idx<T>(y1)];
            Cx<T> h2 = has2 ? Hb[pad_idx<T>(y2)] : cx<T>(0, 0);
            return cx<T>(h1.re, h2.re);
        }
        if (pos <= K) {
            Cx<T> h1 = Hb[(size_t)pos * ls + pad_idx<T>(y1)];
            Cx<T> h2 = has2 ? Hb[(size_t)pos * ls + pad_idx<T>(y2)] : cx<T>(0, 0);
            return cx<T>(h1.re - h2.im, h1.im + h2.re);
        }
        if (pos >= n - K) {
            const int kz = n - pos;
            Cx<T> h1 = Hb[(size_t)kz * ls + pad_idx<T>(y1)];
            Cx<T> h2 = has2 ? Hb[(size_t)kz * ls + pad_idx<T>(y2)] : cx<T>(0, 0);
            return cx<T>(h1.re + h2.im, h2.re - h1.im);
        }
        return cx<T>(0, 0);
    }
};

// Output layout of the shell fields: natural [s][x][y][z] (tile_ns == 0), or
// cell-tiled [cell / 32][s][cell % 32] over tile_ns shells, so that one 32-cell
// chunk of every shell is one contiguous block (what the contractions stream).
template <typename T, int N>
struct RowPairWriter {  // final stage: real part -> row y1, imaginary part -> row y2
    T* plane;       // natural layout: this plane's first cell
    T* base;        // tiled layout: the whole field array
    int y0, n, x, s, tile_ns;
    PS_DEV size_t at(int y, int z) const {
        const size_t cell = ((size_t)x * n + y) * n + z;
        return (cell >> 5) * (size_t)tile_ns * 32 + (size_t)s * 32 + (cell & 31);
    }
    PS_DEV void write(int l, int pos, Cx<T> v) const {
        const int y1 = y0 + 2 * l, y2 = y1 + 1;
        if (tile_ns > 0) {
            if constexpr (N % 32 == 0) {
                // a row starts a 32-cell block: cell (y, pos) lies in block row(y) + pos / 32 at pos % 32,
                // and row y + 1 starts N / 32 blocks later
                const size_t blk = (((size_t)x * N + y1) * N) >> 5;
                T* r = base + blk * (size_t)tile_ns * 32 + (size_t)s * 32 + (size_t)(pos >> 5) * tile_ns * 32 + (pos & 31);
                r[0] = v.re;
                if (y2 < N) r[(size_t)(N / 32) * tile_ns * 32] = v.im;
            } else {
                base[at(y1, pos)] = v.re;
                if (y2 < n) base[at(y2, pos)] = v.im;
            }
        } else {
            plane[(size_t)y1 * n + pos] = v.re;
            if (y2 < n) plane[(size_t)y2 * n + pos] = v.im;
        }
    }
};

// plane_s0: the shell whose plane x = x0 starts at `out` in the natural layout.
// MINB: blocks per SM the registers must allow (2 for the 8-warp small-shell launches).
template <typename T, int N, bool SPILL, bool UNITY, bool XPRE, int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) inv_plane_kernel(
    const Cx<T>* __restrict__ fhat, const short4* __restrict__ lines, const int* __restrict__ line_off, int s0,
    int K, int x0, const Cx<double>* __restrict__ g_tw, T* __restrict__ out, size_t out_shell_stride,
    Cx<T>* __restrict__ spill, const Cx<T>* __restrict__ xpre, int tile_ns, int plane_s0,
    const int* __restrict__ shell_kz) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ls = line_stride<T>(N);
    constexpr int LPW = fft_lpw(N);
    Cx<T>* s_tw = reinterpret_cast<Cx<T>*>(smem_raw);
    Cx<T>* s_z = s_tw + N;
    Cx<T>* s_h = s_z + (size_t)WARPS * LPW * ls;
    const int x = x0 + blockIdx.x;
    const int s = s0 + blockIdx.y;
    Cx<T>* Hb = SPILL ? spill + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (size_t)(K + 1) * ls : s_h;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int s_kzmax;
    const int lb = line_off[s], le = line_off[s + 1];
    // the shell's largest kz: kz lines above it stay zero through the y pass and are skipped
    // (from the plan's per-shell table when given, else from the shell's lines)
    if (threadIdx.x == 0) s_kzmax = shell_kz ? shell_kz[s] : 0;
    load_twiddles(s_tw, g_tw, N);
    __syncthreads();
    if (!shell_kz) {
        int kzm = 0;
        for (int li = lb + threadIdx.x; li < le; li += blockDim.x) kzm = max(kzm, (int)lines[li].y);
        if (kzm > 0) atomicMax(&s_kzmax, kzm);
        __syncthreads();
    }
    const int Ks = s_kzmax;
    for (int e = threadIdx.x; e < (Ks + 1) * ls; e += blockDim.x) Hb[e] = cx<T>(0, 0);
    __syncthreads();

    if (XPRE) {
        // the x pass already transformed each line: scatter this plane's values (four lines per
        // thread in flight: all loads first, then the stores)
        const Cx<T>* Tx = xpre + (size_t)lb * N + (size_t)x * (le - lb);
        const int nl = le - lb;
        for (int l0 = threadIdx.x; l0 < nl; l0 += 4 * blockDim.x) {
            short4 L[4];
            Cx<T> v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int li = l0 + u * blockDim.x;
                if (li < nl) {
                    L[u] = lines[lb + li];
                    v[u] = Tx[li];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (l0 + u * blockDim.x < nl) Hb[(size_t)L[u].y * ls + pad_idx<T>((L[u].x + N) % N)] = v[u];
        }
    }
    // gather along x
    const int nk = 2 * K + 1;
    for (int li = lb + threadIdx.x; !XPRE && li < le; li += blockDim.x) {
        const short4 L = lines[li];
        const int ky = L.x, kz = L.y, a = L.z, b = L.w;
        const Cx<T>* Fl = fhat + ((size_t)(ky + K) * (K + 1) + kz) * nk + K;
        T sr = 0, si = 0;
        // kx in [a, b] and kx in [-b, -max(a, 1)]
        int m = (int)(((long long)a * x) % N);
        for (int kx = a; kx <= b; kx++) {
            const Cx<T> w = s_tw[m];
            if (UNITY) {
                sr += w.re;
                si += w.im;
            } else {
                const Cx<T> f = Fl[kx];
                sr += f.re * w.re - f.im * w.im;
                si += f.re * w.im + f.im * w.re;
            }
            m += x;
            if (m >= N) m -= N;
        }
        const int an = a > 0 ? a : 1;  // the negative run, kx in [-b, -max(a, 1)]
        if (b >= an) {
            m = (int)(((long long)(N - an) * x) % N);  // -an * x mod N
            for (int kx = -an; kx >= -b; kx--) {
                const Cx<T> w = s_tw[m];
                if (UNITY) {
                    sr += w.re;
                    si += w.im;
                } else {
                    const Cx<T> f = Fl[kx];
                    sr += f.re * w.re - f.im * w.im;
                    si += f.re * w.im + f.im * w.re;
                }
                m -= x;
                if (m < 0) m += N;
            }
        }
        Hb[(size_t)kz * ls + pad_idx<T>((ky + N) % N)] = cx<T>(sr, si);
    }
    __syncthreads();
    // DFT along y of the Ks + 1 kz lines
    for (int g = warp * LPW; g <= Ks; g += WARPS * LPW) {
        SmemLines<T> hb{Hb + (size_t)g * ls, ls};
        warp_fft_inplace<T, N, +1>(hb, min(LPW, Ks + 1 - g), s_tw, lane);
    }
    __syncthreads();
    // real transform along z, two rows per complex line, written straight to global
    T* plane = out + (size_t)(s - plane_s0) * out_shell_stride + (size_t)blockIdx.x * N * N;
    SmemLines<T> zb{s_z + (size_t)warp * LPW * ls, ls};
    const int npairs = (N + 1) / 2;
    for (int p0 = warp * LPW; p0 < npairs; p0 += WARPS * LPW) {
        const int nl = min(LPW, npairs - p0);
        HalfPairReader<T> rd{Hb, ls, Ks, N, 2 * p0};
        RowPairWriter<T, N> wr{plane, out, 2 * p0, N, x, s, tile_ns};
        warp_fft<T, N, +1>(zb, nl, s_tw, lane, rd, wr);
    }
}

// ------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------
template <typename T, int N>
static size_t plane_smem_n(int K, bool spill, int warps = kPlaneWarps) {
    const int ls = line_stride<T>(N);
    size_t e = N + (size_t)warps * fft_lpw(N) * ls + (spill ? 0 : (size_t)(K + 1) * ls);
    return e * sizeof(Cx<T>);
}

template <typename T, int N>
static size_t xlines_smem_n() {
    return ((size_t)N + (size_t)kXLines * line_stride<T>(N)) * sizeof(Cx<T>);
}

constexpr size_t kMaxSmem = 227 * 1024;

// nfields fields N^3 apart -> W and fhat of each, (N (2K+1)(K+1)) and ((2K+1)(K+1)(2K+1)) apart; the spill
// buffer (when the plane does not fit shared memory) holds nfields * N blocks
template <typename T, int N>
static cudaError_t forward_n(const T* delta, int K, const Cx<double>* tw_fwd, Cx<T>* W, Cx<T>* fhat, Cx<T>* spill,
                             cudaStream_t st, int nfields = 1) {
    bool spill_on = plane_smem_n<T, N>(K, false) > kMaxSmem;
    if (spill_on && !spill) return cudaErrorInvalidValue;
    size_t sm = plane_smem_n<T, N>(K, spill_on);
    cudaError_t e;
    if (spill_on) {
        auto k = fwd_plane_kernel<T, N, true>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
        k<<<dim3(N, nfields), kPlaneThreads, sm, st>>>(delta, K, tw_fwd, W, spill);
    } else {
        auto k = fwd_plane_kernel<T, N, false>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
        k<<<dim3(N, nfields), kPlaneThreads, sm, st>>>(delta, K, tw_fwd, W, nullptr);
    }
    if ((e = cudaGetLastError())) return e;
    const int nl = (2 * K + 1) * (K + 1);
    size_t smx = xlines_smem_n<T, N>();
    auto kx = fwd_xlines_kernel<T, N>;
    if ((e = cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx))) return e;
    kx<<<dim3((nl + kXLines - 1) / kXLines, nfields), kPlaneThreads, smx, st>>>(W, K, tw_fwd, fhat);
    return cudaGetLastError();
}

template <typename T, int N, bool UNITY>
static cudaError_t inverse_n(const Cx<T>* fhat, const short4* lines, const int* line_off, int s0, int ns, int K,
                             int x0, int nx, const Cx<double>* tw_inv, T* out, size_t out_stride, Cx<T>* spill,
                             Cx<T>* xpre, int max_lines, int tile_ns, cudaStream_t st) {
    bool spill_on = plane_smem_n<T, N>(K, false) > kMaxSmem;
    if (spill_on && !spill) return cudaErrorInvalidValue;
    size_t sm = plane_smem_n<T, N>(K, spill_on);
    dim3 grid(nx, ns);
    cudaError_t e;
    const bool pre = !UNITY && xpre != nullptr;
    if (pre) {
        const size_t smx = xpass_smem_n<T, N>(K);
        auto kx = xpass_kernel<T, N>;
        if ((e = cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx))) return e;
        kx<<<dim3((max_lines + 31) / 32, ns), 256, smx, st>>>(fhat, lines, line_off, s0, K, tw_inv, xpre);
        if ((e = cudaGetLastError())) return e;
    }
#define PS_LAUNCH_INV(SP, PRE, W)                                                                                \
    {                                                                                                             \
        auto k = inv_plane_kernel<T, N, SP, UNITY, PRE, W, 1>;                                                    \
        const size_t smw = plane_smem_n<T, N>(K, SP, W);                                                          \
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw))) return e;       \
        k<<<grid, W * 32, smw, st>>>(fhat, lines, line_off, s0, K, x0, tw_inv, out, out_stride,                   \
                                     SP ? spill : nullptr, xpre, tile_ns, s0, nullptr);                           \
    }
    // 16 warps per block for FP32 when the plane still fits in shared memory (latency hiding), else 8
    const bool wide = sizeof(T) == 4 && !spill_on && plane_smem_n<T, N>(K, false, 16) <= kMaxSmem;
    if (spill_on) {
        if (pre) PS_LAUNCH_INV(true, true, 8) else PS_LAUNCH_INV(true, false, 8)
    } else if (wide) {
        if constexpr (sizeof(T) == 4) {
            if (pre) PS_LAUNCH_INV(false, true, 16) else PS_LAUNCH_INV(false, false, 16)
        }
    } else {
        if (pre) PS_LAUNCH_INV(false, true, 8) else PS_LAUNCH_INV(false, false, 8)
    }
#undef PS_LAUNCH_INV
    return cudaGetLastError();
}

// The inverse for the estimate path (FP32, natural or tiled output, x pass in
// front) in runs of consecutive shells, each launched with the shared memory
// its own largest kz needs: shells whose plane buffer fits twice per SM run as
// 8-warp blocks, two per SM, so that one block's transform phases overlap the
// other's; the rest run as one 16-warp block per SM.  kz_host[s] is shell s's
// largest kz (host array), kz_dev the same table on the device (or NULL).
template <typename T, int N>
static cudaError_t inverse_ranged_n(const Cx<T>* fhat, const short4* lines, const int* line_off, int s0, int ns, int K,
                                    const Cx<double>* tw_inv, T* out, size_t out_stride, Cx<T>* xpre, int max_lines,
                                    int tile_ns, const int* kz_host, const int* kz_dev, cudaStream_t st) {
    if (plane_smem_n<T, N>(K, false, 16) > kMaxSmem || !xpre)
        return inverse_n<T, N, false>(fhat, lines, line_off, s0, ns, K, 0, N, tw_inv, out, out_stride, nullptr, xpre,
                                      max_lines, tile_ns, st);
    cudaError_t e;
    const size_t smx = xpass_smem_n<T, N>(K);
    auto kx = xpass_kernel<T, N>;
    if ((e = cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx))) return e;
    kx<<<dim3((max_lines + 31) / 32, ns), 256, smx, st>>>(fhat, lines, line_off, s0, K, tw_inv, xpre);
    if ((e = cudaGetLastError())) return e;
    // largest kz whose 8-warp block fits twice per SM (228 KB per SM, 1 KB reserved per block)
    constexpr size_t kHalfSm = 228 * 1024 / 2 - 1024;
    int ksmall = -1;
    while (ksmall < K && plane_smem_n<T, N>(ksmall + 1, false, 8) <= kHalfSm) ksmall++;
    for (int r0 = s0; r0 < s0 + ns;) {
        const bool small = kz_host[r0] <= ksmall;
        int r1 = r0 + 1, kzm = kz_host[r0];
        while (r1 < s0 + ns && (kz_host[r1] <= ksmall) == small) kzm = std::max(kzm, kz_host[r1++]);
        const dim3 grid(N, r1 - r0);
        if (small) {
            auto k = inv_plane_kernel<T, N, false, false, true, 8, 2>;
            const size_t sm = plane_smem_n<T, N>(kzm, false, 8);
            if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
            k<<<grid, 8 * 32, sm, st>>>(fhat, lines, line_off, r0, K, 0, tw_inv, out, out_stride, nullptr, xpre, tile_ns,
                                        s0, kz_dev);
        } else {
            auto k = inv_plane_kernel<T, N, false, false, true, 16, 1>;
            const size_t sm = plane_smem_n<T, N>(kzm, false, 16);
            if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
            k<<<grid, 16 * 32, sm, st>>>(fhat, lines, line_off, r0, K, 0, tw_inv, out, out_stride, nullptr, xpre,
                                         tile_ns, s0, kz_dev);
        }
        if ((e = cudaGetLastError())) return e;
        r0 = r1;
    }
    return cudaSuccess;
}

}  // namespace ps
