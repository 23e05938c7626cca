// Warp-level mixed-radix Stockham FFT over lines held in (padded) shared memory.
//
// A line of length N is transformed in place, X[k] = sum_j x[j] e^{SIGN 2 pi i jk/N}
// (unnormalised).  Radices are 16 first, then 8, 4, 2, 3, 5; stage s with radix R
// and Ns = product of earlier radices maps butterfly j (0 <= j < N/R):
//   v[r] = x[j + r N/R] * W_{Ns R}^{SIGN (j mod Ns) r},  V = DFT_R(v),
//   y[(j / Ns) Ns R + (j mod Ns) + r Ns] = V[r].
// One warp owns LPW lines at a time, so only __syncwarp is needed between the
// read and write halves of a stage.  The first stage can read through a
// functor and the last stage can write through a functor (e.g. straight to
// global memory, coalesced, or from a half-spectrum built on the fly).
#pragma once
#include "common.cuh"

namespace ps {

// ---- radix plan (compile time) --------------------------------------------
__host__ __device__ constexpr int fft_nstages(int n) {
    int s = 0;
    while (n % 16 == 0) { n /= 16; s++; }
    for (int r : {8, 4, 2, 3, 5})
        while (n % r == 0) { n /= r; s++; }
    return n == 1 ? s : -1;
}
__host__ __device__ constexpr int fft_radix(int n, int stage) {
    int s = 0;
    while (n % 16 == 0) {
        if (s == stage) return 16;
        n /= 16;
        s++;
    }
    for (int r : {8, 4, 2, 3, 5})
        while (n % r == 0) {
            if (s == stage) return r;
            n /= r;
            s++;
        }
    return 1;
}
__host__ __device__ constexpr int fft_ns(int n, int stage) {  // product of radices before `stage`
    int p = 1;
    for (int s = 0; s < stage; s++) p *= fft_radix(n, s);
    return p;
}
// lines per warp: enough butterflies in the first stage to occupy the lanes
__host__ __device__ constexpr int fft_lpw(int n) {
    int b = n / fft_radix(n, 0);
    int l = 32 / b;
    return l < 1 ? 1 : l;
}

// ---- small DFTs in registers (sign SIGN) ---------------------------------
template <typename T, int SIGN>
PS_DEV void dft2(Cx<T>* v) {
    Cx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <typename T, int SIGN>
PS_DEV void dft4(Cx<T>& x0, Cx<T>& x1, Cx<T>& x2, Cx<T>& x3) {
    Cx<T> t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = cmul_si<SIGN>(csub(x1, x3));
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

template <typename T, int SIGN>
PS_DEV void dft3(Cx<T>* v) {
    const T h = (T)0.86602540378443864676;  // sin(2 pi / 3)
    Cx<T> a = v[0], t = cadd(v[1], v[2]);
    Cx<T> u = cscale(cmul_si<SIGN>(csub(v[1], v[2])), h);
    Cx<T> m = cx<T>(a.re - (T)0.5 * t.re, a.im - (T)0.5 * t.im);
    v[0] = cadd(a, t);
    v[1] = cadd(m, u);
    v[2] = csub(m, u);
}

template <typename T, int SIGN>
PS_DEV void dft5(Cx<T>* v) {
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;   // sin(2pi/5), sin(4pi/5)
    Cx<T> x0 = v[0];
    Cx<T> t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]), t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    Cx<T> a1 = cx<T>(x0.re + c1 * t1.re + c2 * t2.re, x0.im + c1 * t1.im + c2 * t2.im);
    Cx<T> a2 = cx<T>(x0.re + c2 * t1.re + c1 * t2.re, x0.im + c2 * t1.im + c1 * t2.im);
    Cx<T> b1 = cmul_si<SIGN>(cx<T>(s1 * t3.re + s2 * t4.re, s1 * t3.im + s2 * t4.im));
    Cx<T> b2 = cmul_si<SIGN>(cx<T>(s2 * t3.re - s1 * t4.re, s2 * t3.im - s1 * t4.im));
    v[0] = cx<T>(x0.re + t1.re + t2.re, x0.im + t1.im + t2.im);
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}

template <typename T, int SIGN>
PS_DEV void dft8(Cx<T>* v) {
    const T r = (T)0.70710678118654752440;  // cos(pi/4)
    Cx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    Cx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<T, SIGN>(e0, e1, e2, e3);
    dft4<T, SIGN>(o0, o1, o2, o3);
    // w^k, w = e^{SIGN 2 pi i / 8}
    Cx<T> w1 = cx<T>(r, (T)SIGN * r), w3 = cx<T>(-r, (T)SIGN * r);
    o1 = cmul(o1, w1);
    o2 = cmul_si<SIGN>(o2);
    o3 = cmul(o3, w3);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

template <typename T, int SIGN>
PS_DEV void dft16(Cx<T>* v) {
    // 16 = 4 x 4: inner DFT4 over n1 (stride 4), twiddle W16^{n2 k1}, outer DFT4 over n2.
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;  // cos, sin(pi/8)
    const T r = (T)0.70710678118654752440;
#pragma unroll
    for (int n2 = 0; n2 < 4; n2++) dft4<T, SIGN>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    // now v[4*k1 + n2] holds Y[n2][k1]; multiply by W16^{n2 k1}
    const Cx<T> w[10] = {cx<T>(1, 0),
                         cx<T>(c1, (T)SIGN * s1),
                         cx<T>(r, (T)SIGN * r),
                         cx<T>(s1, (T)SIGN * c1),
                         cx<T>(0, (T)SIGN),
                         cx<T>(-s1, (T)SIGN * c1),
                         cx<T>(-r, (T)SIGN * r),
                         cx<T>(-c1, (T)SIGN * s1),
                         cx<T>(-1, 0),
                         cx<T>(-c1, -(T)SIGN * s1)};
#pragma unroll
    for (int k1 = 1; k1 < 4; k1++)
#pragma unroll
        for (int n2 = 1; n2 < 4; n2++) v[4 * k1 + n2] = cmul(v[4 * k1 + n2], w[k1 * n2]);
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) dft4<T, SIGN>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // v[4*k1 + k2] holds X[k1 + 4 k2]; transpose to natural order
    Cx<T> t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++)
#pragma unroll
        for (int k2 = 0; k2 < 4; k2++) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = t[i];
}

template <typename T, int R, int SIGN>
PS_DEV void dft(Cx<T>* v) {
    if constexpr (R == 2) dft2<T, SIGN>(v);
    else if constexpr (R == 3) dft3<T, SIGN>(v);
    else if constexpr (R == 4) dft4<T, SIGN>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 5) dft5<T, SIGN>(v);
    else if constexpr (R == 8) dft8<T, SIGN>(v);
    else if constexpr (R == 16) dft16<T, SIGN>(v);
}

// ---- default readers / writers -------------------------------------------
template <typename T>
struct SmemLines {
    Cx<T>* base;
    int ls;
    PS_DEV Cx<T> read(int l, int pos) const { return base[l * ls + pad_idx<T>(pos)]; }
    PS_DEV void write(int l, int pos, Cx<T> v) const { base[l * ls + pad_idx<T>(pos)] = v; }
};

// ---- one Stockham stage ----------------------------------------------------
template <typename T, int N, int STAGE, int SIGN, int LPW, class Reader, class Writer>
PS_DEV void fft_stage(const SmemLines<T>& buf, int nl, const Cx<T>* tw, int lane, const Reader& rd,
                      const Writer& wr) {
    constexpr int NST = fft_nstages(N);
    constexpr int R = fft_radix(N, STAGE);
    constexpr int NS = fft_ns(N, STAGE);
    constexpr int B = N / R;
    constexpr int TOT = LPW * B;
    constexpr int CNT = (TOT + 31) / 32;
    Cx<T> v[CNT][R];
#pragma unroll
    for (int c = 0; c < CNT; c++) {
        const int t = lane + 32 * c;
        const int l = t / B, j = t - (t / B) * B;
        if (t < TOT && l < nl) {
#pragma unroll
            for (int r = 0; r < R; r++) {
                if constexpr (STAGE == 0) v[c][r] = rd.read(l, j + r * B);
                else v[c][r] = buf.read(l, j + r * B);
            }
            if constexpr (NS > 1) {
                const int k = j % NS;
#pragma unroll
                for (int r = 1; r < R; r++) v[c][r] = cmul(v[c][r], tw[(k * r) * (N / (NS * R))]);
            }
            dft<T, R, SIGN>(v[c]);
        }
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < CNT; c++) {
        const int t = lane + 32 * c;
        const int l = t / B, j = t - (t / B) * B;
        if (t < TOT && l < nl) {
            const int k = j % NS;
            const int o = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; r++) {
                if constexpr (STAGE == NST - 1) wr.write(l, o + r * NS, v[c][r]);
                else buf.write(l, o + r * NS, v[c][r]);
            }
        }
    }
    __syncwarp();
}

template <typename T, int N, int STAGE, int SIGN, int LPW, class Reader, class Writer>
PS_DEV void fft_stages(const SmemLines<T>& buf, int nl, const Cx<T>* tw, int lane, const Reader& rd,
                       const Writer& wr) {
    if constexpr (STAGE < fft_nstages(N)) {
        fft_stage<T, N, STAGE, SIGN, LPW>(buf, nl, tw, lane, rd, wr);
        fft_stages<T, N, STAGE + 1, SIGN, LPW>(buf, nl, tw, lane, rd, wr);
    }
}

// Transform nl <= fft_lpw(N) lines whose intermediate storage is `buf`
// (line l at buf.base + l * buf.ls).  tw[m] = e^{SIGN 2 pi i m / N}.
template <typename T, int N, int SIGN, class Reader, class Writer>
PS_DEV void warp_fft(const SmemLines<T>& buf, int nl, const Cx<T>* tw, int lane, const Reader& rd,
                     const Writer& wr) {
    static_assert(fft_nstages(N) > 0, "unsupported FFT length");
    fft_stages<T, N, 0, SIGN, fft_lpw(N)>(buf, nl, tw, lane, rd, wr);
}

template <typename T, int N, int SIGN>
PS_DEV void warp_fft_inplace(const SmemLines<T>& buf, int nl, const Cx<T>* tw, int lane) {
    warp_fft<T, N, SIGN>(buf, nl, tw, lane, buf, buf);
}

}  // namespace ps
