// Shared device/host helpers for the polyspectrum library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#define PS_DEV __device__ __forceinline__
#define PS_HD __host__ __device__ __forceinline__

namespace ps {

// Complex number stored as two consecutive reals (8 B for float, 16 B for double).
template <typename T>
struct alignas(2 * sizeof(T)) Cx {
    T re, im;
};

template <typename T>
PS_HD Cx<T> cx(T r, T i) {
    Cx<T> c;
    c.re = r;
    c.im = i;
    return c;
}
// Sums and differences of single-precision complex numbers take one packed FP32 pair
// instruction on sm_100 and later (each part rounded to nearest, as the scalar form;
// a - b as fma(-1, b, a), exact before its one rounding).
template <typename T>
PS_HD Cx<T> cadd(Cx<T> a, Cx<T> b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    if constexpr (std::is_same_v<T, float>) {
        const float2 r = __fadd2_rn(make_float2(a.re, a.im), make_float2(b.re, b.im));
        return cx<float>(r.x, r.y);
    }
#endif
    return cx<T>(a.re + b.re, a.im + b.im);
}
template <typename T>
PS_HD Cx<T> csub(Cx<T> a, Cx<T> b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    if constexpr (std::is_same_v<T, float>) {
        const float2 r = __ffma2_rn(make_float2(-1.f, -1.f), make_float2(b.re, b.im), make_float2(a.re, a.im));
        return cx<float>(r.x, r.y);
    }
#endif
    return cx<T>(a.re - b.re, a.im - b.im);
}
template <typename T>
PS_HD Cx<T> cmul(Cx<T> a, Cx<T> b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    if constexpr (std::is_same_v<T, float>) {  // (a.re b.re - a.im b.im, a.re b.im + a.im b.re) in two pair operations
        const float2 t = __fmul2_rn(make_float2(a.im, a.im), make_float2(-b.im, b.re));
        const float2 r = __ffma2_rn(make_float2(a.re, a.re), make_float2(b.re, b.im), t);
        return cx<float>(r.x, r.y);
    }
#endif
    return cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
PS_HD Cx<T> cconj(Cx<T> a) { return cx<T>(a.re, -a.im); }
template <typename T>
PS_HD Cx<T> cscale(Cx<T> a, T s) { return cx<T>(a.re * s, a.im * s); }
// a * (sign * i)
template <int SIGN, typename T>
PS_HD Cx<T> cmul_si(Cx<T> a) { return SIGN > 0 ? cx<T>(-a.im, a.re) : cx<T>(a.im, -a.re); }

// Shared-memory index padded with one element per 128 bytes, so that the
// Stockham write pattern (stride = radix) and strided column reads spread
// over the 32 banks.
template <typename T>
PS_HD int pad_idx(int i) { return i + i / (int)(128 / (2 * sizeof(T))); }

// Stride between lines of length n in padded shared memory.  Chosen so that
// reading element `pos` of consecutive lines (a column) is bank-conflict
// free: stride == 1 (mod 16) complex floats, == 1 (mod 8) complex doubles.
template <typename T>
PS_HD int line_stride(int n) {
    const int m = (int)(128 / (2 * sizeof(T)));
    int s = pad_idx<T>(n);
    while (s % m != 1) s++;
    return s;
}

// Supported grid sizes: the FFT plans below are instantiated for these.
#define PS_FOR_EACH_N(X) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(160) X(256)

}  // namespace ps
