// Shared device/host helpers of libggf: a small complex type, scalar traits
// over the four storage types (double, float, complex double, complex float),
// the Philox4x64-10 counter generator, error plumbing.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define GGF_HD __host__ __device__ __forceinline__

template <class R>
struct cx {
    R x, y;
};

template <class R> GGF_HD cx<R> mkc(R a, R b) { return cx<R>{a, b}; }
template <class R> GGF_HD cx<R> operator+(cx<R> a, cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <class R> GGF_HD cx<R> operator-(cx<R> a, cx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <class R> GGF_HD cx<R> operator-(cx<R> a) { return {-a.x, -a.y}; }
template <class R> GGF_HD cx<R> operator*(cx<R> a, cx<R> b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <class R> GGF_HD cx<R> operator*(R s, cx<R> a) { return {s * a.x, s * a.y}; }
template <class R> GGF_HD cx<R> operator*(cx<R> a, R s) { return {s * a.x, s * a.y}; }
template <class R> GGF_HD cx<R> conjg(cx<R> a) { return {a.x, -a.y}; }
template <class R> GGF_HD R abs2(cx<R> a) { return a.x * a.x + a.y * a.y; }
template <class R> GGF_HD cx<R> operator/(cx<R> a, cx<R> b) {
    // scaled division (Smith's method) to avoid overflow
    if (fabs(b.x) >= fabs(b.y)) {
        R t = b.y / b.x, d = b.x + b.y * t;
        return {(a.x + a.y * t) / d, (a.y - a.x * t) / d};
    }
    R t = b.x / b.y, d = b.y + b.x * t;
    return {(a.x * t + a.y) / d, (a.y * t - a.x) / d};
}
template <class R> GGF_HD cx<R>& operator+=(cx<R>& a, cx<R> b) { a.x += b.x; a.y += b.y; return a; }
template <class R> GGF_HD cx<R>& operator-=(cx<R>& a, cx<R> b) { a.x -= b.x; a.y -= b.y; return a; }

typedef cx<double> cxd;
typedef cx<float> cxf;

GGF_HD double cabs_(cxd a) { return hypot(a.x, a.y); }
GGF_HD cxd cexp_(cxd a) {
    double m = exp(a.x);
    double s, c;
#ifdef __CUDA_ARCH__
    sincos(a.y, &s, &c);
#else
    s = sin(a.y); c = cos(a.y);
#endif
    return {m * c, m * s};
}
GGF_HD cxd clog_(cxd a) { return {log(cabs_(a)), atan2(a.y, a.x)}; }

// ---- scalar traits ---------------------------------------------------------
template <class T> struct Sc;
template <> struct Sc<double> {
    typedef double R;
    static constexpr bool CPLX = false;
    GGF_HD static cxd to(double v) { return {v, 0.0}; }
    GGF_HD static double from(cxd v) { return v.x; }
    GGF_HD static double mag(double v) { return fabs(v); }
    GGF_HD static double zero() { return 0.0; }
    GGF_HD static double one() { return 1.0; }
};
template <> struct Sc<float> {
    typedef float R;
    static constexpr bool CPLX = false;
    GGF_HD static cxd to(float v) { return {(double)v, 0.0}; }
    GGF_HD static float from(cxd v) { return (float)v.x; }
    GGF_HD static float mag(float v) { return fabsf(v); }
    GGF_HD static float zero() { return 0.0f; }
    GGF_HD static float one() { return 1.0f; }
};
template <> struct Sc<cxd> {
    typedef double R;
    static constexpr bool CPLX = true;
    GGF_HD static cxd to(cxd v) { return v; }
    GGF_HD static cxd from(cxd v) { return v; }
    GGF_HD static double mag(cxd v) { return fabs(v.x) + fabs(v.y); }
    GGF_HD static cxd zero() { return {0.0, 0.0}; }
    GGF_HD static cxd one() { return {1.0, 0.0}; }
};
template <> struct Sc<cxf> {
    typedef float R;
    static constexpr bool CPLX = true;
    GGF_HD static cxd to(cxf v) { return {(double)v.x, (double)v.y}; }
    GGF_HD static cxf from(cxd v) { return {(float)v.x, (float)v.y}; }
    GGF_HD static float mag(cxf v) { return fabsf(v.x) + fabsf(v.y); }
    GGF_HD static cxf zero() { return {0.0f, 0.0f}; }
    GGF_HD static cxf one() { return {1.0f, 0.0f}; }
};

// real scalar arithmetic helpers so templates can use one spelling
GGF_HD double operator_mul(double a, double b) { return a * b; }
GGF_HD double conjg(double a) { return a; }
GGF_HD float conjg(float a) { return a; }

// ---- Philox4x64-10 (Salmon et al., SC'11) -----------------------------------
// Round: (c0, c1, c2, c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
// lo(M0 c0)); keys bumped by the Weyl constants after every round.
GGF_HD void mul128(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
#ifdef __CUDA_ARCH__
    *hi = __umul64hi(a, b);
    *lo = a * b;
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
#endif
}

GGF_HD void philox4x64_10(const uint64_t ctr[4], uint64_t k0, uint64_t k1, uint64_t out[4]) {
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mul128(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
        mul128(0xCA5A826395121157ULL, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

GGF_HD double u53(uint64_t w) { return (double)(w >> 11) * (1.0 / 9007199254740992.0); }

#define GGF_TWO_PI 6.283185307179586

// Delayed-update panels (U and V^T planes, N rows x KRM rank columns) are
// stored chunk-major: element (row, q) at ((q / 8) NP + row) 8 + q % 8, with
// NP = N rounded up to a multiple of 256 rows and the rank rounded up to a
// multiple of 8, so that the 8 rank columns of a block of consecutive rows
// (what one tensor-core stage reads) are one contiguous run.
GGF_HD int panel_rows(int N) { return (N + 255) & ~255; }
GGF_HD int panel_cols(int KRM) { return (KRM + 7) & ~7; }
GGF_HD size_t panel_plane(int N, int KRM) { return (size_t)panel_rows(N) * panel_cols(KRM); }
GGF_HD size_t pidx(int row, int q, int NP) { return ((size_t)(q >> 3) * NP + row) * 8 + (q & 7); }
