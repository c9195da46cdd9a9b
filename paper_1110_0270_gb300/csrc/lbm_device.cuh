// Device side of the GB300 lattice Boltzmann step: lattice tables, storage
// formats, equilibria, collisions and the fused A-A stream-and-collide kernel.
//
// Paper: Brownlee, Levesley, Packwood, Gorban, "Add-ons for Lattice Boltzmann
// Methods: Regularization, Filtering and Limiters".  Section numbers below
// refer to it.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_params.h"

namespace lbm {

// ---------------------------------------------------------------------------
// Lattices.  D1Q3 (Section 6): v = -1, 0, +1.  D2Q9 (Section 5 numbering,
// rest, E, then clockwise): 0 rest, 1 E, 2 SE, 3 S, 4 SW, 5 W, 6 NW, 7 N, 8 NE.
// ---------------------------------------------------------------------------
template <int Q> struct Lat;

template <> struct Lat<3> {
    static constexpr int Q = 3;
    static constexpr int rest = 1;
    __host__ __device__ static constexpr int cx(int i) { return i - 1; }
    __host__ __device__ static constexpr int cy(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) { return 2 - i; }
    __host__ __device__ static constexpr double w(int i) { return i == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }
};

template <> struct Lat<9> {
    static constexpr int Q = 9;
    static constexpr int rest = 0;
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 2 || i == 8) ? 1 : ((i == 4 || i == 5 || i == 6) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 6 || i == 7 || i == 8) ? 1 : ((i == 2 || i == 3 || i == 4) ? -1 : 0);
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i + 3) % 8) + 1; }
    __host__ __device__ static constexpr double w(int i) {
        return (cx(i) * cx(i) + cy(i) * cy(i)) == 0 ? 4.0 / 9.0
               : ((cx(i) * cx(i) + cy(i) * cy(i)) == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

// ---------------------------------------------------------------------------
// Storage formats.  T is the arithmetic type, S the stored type.  The 16-bit
// formats hold the deviation f_i - W_i (round to nearest even) so that the
// format's precision is spent on the part that varies.
// ---------------------------------------------------------------------------
// ld2 / st2 move the two consecutive elements p[0], p[1] (p 2-element
// aligned) with one vector access and, for the 16-bit formats, one packed
// conversion.
struct StF64 {
    using S = double;
    using T = double;
    static constexpr int code = LBM_FP64;
    __device__ static T ld(const S* p, T) { return *p; }
    __device__ static void st(S* p, T v, T) { *p = v; }
    __device__ static void ld2(const S* p, T, T& a, T& b) {
        const double2 v = *(const double2*)p;
        a = v.x;
        b = v.y;
    }
    __device__ static void st2(S* p, T a, T b, T) { *(double2*)p = make_double2(a, b); }
};
struct StF32 {
    using S = float;
    using T = float;
    static constexpr int code = LBM_FP32;
    __device__ static T ld(const S* p, T) { return *p; }
    __device__ static void st(S* p, T v, T) { *p = v; }
    __device__ static void ld2(const S* p, T, T& a, T& b) {
        const float2 v = *(const float2*)p;
        a = v.x;
        b = v.y;
    }
    __device__ static void st2(S* p, T a, T b, T) { *(float2*)p = make_float2(a, b); }
};
struct StBF16 {
    using S = __nv_bfloat16;
    using T = float;
    static constexpr int code = LBM_BF16_DEV;
    __device__ static T ld(const S* p, T w) { return w + __bfloat162float(*p); }
    __device__ static void st(S* p, T v, T w) { *p = __float2bfloat16_rn(v - w); }
    __device__ static void ld2(const S* p, T w, T& a, T& b) {
        const float2 v = __bfloat1622float2(*(const __nv_bfloat162*)p);
        a = w + v.x;
        b = w + v.y;
    }
    __device__ static void st2(S* p, T a, T b, T w) { *(__nv_bfloat162*)p = __floats2bfloat162_rn(a - w, b - w); }
    __device__ static T dec(S h) { return __bfloat162float(h); }  // a stored deviation
    __device__ static S enc(T v) { return __float2bfloat16_rn(v); }
    // a pair as one 32-bit word (element at the lower address in the low half)
    __device__ static float2 unpack(uint32_t u) {
        __nv_bfloat162 h;
        *reinterpret_cast<uint32_t*>(&h) = u;
        return __bfloat1622float2(h);
    }
    __device__ static uint32_t pack(float a, float b) {  // round to nearest even, as st2
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
};
struct StF16 {
    using S = __half;
    using T = float;
    static constexpr int code = LBM_FP16_DEV;
    __device__ static T ld(const S* p, T w) { return w + __half2float(*p); }
    __device__ static void st(S* p, T v, T w) { *p = __float2half_rn(v - w); }
    __device__ static void ld2(const S* p, T w, T& a, T& b) {
        const float2 v = __half22float2(*(const __half2*)p);
        a = w + v.x;
        b = w + v.y;
    }
    __device__ static void st2(S* p, T a, T b, T w) { *(__half2*)p = __floats2half2_rn(a - w, b - w); }
    __device__ static T dec(S h) { return __half2float(h); }
    __device__ static S enc(T v) { return __float2half_rn(v); }
    __device__ static float2 unpack(uint32_t u) {
        __half2 h;
        *reinterpret_cast<uint32_t*>(&h) = u;
        return __half22float2(h);
    }
    __device__ static uint32_t pack(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
};

// ---------------------------------------------------------------------------
// FP32 arithmetic on one site (float) or on two sites at once (F2: two FP32
// values in one 64-bit register pair, the packed add / sub / mul / fma
// .rn.f32x2 instructions of sm_100-class GPUs: one instruction, both sites).
// The one-site forms are the same correctly rounded operations (explicit
// _rn intrinsics, which the compiler neither contracts nor reorders), so a
// site computes to the same bits in either form.
// ---------------------------------------------------------------------------
struct F2 {
    uint64_t v;
};
template <class V> struct VLanes;
template <> struct VLanes<float> { static constexpr int n = 1; };
template <> struct VLanes<F2> { static constexpr int n = 2; };

__device__ __forceinline__ float vsplat(float a, float) { return a; }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vlane(float a, int) { return a; }
template <class V> __device__ __forceinline__ V vmake(float a, float b);
template <> __device__ __forceinline__ float vmake<float>(float a, float) { return a; }

template <> __device__ __forceinline__ F2 vmake<F2>(float a, float b) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ F2 vsplat(float a, F2) { return vmake<F2>(a, a); }
__device__ __forceinline__ float vlane(F2 a, int k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
    return k ? hi : lo;
}
__device__ __forceinline__ F2 vadd(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 vsub(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 vmul(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

// ---------------------------------------------------------------------------
// Equilibria.  1D polynomial and entropic equilibria of Section 6 per unit
// density (order -, 0, +); the D2Q9 quasi-equilibrium is their product
// (Section 8).  The textbook polynomial is an option.
// ---------------------------------------------------------------------------
// Both 1D equilibria have the form phi_-+ = a -+ u/2, phi_0 = 1 - 2a, with
// a = (1 + 3u^2)/6 (polynomial) or (2 sqrt(1 + 3u^2) - 1)/6 (entropic) -
// the printed formulas of Section 6 regrouped into even and odd parts.
// Written this way the zeroth and first moments are exact up to unbiased
// rounding: u/2 is exact in binary, and the rounded constants 1/6, 2/3 that
// the printed forms carry would otherwise bias sum f* (mass) and
// sum v f* (momentum) upwards by ~6e-8 per step in FP32, a steady drift.
template <class T>
__device__ __forceinline__ void eq1d_poly(T u, T& m, T& z, T& p) {
    const T a = (T(1) + T(3) * u * u) * (T(1) / T(6));
    const T h = T(0.5) * u;
    m = a - h;
    p = a + h;
    z = T(1) - T(2) * a;
}

template <class T>
__device__ __forceinline__ void eq1d_entropic(T u, T& m, T& z, T& p) {
    const T s = sqrt(T(1) + T(3) * u * u);
    const T a = (T(2) * s - T(1)) * (T(1) / T(6));
    const T h = T(0.5) * u;
    m = a - h;
    p = a + h;
    z = T(1) - T(2) * a;
}

template <int Q, class T>
__device__ __forceinline__ void equilibrium(int kind, T rho, T ux, T uy, T* feq) {
    using L = Lat<Q>;
    if (Q == 9 && kind == LBM_EQ_POLY_STD) {
        T uu = ux * ux + uy * uy, rest = rho;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            T cu = T(L::cx(i)) * ux + T(L::cy(i)) * uy;
            feq[i] = T(L::w(i)) * rho * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
            rest -= feq[i];
        }
        feq[0] = rest;  // = 4/9 rho (1 - 3/2 u^2); keeps sum f* = rho unbiased
        return;
    }
    T ax[3], ay[3];
    if (kind == LBM_EQ_ENTROPIC) {
        eq1d_entropic<T>(ux, ax[0], ax[1], ax[2]);
        if (Q == 9) eq1d_entropic<T>(uy, ay[0], ay[1], ay[2]);
    } else {
        eq1d_poly<T>(ux, ax[0], ax[1], ax[2]);
        if (Q == 9) eq1d_poly<T>(uy, ay[0], ay[1], ay[2]);
    }
    if (Q == 3) {
#pragma unroll
        for (int i = 0; i < Q; ++i) feq[i] = rho * ax[i];
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) feq[i] = rho * ax[L::cx(i) + 1] * ay[L::cy(i) + 1];
    }
}

template <int Q, class T>
__device__ __forceinline__ void moments(const T* f, T& rho, T& ux, T& uy) {
    using L = Lat<Q>;
    T r = T(0), jx = T(0), jy = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        r += f[i];
        if (L::cx(i) > 0) jx += f[i];
        if (L::cx(i) < 0) jx -= f[i];
        if (L::cy(i) > 0) jy += f[i];
        if (L::cy(i) < 0) jy -= f[i];
    }
    rho = r;
    T inv = T(1) / r;
    ux = jx * inv;
    uy = jy * inv;
}

// ---------------------------------------------------------------------------
// g(x) = (1+x) ln(1+x) - x, the per-population term of the nonequilibrium
// entropy Delta S = sum f*_i g((f_i - f*_i)/f*_i) (Eq. DelS with the zero sum
// sum (f* - f) added).  For |x| < 1/4 the Taylor series
// x^2 sum_k (-1)^k x^k / ((k+1)(k+2)) replaces the closed form, whose two
// terms cancel; the truncation is below one unit in the last place.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ double gseries_d(double x) {
    double p = ((K & 1) ? -1.0 : 1.0) / (double)((K + 1) * (K + 2));
#pragma unroll
    for (int k = K - 1; k >= 0; --k) p = fma(p, x, ((k & 1) ? -1.0 : 1.0) / (double)((k + 1) * (k + 2)));
    return x * x * p;
}

// The series length follows |x|: the first omitted term, relative to the
// leading x^2/2, is below 2^-56 (FP64) or 2^-26 (FP32) in every tier.
__device__ __forceinline__ double gfun_d(double x) {
    if (x <= -1.0) return 1.0;  // g(-1) = 1; below -1 only for negative populations
    const double ax = fabs(x);
    if (ax < 0.015625) return gseries_d<8>(x);
    if (ax < 0.125) return gseries_d<16>(x);
    if (ax < 0.25) return gseries_d<26>(x);
    return (1.0 + x) * log1p(x) - x;
}

// P(x) = sum_{k <= K} (-1)^k x^k / ((k+1)(k+2)), so that g(x) ~ x^2 P(x).
template <int K>
__device__ __forceinline__ float gpoly_f(float x) {
    float p = ((K & 1) ? -1.0f : 1.0f) / (float)((K + 1) * (K + 2));
#pragma unroll
    for (int k = K - 1; k >= 0; --k) p = fmaf(p, x, ((k & 1) ? -1.0f : 1.0f) / (float)((k + 1) * (k + 2)));
    return p;
}

template <int K>
__device__ __forceinline__ float gseries_f(float x) {
    return x * x * gpoly_f<K>(x);
}

__device__ __forceinline__ float gfun_f(float x) {
    if (x <= -1.0f) return 1.0f;
    const float ax = fabsf(x);
    if (ax < 0.03125f) return gseries_f<4>(x);
    if (ax < 0.25f) return gseries_f<11>(x);
    return (1.0f + x) * log1pf(x) - x;
}

template <class T> __device__ __forceinline__ T gfun(T x);
template <> __device__ __forceinline__ double gfun<double>(double x) { return gfun_d(x); }
template <> __device__ __forceinline__ float gfun<float>(float x) { return gfun_f(x); }

// Delta S in FP64 from populations f (any type, converted exactly).  The
// equilibrium is recomputed in FP64 from the FP64 moments of f.  A negative
// population gives +inf.
template <int Q, class T>
__device__ double delta_s_fp64(const T* f, int eqkind) {
    double fd[Q], feq[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fd[i] = (double)f[i];
    double rho, ux, uy;
    moments<Q, double>(fd, rho, ux, uy);
    equilibrium<Q, double>(eqkind, rho, ux, uy, feq);
    double s = 0.0;
    bool neg = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        neg |= (fd[i] < 0.0) || !(feq[i] > 0.0);
        s += feq[i] * gfun_d((fd[i] - feq[i]) / feq[i]);
    }
    return neg ? __longlong_as_double(0x7ff0000000000000ULL) : s;
}

// Delta S in the arithmetic type T from f and its equilibrium (FP32: the
// relative deviation by the approximate division, good to 2 ulp, which the
// FP32 field tolerates).
// x^k for x >= 0 in the limiter functions of Sections 4.2-4.3.  FP64: pow.
// FP32: the exponents 0, +-1/2, 1, 3/2 and 2 by sqrt, rsqrt and products,
// others as exp2(k log2 x) (a few units in the last place, well inside the
// FP32 parity bound) instead of powf's special-case handling; k is the same
// for every thread, so the branches do not diverge.
__device__ __forceinline__ double pow_lim(double x, double k) { return pow(x, k); }
__device__ __forceinline__ float pow_lim(float x, float k) {
    if (k == 1.f) return x;
    if (k == 0.5f) return sqrtf(x);
    if (k == 2.f) return x * x;
    if (k == 1.5f) return x * sqrtf(x);
    if (k == 0.f) return 1.f;
    if (k == -0.5f) return rsqrtf(x);
    return exp2f(k * log2f(x));
}

__device__ __forceinline__ double rel_dev(double d, double q) { return d / q; }
__device__ __forceinline__ float rel_dev(float d, float q) { return __fdividef(d, q); }

template <int Q, class T>
__device__ __forceinline__ T delta_s_t(const T* f, const T* feq) {
    T s = T(0);
    bool neg = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        neg |= (f[i] < T(0)) || !(feq[i] > T(0));
        s += feq[i] * gfun<T>(rel_dev(f[i] - feq[i], feq[i]));
    }
    return neg ? T(INFINITY) : s;
}

// Limiter screens (FP32, no FP64 instruction: GB300's FP64 rate is a small
// fraction of its FP32 rate).  Each returns true when the site may exceed
// delta and needs the exact FP64 Delta S.  With d = f - f*, x = d / f* and
// q = sum d^2 / f*, rounding f* and d to FP32 moves q by at most about
// 3e-7 sqrt(q rho) + 2e-6 q (|d| summed by Cauchy-Schwarz); the relative
// 1e-3 and absolute 1e-6 sqrt(q rho) slack covers it.
//
// v (1 + 1e-3) + 1e-6 sqrt(|q rho|) >= delta, without the square root: true
// when v alone reaches delta, else compares the squares (also true for NaN).
__device__ __forceinline__ bool slack_reaches(float v, float q, float rho, float delta) {
    const float t = delta - 1.001f * v;
    return !(t > 0.f) || 1e-12f * fabsf(q * rho) >= t * t;
}

// Ehrenfest: g(x) <= x^2 for |x| < 1/2, and with m = min_i f*_i > 0 and
// s2 = sum d^2, max |x| <= max |d| / m <= sqrt(s2) / m, so s2 < m^2 / 4 gives
// Delta S <= sum d^2 / f* <= s2 / m.  One approximate division per site and no
// per-population division; the looseness (up to ~30x near equilibrium) only
// lets more sites through to the exact test.  A negative population fails
// the first test (|d_i| > f*_i >= m).
template <int Q>
__device__ __forceinline__ bool maybe_above_loose(const float* f, const float* feq, float rho, float delta) {
    float s2 = 0.f, m = feq[0];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float d = f[i] - feq[i];
        s2 = fmaf(d, d, s2);
        m = fminf(m, feq[i]);
    }
    // quiet without the division: s2 < m min(m / 4, 0.998 delta) and
    // rho < 1e6 delta give Delta S <= s2 / m < 0.998 delta, the FP32
    // rounding inside the 0.2% margin (for rho < 4e7 delta)
    if (m > 0.f && s2 < m * fminf(0.25f * m, 0.998f * delta) && rho < 1e6f * delta) return false;
    if (!(m > 0.f) || !(s2 < 0.25f * m * m)) return true;  // also NaN
    const float q = __fdividef(s2, m);  // approximate (2 ulp), far inside the slack
    return slack_reaches(q, q, rho, delta);
}

// Median with a Delta S field (1 - 2 beta near 0): the
// site's Delta S in the arithmetic type is computed anyway (the filter's
// field), so it is the screen itself; it also serves the threshold limiter,
// the selection kernel's FP32 settling and the limiters of Sections 4.2-4.3
// (their phi).  In the form sum f* g(x) the
// rounding of the mass of f* cancels to first order (dDelta S / df*_i =
// -x_i), leaving sum x_i df*_i <= sqrt(q) sqrt(sum df*_i^2 / f*_i), inside the
// same slack; the series and log1p evaluation of g is accurate to ~1e-5
// relative.  +inf (a non-positive population) and NaN pass.
template <int Q, class T>
__device__ __forceinline__ T delta_s_and_q(const T* f, const T* feq, T& q);

// FP32: one series length per site, chosen by max |x| (the tiers of gfun_f),
// so the populations share one branch; f* g(x) = d x P(x) with
// g(x) = x^2 P(x).
template <>
__device__ __forceinline__ float delta_s_and_q<9, float>(const float* f, const float* feq, float& q) {
    float x[9], dx[9], amax = 0.f, emin = feq[0];
    q = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float d = f[i] - feq[i];
        x[i] = __fdividef(d, feq[i]);
        dx[i] = d * x[i];
        q += dx[i];
        amax = fmaxf(amax, fabsf(x[i]));
        emin = fminf(emin, feq[i]);
    }
    // with f* > 0, a negative population has x < -1: only the last tier sees one
    if (!(emin > 0.f)) return INFINITY;
    float s = 0.f;
    if (amax < 0x1p-12f) {  // fluid at rest or nearly: the omitted x^4/12 is below 2^-26 of x^2/2
#pragma unroll
        for (int i = 0; i < 9; ++i) s = fmaf(dx[i], gpoly_f<1>(x[i]), s);
    } else if (amax < 0.03125f) {
#pragma unroll
        for (int i = 0; i < 9; ++i) s = fmaf(dx[i], gpoly_f<4>(x[i]), s);
    } else if (amax < 0.25f) {
#pragma unroll
        for (int i = 0; i < 9; ++i) s = fmaf(dx[i], gpoly_f<11>(x[i]), s);
    } else {
        bool neg = false;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            neg |= f[i] < 0.f;
            s = fmaf(feq[i], gfun_f(x[i]), s);
        }
        if (neg) return INFINITY;
    }
    return s;
}

template <int Q, class T>
__device__ __forceinline__ T delta_s_and_q(const T* f, const T* feq, T& q) {
    T s = T(0);
    q = T(0);
    bool neg = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        neg |= (f[i] < T(0)) || !(feq[i] > T(0));
        const T d = f[i] - feq[i];
        const T x = rel_dev(d, feq[i]);
        s += feq[i] * gfun<T>(x);
        q += d * x;
    }
    return neg ? T(INFINITY) : s;
}

__device__ __forceinline__ bool median_maybe_above(float ds, float q, float rho, float delta) {
    return slack_reaches(ds, q, rho, delta);
}

// ---------------------------------------------------------------------------
// Collisions.
// ---------------------------------------------------------------------------

// Every collision and limiter here conserves mass exactly (Section 2), so the
// rest population of the post-collision state equals rho minus the others.
// Writing it that way leaves one unbiased rounding per site; computing it
// like the others lets the rounding of f* and of the update accumulate a
// steady mass drift in FP32 (about 2e-8 of rho per step).
template <int Q, class T>
__device__ __forceinline__ void conserve_mass(T rho, T* F) {
    using L = Lat<Q>;
    T s = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (i != L::rest) s += F[i];
    F[L::rest] = rho - s;
}

// Section 5's A_2 = M_2^-1 C_2 M_2 on D2Q9: with C_2 = 1 on every monomial
// moment except v_x^2 - v_y^2 and v_x v_y (rate s_nu = 2 beta), and M_2's
// rows for those two orthogonal to the others with squared norm 4,
// A_2 = I + (s_nu - 1)/4 (r4 r4^T + r5 r5^T), r4 = v_x^2 - v_y^2,
// r5 = v_x v_y per velocity, so F = f - A_2 (f - f*) =
// f* + (1 - s_nu)/4 (m4 r4 + m5 r5), m = r . (f - f*).
template <class T>
__device__ __forceinline__ void mrt2_d2q9(const T* f, const T* feq, T om, T* F) {
    using L = Lat<9>;
    T m4 = T(0), m5 = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const T d = f[i] - feq[i];
        const int r4 = L::cx(i) * L::cx(i) - L::cy(i) * L::cy(i), r5 = L::cx(i) * L::cy(i);
        if (r4 > 0) m4 += d;
        if (r4 < 0) m4 -= d;
        if (r5 > 0) m5 += d;
        if (r5 < 0) m5 -= d;
    }
    const T c = (T(1) - om) * T(0.25);
    m4 *= c;
    m5 *= c;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int r4 = L::cx(i) * L::cx(i) - L::cy(i) * L::cy(i), r5 = L::cx(i) * L::cy(i);
        F[i] = feq[i] + T(r4) * m4 + T(r5) * m5;
    }
}

// LBGK with over-relaxation, Eq. (CollisionIntegral) with alpha = 2.
template <int Q, class T>
__device__ __forceinline__ void lbgk(const T* f, const T* feq, T beta, T* F) {
    T om = T(2) * beta;
#pragma unroll
    for (int i = 0; i < Q; ++i) F[i] = f[i] - om * (f[i] - feq[i]);  // shares d = f - f* with the screens
}

// Positivity rule (Section 4, Eq. StrLine): a state with a negative
// component moves along the line through f* to the nearest nonnegative point.
template <int Q, class T>
__device__ __forceinline__ bool positivity(const T* feq, T* F) {
    T lam = T(1);
    bool hit = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (F[i] < T(0)) {
            T l = feq[i] / (feq[i] - F[i]);
            lam = l < lam ? l : lam;
            hit = true;
        }
    }
    if (hit) {
#pragma unroll
        for (int i = 0; i < Q; ++i) F[i] = feq[i] + lam * (F[i] - feq[i]);
    }
    return hit;
}

// MRT of Section 5 in moment space: with the orthogonal basis M1 (rows
// rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy; squared norms 9, 36, 36, 6, 12,
// 6, 12, 4, 4) the inverse is M1^T N^-1, so
// F = f - M1^T (C1 N^-1) M1 (f - f*).  The conserved rows contribute zero
// (f and f* share rho and rho u) and are skipped.  rate[k] = C1_k / N_k.
template <class T>
__device__ __forceinline__ void mrt_d2q9(const T* f, const T* feq, const MrtRates& rd,
                                         const MrtRatesF& rf, T* F) {
    // rates in T (FP32 copies avoid per-site FP64 conversions)
    struct {
        T e, eps, q, nu;
    } r = {sizeof(T) == 8 ? T(rd.e) : T(rf.e), sizeof(T) == 8 ? T(rd.eps) : T(rf.eps),
           sizeof(T) == 8 ? T(rd.q) : T(rf.q), sizeof(T) == 8 ? T(rd.nu) : T(rf.nu)};
    T d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = f[i] - feq[i];
    // rows of M1 in the paper numbering (rest, E, SE, S, SW, W, NW, N, NE)
    T se = d[2] + d[4] + d[6] + d[8];  // diagonals
    T ax = d[1] + d[3] + d[5] + d[7];  // axis
    T e = T(-4) * d[0] - ax + T(2) * se;
    T ep = T(4) * d[0] - T(2) * ax + se;
    T qx = T(-2) * d[1] + d[2] - d[4] + T(2) * d[5] - d[6] + d[8];
    T qy = -d[2] + T(2) * d[3] - d[4] + d[6] - T(2) * d[7] + d[8];
    T pxx = d[1] - d[3] + d[5] - d[7];
    T pxy = -d[2] + d[4] - d[6] + d[8];
    e *= r.e;
    ep *= r.eps;
    qx *= r.q;
    qy *= r.q;
    pxx *= r.nu;
    pxy *= r.nu;
    // F_i = f_i - sum_k M1[k][i] * m_k
    F[0] = f[0] - (T(-4) * e + T(4) * ep);
    F[1] = f[1] - (-e - T(2) * ep - T(2) * qx + pxx);
    F[2] = f[2] - (T(2) * e + ep + qx - qy - pxy);
    F[3] = f[3] - (-e - T(2) * ep + T(2) * qy - pxx);
    F[4] = f[4] - (T(2) * e + ep - qx - qy + pxy);
    F[5] = f[5] - (-e - T(2) * ep + T(2) * qx + pxx);
    F[6] = f[6] - (T(2) * e + ep - qx + qy - pxy);
    F[7] = f[7] - (-e - T(2) * ep - T(2) * qy - pxx);
    F[8] = f[8] - (T(2) * e + ep + qx + qy + pxy);
}

// ELBM (Section 3).  S_f(alpha) = S(f + alpha Delta) - S(f), Delta = f* - f,
// written without cancellation via the entropic equilibrium's identity
// S(y) = S(f*) - DeltaS(y): with d_i = Delta_i / f*_i and x_i = (alpha-1) d_i,
//   S_f = sum f*_i [g(-d_i) - g(x_i)],  S_f' = -sum Delta_i ln(1 + x_i),
//   S_f'' = -sum Delta_i^2 / (f_i + alpha Delta_i).
// g(x) and ln(1+x) from one Taylor series (one tier per evaluation, chosen
// from max |x| so that the lanes of a site stay together):
// ln(1+x) = x (1 + m(x)) with m(x) = sum_{k=1..K} (-1)^k x^k / (k+1), and
// g(x) = (1+x) ln(1+x) - x = x (x + (1+x) m(x)), which has no cancellation
// (x + (1+x) m = x/2 - x^2/6 + ...).  With K = max(KL, KG + 1) the first
// omitted term is below 2^-54 of the leading one for both (KG, KL: the
// lengths two separate series of g / x^2 and ln(1+x) / x would need).
template <int KG, int KL>
__device__ __forceinline__ void gl_series(double x, double& g, double& l) {
    constexpr int K = KL > KG + 1 ? KL : KG + 1;
    // m / x = sum_{j=0..K-1} (-1)^(j+1) x^j / (j+2)
    double p = ((K & 1) ? -1.0 : 1.0) / (double)(K + 1);
#pragma unroll
    for (int j = K - 2; j >= 0; --j) p = fma(p, x, ((j & 1) ? 1.0 : -1.0) / (double)(j + 2));
    const double m = x * p;
    l = fma(x, m, x);
    g = x * fma(m, 1.0 + x, x);
}

template <int Q, int KG, int KL>
__device__ __forceinline__ void elbm_sum(const double* feq, const double* D, const double* R,
                                         const double* gm, const float* Df, const float* gf, double a,
                                         double& s0, double& s1, float& s2) {
    double A = 0.0, B = 0.0;
    float C = 0.f;
    const float af = (float)a;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double x = (a - 1.0) * R[i];  // R = Delta / f*, once per site
        double g, l;
        if (KG > 0) {
            gl_series<KG, KL>(x, g, l);
        } else {
            const double xc = x < -1.0 ? -1.0 : x;
            l = log1p(xc);
            g = xc <= -1.0 ? 1.0 : (1.0 + xc) * l - xc;
        }
        A += feq[i] * (gm[i] - g);
        B -= D[i] * l;
        // S_f'' only shapes the parabola (S_f and S_f' decide the root and the
        // stopping test), so FP32 is enough for it
        C -= Df[i] * Df[i] / fmaxf(gf[i] + af * Df[i], 1e-37f);
    }
    s0 = A;
    s1 = B;
    s2 = C;
}

// S_f(alpha), S_f'(alpha) (FP64) and S_f''(alpha) (FP32) at one site.
template <int Q>
__device__ __forceinline__ void elbm_eval(const double* feq, const double* D, const double* R,
                                          const double* gm, const float* Df, const float* gf,
                                          double amax_d, double a, double& s0, double& s1,
                                          double& s2) {
    const double ax = fabs(a - 1.0) * amax_d;  // max |x_i| at this alpha
    float c;
    if (ax < 0x1p-20)
        elbm_sum<Q, 2, 2>(feq, D, R, gm, Df, gf, a, s0, s1, c);
    else if (ax < 0x1p-10)
        elbm_sum<Q, 5, 5>(feq, D, R, gm, Df, gf, a, s0, s1, c);
    else if (ax < 0.015625)
        elbm_sum<Q, 8, 9>(feq, D, R, gm, Df, gf, a, s0, s1, c);
    else if (ax < 0.125)
        elbm_sum<Q, 16, 18>(feq, D, R, gm, Df, gf, a, s0, s1, c);
    else if (ax < 0.25)
        elbm_sum<Q, 26, 27>(feq, D, R, gm, Df, gf, a, s0, s1, c);
    else
        elbm_sum<Q, 0, 0>(feq, D, R, gm, Df, gf, a, s0, s1, c);
    s2 = (double)c;
}

// FP32 evaluation of S_f, S_f', S_f'' (the same cancellation-free form),
// for the iterations that bring alpha near the root before the FP64 ones.
// Series tiers for FP32 (first omitted term below 2^-24 of the leading one).
template <int K>
__device__ __forceinline__ float lpoly_f(float x) {
    float p = ((K & 1) ? -1.0f : 1.0f) / (float)(K + 1);
#pragma unroll
    for (int k = K - 1; k >= 0; --k) p = fmaf(p, x, ((k & 1) ? -1.0f : 1.0f) / (float)(k + 1));
    return p;
}

template <int Q, int K>
__device__ __forceinline__ void elbm_sum_f(const float* fe, const float* Df, const float* Rf, const float* gmf,
                                           const float* gf, float a, float& s0, float& s1, float& s2) {
    float A = 0.f, B = 0.f, C = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float x = (a - 1.f) * Rf[i];
        float g, l;
        if (K > 0) {
            g = x * x * gpoly_f<K>(x);
            l = x * lpoly_f<K>(x);
        } else {
            const float xc = x < -1.f ? -1.f : x;
            l = log1pf(xc);
            g = xc <= -1.f ? 1.f : (1.f + xc) * l - xc;
        }
        A = fmaf(fe[i], gmf[i] - g, A);
        B = fmaf(-Df[i], l, B);
        C -= Df[i] * Df[i] / fmaxf(gf[i] + a * Df[i], 1e-37f);
    }
    s0 = A;
    s1 = B;
    s2 = C;
}

template <int Q>
__device__ __forceinline__ void elbm_eval_f(const float* fe, const float* Df, const float* Rf, const float* gmf,
                                            const float* gf, float amax_d, float a, float& s0, float& s1,
                                            float& s2) {
    const float ax = fabsf(a - 1.f) * amax_d;
    if (ax < 0.015625f)
        elbm_sum_f<Q, 4>(fe, Df, Rf, gmf, gf, a, s0, s1, s2);
    else if (ax < 0.25f)
        elbm_sum_f<Q, 11>(fe, Df, Rf, gmf, gf, a, s0, s1, s2);
    else
        elbm_sum_f<Q, 0>(fe, Df, Rf, gmf, gf, a, s0, s1, s2);
}

struct ElbmOut {
    double alpha;
    int code;   // 0 root, 1 near-equilibrium skip, 2 fallback
    int iters;
};

// The near-equilibrium skip decided in FP32 where that is certain.  With
// x_i = (f_i - f*_i) / f*_i, Delta S = sum f*_i g(x_i) and, for |x| <= 1/2,
// g(x) = (x^2 / 2)(1 - x/3 + x^2/6 - ...) <= (x^2 / 2)(1 + |x|), so
// Delta S <= (q / 2)(1 + max |x|) with q = sum (f*_i - f_i)^2 / f*_i.  q and
// max |x| formed in FP32 from the FP64 differences carry < 1e-6 relative
// error, inside the factor 1 + 1e-5.  A site this clears takes the LBGK step
// that the FP64 test would also give it; every other site goes to that test.
template <int Q>
__device__ __forceinline__ bool elbm_skip_certain(const double* f, const double* feq, const double* Dd,
                                                  double thr) {
    float q = 0.f, amax = 0.f;
    bool pos = true;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float D = (float)Dd[i];
        const float e = (float)feq[i];
        pos &= f[i] > 0.0 && e > 0.f;
        const float x = __fdividef(D, e);
        q = fmaf(D, x, q);
        amax = fmaxf(amax, fabsf(x));
    }
    return pos && amax <= 0.5f && 0.5f * q * (1.f + amax) * 1.00001f < (float)thr;
}

// Root finder of Section 3.3 (Dd = f* - f, formed by the caller): start at
// the LBGK value alpha = 2, step to the
// greater root of the local second-order Taylor parabola, stop when
// |S_f / S_f'| ||f* - f|| < eps (Eqs. Stopping, ConvergenceTwo), and take the
// double Newton step back if the estimate ended above the root.  The first
// steps run in FP32, the rest - and every decision - in FP64 (the reported
// iteration count is that of the FP64 steps).  Sites with
// Delta S < 1e-15 take the LBGK step (in FP32 or 16-bit storage: below
// 1e-15 + 2^-48 rho, the floor the storage rounding alone produces).  Where
// the paper is silent: iterates are
// kept inside the admissible bracket (1, alpha_max] by bisection; existence
// of a non-trivial root is decided by the sign of S_f(alpha_max); without a
// root the configured rule of Section 3.2 applies.
template <int Q>
__device__ ElbmOut elbm_alpha(const double* f, const double* feq, const double* Dd, double rho, const Params& p) {
    ElbmOut o;
    o.iters = 0;
    if (elbm_skip_certain<Q>(f, feq, Dd, 1e-15 + p.elbm_skip_rel * rho)) {
        o.alpha = 2.0;
        o.code = 1;
        return o;
    }
    double D[Q], R[Q], gm[Q];
    float Df[Q], gf[Q];
    double dS = 0.0, rneg = 0.0, dmax = 0.0;
    bool neg = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        D[i] = Dd[i];
        const double d = D[i] / feq[i];
        R[i] = d;
        dmax = fmax(dmax, fabs(d));
        gm[i] = gfun_d(-d);
        dS += feq[i] * gm[i];
        neg |= f[i] < 0.0;
        rneg = fmax(rneg, -d);
        Df[i] = (float)D[i];
        gf[i] = (float)f[i];
    }
    // alpha_max = min over Delta_i < 0 of -f_i / Delta_i = 1 - f*_i / Delta_i
    // (f = f* - Delta) = 1 + 1 / max(-Delta_i / f*_i): one division
    const double amax = rneg > 0.0 ? 1.0 + 1.0 / rneg : __longlong_as_double(0x7ff0000000000000ULL);
    if (!neg && dS < 1e-15 + p.elbm_skip_rel * rho) {
        o.alpha = 2.0;
        o.code = 1;
        return o;
    }
    double fb = p.elbm_fallback == LBM_FALLBACK_EHRENFEST ? 1.0 : amax;
    if (neg) {
        o.alpha = fb;
        o.code = 2;
        return o;
    }
    double nrm = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) nrm += p.elbm_norm == LBM_NORM_L1 ? fabs(D[i]) : D[i] * R[i];  // D^2 / f*
    if (p.elbm_norm != LBM_NORM_L1) nrm = sqrt(nrm);
    double lo = 1.0, hi = amax;
    double a = (2.0 < amax) ? 2.0 : 0.5 * (1.0 + amax);
    {
        // FP32 parabola iterations from the same start: they bring alpha to
        // about 1e-6 of the root (their S_f carries ~1e-6 of Delta S in
        // rounding), so that the FP64 iterations below - which decide the
        // root's existence, take the steps to the stopping test and the final
        // correction - start next to it and mostly need one step.  FP64
        // evaluations are the cost of this solve on GB300.
        float fe32[Q], R32[Q], gm32[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            fe32[i] = (float)feq[i];
            R32[i] = (float)R[i];
            gm32[i] = (float)gm[i];
        }
        const float amf = (float)amax, dmf = (float)dmax;
        float af = (float)a, lof = 1.f, hif = amf;
        for (int k = 0; k < 8; ++k) {
            float t0, t1, t2;
            elbm_eval_f<Q>(fe32, Df, R32, gm32, gf, dmf, af, t0, t1, t2);
            if (t0 > 0.f)
                lof = af;
            else
                hif = af;
            const float disc = t1 * t1 - 2.f * t0 * t2;
            float next = __int_as_float(0x7fc00000);
            if (disc >= 0.f) {
                const float q = -0.5f * (t1 + copysignf(sqrtf(disc), t1));
                next = af + fmaxf(q / (0.5f * t2), t0 / q);
            }
            if (!(next > lof && next < hif)) next = 0.5f * (lof + hif);
            const bool done = fabsf(next - af) <= 1e-6f * af;
            af = next;
            if (done) break;
        }
        const double ad = (double)af;
        if (ad > 1.0 && ad < amax) a = ad;
    }
    double s0, s1, s2;
    elbm_eval<Q>(feq, D, R, gm, Df, gf, dmax, a, s0, s1, s2);
    if (s0 > 0.0) {
        // S_f is concave in alpha, so it lies below its tangent at a: if the
        // tangent reaches zero before alpha_max, so does S_f (a root exists
        // in (a, alpha_max)); only otherwise is S_f(alpha_max) evaluated.
        const double at = a - s0 / s1;
        if (!(s1 < 0.0 && at < amax)) {
            double m0, m1, m2;
            elbm_eval<Q>(feq, D, R, gm, Df, gf, dmax, amax, m0, m1, m2);
            if (m0 > 0.0) {
                o.alpha = fb;
                o.code = 2;
                return o;
            }
        }
        lo = a;
    } else {
        hi = a;
    }
    int it = 0;
    while (it < p.elbm_max_iter) {
        if (fabs(s0 / s1) * nrm < p.elbm_eps) break;
        ++it;
        double disc = s1 * s1 - 2.0 * s0 * s2;
        double next = __longlong_as_double(0x7ff8000000000000ULL);
        if (disc >= 0.0) {
            // greater root of (s2/2) h^2 + s1 h + s0 = 0, cancellation-free
            double q = -0.5 * (s1 + copysign(sqrt(disc), s1));
            double r1 = q / (0.5 * s2);
            double r2 = s0 / q;
            next = a + fmax(r1, r2);
        }
        if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
        a = next;
        elbm_eval<Q>(feq, D, R, gm, Df, gf, dmax, a, s0, s1, s2);
        if (s0 > 0.0)
            lo = a;
        else
            hi = a;
    }
    if (s0 < 0.0) a = a - 2.0 * s0 / s1;
    o.alpha = a;
    o.code = 0;
    o.iters = it;
    return o;
}

// ---------------------------------------------------------------------------
// A-A addressing.  For each direction i a site owns one address R_i; it loads
// its pre-collision f_i from R_i and stores its post-collision F_opp(i) to
// R_i, so that every address is read and written by exactly one thread.
//   even step:  R_i = (slot i, site x): F_j lands in slot opp(j) unstreamed.
//   odd step:   R_i = (slot opp(i), x - v_i) when x - v_i is in the domain
//               (the F_i that site streamed towards x), else (slot i, x): a
//               link through a wall, whose population bounces back half-way,
//               picking up -6 W_j (v_j . u_wall) (j = opp(i)) on the lid.
// After an odd step the array is in natural layout again.
// ---------------------------------------------------------------------------
template <int Q, class T>
__device__ __forceinline__ int64_t aa_address(const Params& p, int x, int y, int i, bool odd,
                                              T& lidc) {
    using L = Lat<Q>;
    lidc = T(0);
    if (!odd) return (int64_t)i * p.plane + (int64_t)y * p.pitch + x;
    int sx = x - L::cx(i), sy = y - L::cy(i);
    if (p.periodic_x) sx = sx < 0 ? sx + p.nx : (sx >= p.nx ? sx - p.nx : sx);
    if (p.periodic_y) sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
    if (sx >= 0 && sx < p.nx && sy >= 0 && sy < p.ny)
        return (int64_t)L::opp(i) * p.plane + (int64_t)sy * p.pitch + sx;
    // the population that left x along j = opp(i) crossed the top wall
    if (y - L::cy(i) >= p.ny)
        lidc = T(6.0 * L::w(L::opp(i)) * L::cx(L::opp(i))) *
               (sizeof(T) == 8 ? T(p.lid_u) : T(p.lid_u_f));
    return (int64_t)i * p.plane + (int64_t)y * p.pitch + x;
}

// Interior sites (all neighbours in the domain, so no wall terms): the
// offsets are 32-bit (the library keeps Q * ny * pitch below 2^31) and every
// address is a kernel-uniform base plus the site offset o = y * pitch + x.
template <int Q, class ST, bool ODD>
__device__ __forceinline__ int interior_offset(const Params& p, int o, int i) {
    using L = Lat<Q>;
    return ODD ? L::opp(i) * p.plane32 + o - L::cy(i) * p.pitch - L::cx(i) : i * p.plane32 + o;
}

// DEV: move the stored deviation f_i - W_i itself (16-bit formats; the
// lid term is additive, so it applies to the deviation unchanged).
template <int Q, class ST, bool ODD, bool DEV = false>
__device__ __forceinline__ void load_interior(const Params& p, int o, typename ST::T* f) {
    using T = typename ST::T;
    using L = Lat<Q>;
    const typename ST::S* base = (const typename ST::S*)p.f;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        f[i] = ST::ld(base + interior_offset<Q, ST, ODD>(p, o, i), DEV ? T(0) : T(L::w(i)));
}

template <int Q, class ST, bool ODD, bool DEV = false>
__device__ __forceinline__ void store_interior(const Params& p, int o, const typename ST::T* F) {
    using T = typename ST::T;
    using L = Lat<Q>;
    typename ST::S* base = (typename ST::S*)p.f;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        ST::st(base + interior_offset<Q, ST, ODD>(p, o, i), F[L::opp(i)], DEV ? T(0) : T(L::w(i)));
}

// Boundary (or any) site: the general addressing with wrap-around and walls,
// one direction at a time so that no address array stays live.
// (W_i = W_opp(i), so the deviation formats need no slot bookkeeping.)
template <int Q, class ST, bool ODD, bool DEV = false>
__device__ __forceinline__ void load_general(const Params& p, int x, int y, typename ST::T* f) {
    using T = typename ST::T;
    using L = Lat<Q>;
    const typename ST::S* base = (const typename ST::S*)p.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T lidc;
        const int64_t r = aa_address<Q, T>(p, x, y, i, ODD, lidc);
        f[i] = ST::ld(base + r, DEV ? T(0) : T(L::w(i))) - lidc;
    }
}

template <int Q, class ST, bool ODD, bool DEV = false>
__device__ __forceinline__ void store_general(const Params& p, int x, int y,
                                              const typename ST::T* F) {
    using T = typename ST::T;
    using L = Lat<Q>;
    typename ST::S* base = (typename ST::S*)p.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T lidc;
        const int64_t r = aa_address<Q, T>(p, x, y, i, ODD, lidc);
        ST::st(base + r, F[L::opp(i)] - lidc, DEV ? T(0) : T(L::w(i)));
    }
}

}  // namespace lbm
