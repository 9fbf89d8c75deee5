// rgf_common.cuh -- number types and small helpers shared by the RGF kernels.
//
// Two arithmetic types carry the slice recursion:
//   double  -- IEEE binary64 (the RGF_FP64 path, FP64 pipe);
//   df32    -- "double-float": an unevaluated sum hi + lo of two binary32 values
//              (|lo| <= ulp(hi)/2 after normalisation, ~48-bit significand),
//              evaluated on the FP32 pipes (the RGF_MIXED path).
// The double-float operations below are the classical error-free
// transformations: Knuth's TwoSum, the FMA form of Dekker's TwoProduct and
// Dekker's Fast2Sum (T. J. Dekker, Numer. Math. 18 (1971) 224; D. E. Knuth,
// TAOCP vol. 2, 4.2.2).  They are written with explicit round-to-nearest
// intrinsics so that the compiler cannot contract or reorder them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifndef RGF_NT
#define RGF_NT 512
#endif

namespace rgf {

// Threads per block of the slice kernels (and warps).
constexpr int NT = RGF_NT;
constexpr int NWARP = NT / 32;

// ---------------------------------------------------------------------------
// double-float
// ---------------------------------------------------------------------------
struct df32 {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df32 df_from_double(double x) {
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return {h, l};
}
__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    df32 r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ df32 df_neg(df32 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df32 df_sub(df32 a, df32 b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    df32 r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// ---------------------------------------------------------------------------
// complex numbers over a real type R (double or df32)
// ---------------------------------------------------------------------------
template <class R> struct cx { R re, im; };
using zd = cx<double>;
using zf = cx<df32>;

// Conversions to / from binary64 complex.
__device__ __forceinline__ zd to_z(zd a) { return a; }
__device__ __forceinline__ zd to_z(zf a) { return {df_to_double(a.re), df_to_double(a.im)}; }
template <class R> __device__ __forceinline__ cx<R> from_z(double re, double im);
template <> __device__ __forceinline__ zd from_z<double>(double re, double im) { return {re, im}; }
template <> __device__ __forceinline__ zf from_z<df32>(double re, double im) {
    return {df_from_double(re), df_from_double(im)};
}
template <class R> __device__ __forceinline__ cx<R> czero() { return from_z<R>(0.0, 0.0); }

// a + b, a - b, a * b
__device__ __forceinline__ zd cadd(zd a, zd b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ zd csub(zd a, zd b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ zd cmul(zd a, zd b) {
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ zf cadd(zf a, zf b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ zf csub(zf a, zf b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ zf cmul(zf a, zf b) {
    return {df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)),
            df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}

// c + s * a * b with s = +1 or -1 (multiply-accumulate).
__device__ __forceinline__ zd cmac(zd c, zd a, zd b, bool neg) {
    double ar = neg ? -a.re : a.re, ai = neg ? -a.im : a.im;
    c.re = fma(ar, b.re, c.re);
    c.re = fma(-ai, b.im, c.re);
    c.im = fma(ar, b.im, c.im);
    c.im = fma(ai, b.re, c.im);
    return c;
}

// One real component of c + x1*y1 - x2*y2 in double-float, unnormalised
// result (hi, lo) with the product errors and cross terms folded into lo.
__device__ __forceinline__ df32 df_dot2(df32 c, df32 x1, df32 y1, df32 x2, df32 y2) {
    float p1 = __fmul_rn(x1.hi, y1.hi);
    float e1 = __fmaf_rn(x1.hi, y1.hi, -p1);
    float p2 = __fmul_rn(x2.hi, y2.hi);
    float e2 = __fmaf_rn(x2.hi, y2.hi, -p2);
    float x = __fmaf_rn(x1.hi, y1.lo, __fmaf_rn(x1.lo, y1.hi, e1));
    x = __fsub_rn(x, __fmaf_rn(x2.hi, y2.lo, __fmaf_rn(x2.lo, y2.hi, e2)));
    float s1, t1, s2, t2;
    two_sum(c.hi, p1, s1, t1);
    two_sum(s1, -p2, s2, t2);
    float lo = __fadd_rn(__fadd_rn(c.lo, x), __fadd_rn(t1, t2));
    df32 r;
    fast_two_sum(s2, lo, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ zf cmac(zf c, zf a, zf b, bool neg) {
    df32 ar = neg ? df_neg(a.re) : a.re, ai = neg ? df_neg(a.im) : a.im;
    zf r;
    r.re = df_dot2(c.re, ar, b.re, ai, b.im);      // c.re + ar*br - ai*bi
    r.im = df_dot2(c.im, ar, b.im, df_neg(ai), b.re);  // c.im + ar*bi + ai*br
    return r;
}

__device__ __forceinline__ zd cconj(zd a) { return {a.re, -a.im}; }
__device__ __forceinline__ zf cconj(zf a) { return {a.re, df_neg(a.im)}; }

// Scale by a real binary64 constant.
__device__ __forceinline__ zd cscale(zd a, double s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ zf cscale(zf a, double s) {
    df32 d = df_from_double(s);
    return {df_mul(a.re, d), df_mul(a.im, d)};
}
// Scale by a real constant already in double-float (no binary64 work).
__device__ __forceinline__ zf cscale(zf a, df32 d) { return {df_mul(a.re, d), df_mul(a.im, d)}; }

// 1/a in the working precision.  Binary64: conj(a) times one reciprocal of
// |a|^2.  Double-float:
// d = |a|^2 in double-float, 1/d from the binary32 reciprocal of d.hi refined by
// one Newton step r <- r + r (1 - d r) in double-float (doubles the ~24 correct
// bits), then conj(a) / d -- all on the FP32 pipes.
__device__ __forceinline__ zd crecip(zd a) {
    const double r = 1.0 / (a.re * a.re + a.im * a.im);
    return {a.re * r, -a.im * r};
}
__device__ __forceinline__ zf crecip(zf a) {
    const df32 d = df_add(df_mul(a.re, a.re), df_mul(a.im, a.im));
    const float r0 = __frcp_rn(d.hi);
    const df32 r0d = {r0, 0.0f};
    const df32 e = df_sub(df32{1.0f, 0.0f}, df_mul(d, r0d));   // 1 - d r0
    const df32 r = df_add(r0d, df_mul(r0d, e));
    return {df_mul(a.re, r), df_neg(df_mul(a.im, r))};
}

// |a|^2 as a binary64 estimate (pivot selection only).
__device__ __forceinline__ double cabs2(zd a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ double cabs2(zf a) {
    double r = a.re.hi, i = a.im.hi;
    return r * r + i * i;
}

// |a|^2 in binary32 (pivot search only; overflow to inf still orders correctly
// against finite values and the winner is rechecked in binary64).
__device__ __forceinline__ float cabs2f(zd a) {
    float r = (float)a.re, i = (float)a.im;
    return r * r + i * i;
}
__device__ __forceinline__ float cabs2f(zf a) { return a.re.hi * a.re.hi + a.im.hi * a.im.hi; }

__device__ __forceinline__ bool cfinite(zd a) { return isfinite(a.re) && isfinite(a.im); }
__device__ __forceinline__ bool cfinite(zf a) { return isfinite(a.re.hi) && isfinite(a.im.hi); }

// ---------------------------------------------------------------------------
// Status codes (mirror rgf_status in include/rgf.h).
// ---------------------------------------------------------------------------
enum : int {
    ST_OK = 0, ST_EINVAL = 1, ST_ENOMEM = 2, ST_ECUDA = 3, ST_ENOCONV = 4,
    ST_ESINGULAR = 5, ST_ENONFINITE = 6, ST_ETIMEOUT = 7, ST_EBOUNDS = 8
};

// Unit roundoff of the working precision (binary64: 2^-53; double-float: 2^-48).
template <class R> struct Unit;
template <> struct Unit<double> { static constexpr double u = 1.1102230246251565e-16; };
template <> struct Unit<df32> { static constexpr double u = 3.552713678800501e-15; };

// Number of propagating channels of a pristine armchair ribbon of N lines at
// energy E: modes p with |t| |1 + 2 c_p| <= |E| < |t| (1 + 2 |c_p|),
// c_p = cos(p pi / (N + 1)) (the band edges of the transverse modes).  A lower
// edge within 1e-12 |t| of |E| counts: the metallic mode of N = 3q + 2 has its
// edge at exactly 0 (a linear crossing that carries a channel at E = 0), which
// the rounding of c_p puts a few 1e-16 eV to either side.
__device__ __forceinline__ int channels(int N, double t, double E) {
    int n = 0;
    const double at = fabs(t), ae = fabs(E);
    for (int p = 1; p <= N; ++p) {
        double c = cospi((double)p / (double)(N + 1));
        if (at * fabs(1.0 + 2.0 * c) <= ae + 1e-12 * at && ae < at * (1.0 + 2.0 * fabs(c))) ++n;
    }
    return n;
}

}  // namespace rgf
