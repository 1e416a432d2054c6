// raptor_df64.cuh -- double-float ("df64") arithmetic on the FP32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2: a 48-bit
// significand (relative rounding ~2^-48 ~ 3.6e-15) with FP32's exponent range.  On B300 one
// FP64 instruction costs about as much issue bandwidth as 73 FP32 instructions, while a
// df64 add or multiply is ~10 FP32 instructions, so df64 delivers FP64-class precision for
// the inner-region geodesic steps several times faster than native FP64.
//
// The building blocks are the classical error-free transformations:
//   two-sum (Knuth, TAOCP vol. 2, 4.2.2): s = a + b exactly as s + e;
//   fast-two-sum (Dekker 1971) for |a| >= |b|;
//   two-product with a fused multiply-add: p = a b exactly as p + fma(a, b, -p).
// Division uses one Newton correction of the float quotient; sin/cos reduce the argument by
// multiples of pi/2 (pi/2 stored as three floats) and sum the Taylor series of sin and cos
// on [-pi/4, pi/4] (terms to x^15 / 15! and x^16 / 16!; the small high-order terms in float).
#pragma once

#include "raptor_math.cuh"

namespace raptor {
// The type and its overloads live in a nested namespace and are found by argument-dependent
// lookup, so they do not hide the global fmin/fmax/fabs for double arguments.
namespace dfns {

struct df64 {
    float hi, lo;
    constexpr RAPTOR_HD df64() : hi(0.f), lo(0.f) {}
    constexpr RAPTOR_HD df64(float h, float l) : hi(h), lo(l) {}
    // from a double (constants fold at compile time; run-time conversions cost FP64 work)
    constexpr RAPTOR_HD df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    constexpr RAPTOR_HD df64(int i) : hi((float)i), lo(0.f) {}
    RAPTOR_HD explicit operator double() const { return (double)hi + (double)lo; }
    RAPTOR_HD explicit operator float() const { return hi + lo; }
};

RAPTOR_HD df64 df_fast_two_sum(float a, float b) {
    const float s = a + b;
    return df64(s, b - (s - a));
}
RAPTOR_HD df64 df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return df64(s, (a - (s - bb)) + (b - bb));
}
RAPTOR_HD df64 df_two_prod(float a, float b) {
    const float p = a * b;
    return df64(p, fmaf(a, b, -p));
}

// Addition with one error-free transformation of the leading parts: the low parts are
// added in plain float, so the error is bounded by a few units of 2^-48 of |a| + |b|
// (not of |a + b|), like the rounding of the operands themselves.
RAPTOR_HD df64 operator+(df64 a, df64 b) {
    df64 s = df_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return df_fast_two_sum(s.hi, s.lo);
}
RAPTOR_HD df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
RAPTOR_HD df64 operator-(df64 a, df64 b) { return a + (-b); }
// Products are left unrenormalised: (p, e + cross terms) has |lo| <= ~1.5 ulp(p) (a product
// has no cancellation), so the pair is nearly normalised and every operation that consumes
// it keeps its error bound within a small factor; the value is the one fast-two-sum would
// give (that transformation is exact).  Sums, where cancellation can leave a large low
// part, are renormalised.
RAPTOR_HD df64 operator*(df64 a, df64 b) {
    df64 p = df_two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return p;
}
// b * q for a float q: the leading product exact, the low part's product rounded.
RAPTOR_HD df64 df_mul_f(df64 b, float q) {
    df64 p = df_two_prod(b.hi, q);
    p.lo = fmaf(b.lo, q, p.lo);
    return p;
}
// Approximate float reciprocal (a few ulp): it only seeds quotients that the df64
// residuals below correct.
RAPTOR_HD float df_rcp_approx(float v) {
#ifdef __CUDA_ARCH__
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
#else
    return 1.f / v;
#endif
}
RAPTOR_HD df64 operator/(df64 a, df64 b) {
    // q1 = a/b from the float reciprocal, r = a - q1 b in df64, q2 = r/b; a second residual
    // gives the last bits: q = q1 + q2 + q3
    const float rb = df_rcp_approx(b.hi);
    const float q1 = a.hi * rb;
    df64 r = a - df_mul_f(b, q1);
    const float q2 = r.hi * rb;
    r = r - df_mul_f(b, q2);
    const float q3 = r.hi * rb;
    df64 q = df_fast_two_sum(q1, q2);
    return q + df64(q3, 0.f);
}
RAPTOR_HD df64& operator+=(df64& a, df64 b) { a = a + b; return a; }
RAPTOR_HD df64& operator-=(df64& a, df64 b) { a = a - b; return a; }
RAPTOR_HD df64& operator*=(df64& a, df64 b) { a = a * b; return a; }
RAPTOR_HD bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
RAPTOR_HD bool operator>(df64 a, df64 b) { return b < a; }
RAPTOR_HD bool operator>=(df64 a, df64 b) { return !(a < b); }
RAPTOR_HD bool operator<=(df64 a, df64 b) { return !(b < a); }
RAPTOR_HD df64 fabs(df64 a) { return a.hi < 0.f ? -a : a; }
RAPTOR_HD df64 fmin(df64 a, df64 b) { return a < b ? a : b; }
RAPTOR_HD df64 fmax(df64 a, df64 b) { return a < b ? b : a; }


RAPTOR_HD df64 df_sqrt(df64 a) {
    // one Newton step on the float square root: s = sqrt(a_hi), s + (a - s^2) / (2 s)
    if (!(a.hi > 0.f)) return df64(0.f, 0.f);
    const float s = sqrtf(a.hi);
    const df64 e = a - df_two_prod(s, s);
    return df_fast_two_sum(s, e.hi * (0.5f * df_rcp_approx(s)));
}

// sin and cos of x (any moderate argument; the geodesic code passes theta in (0, pi)).
// Kept out of line on the device: the table form below calls it only off [0, pi], and
// inlining it at every call site would only grow the integrators' code.
#ifdef __CUDACC__
static __host__ __device__ __noinline__
#else
inline
#endif
void df_sincos(df64 x, df64* s_out, df64* c_out) {
    // pi/2 = P1 + P2 + P3 (three floats; residual ~1e-23)
    const float P1 = 1.57079637f, P2 = -4.37113883e-08f, P3 = -1.71512451e-15f;
    const float kf = rintf((x.hi + x.lo) * 0.636619747f);
    df64 r = x - df_two_prod(kf, P1);
    r = r - df_two_prod(kf, P2);
    r = r - df64(kf * P3, 0.f);
    const int q = ((int)kf) & 3;
    const df64 r2 = r * r;
    // Taylor series on |r| <= pi/4 in r^2 (Horner): (-1)^n/(2n+1)! and (-1)^n/(2n)! as float pairs
    const float so[20] = {1.f, 0.f, -0.166666672f, 4.96705388e-09f, 0.00833333377f, -4.34617203e-10f,
                          -0.000198412701f, 2.72559687e-12f, 2.75573188e-06f, 3.79357122e-14f, -2.50521079e-08f,
                          -4.41762304e-16f, 1.60590444e-10f, -5.35252651e-18f, -7.64716361e-13f, -1.22007105e-20f,
                          2.81145736e-15f, -1.04620847e-22f, -8.22063508e-18f, -1.6814781e-25f};
    const float ce[20] = {1.f, 0.f, -0.5f, 0.f, 0.0416666679f, -1.24176347e-09f, -0.00138888892f, 3.36310944e-11f,
                          2.48015876e-05f, -3.40699609e-13f, -2.755732e-07f, 7.57511221e-15f, 2.08767559e-09f,
                          1.10828391e-16f, -1.14707454e-11f, -2.37220769e-19f, 4.77947726e-14f, 7.62544404e-22f,
                          -1.56192068e-16f, -1.54044715e-24f};
    // Terms whose size on |r| <= pi/4 is below ~2^-24 (sin from r^11, cos from r^12) need
    // only float precision: that tail is summed in float and the leading terms in df64.
    // Truncation: the first omitted terms, r^17 / 17! and r^18 / 18!, are below 5e-17.
    const float r2f = r2.hi;
    float ts = 0.f, tc = 0.f;
#pragma unroll
    for (int n = 7; n >= 5; --n) ts = fmaf(ts, r2f, so[2 * n]);
#pragma unroll
    for (int n = 8; n >= 6; --n) tc = fmaf(tc, r2f, ce[2 * n]);
    df64 ps(ts, 0.f), pc(tc, 0.f);
#pragma unroll
    for (int n = 4; n >= 0; --n) ps = ps * r2 + df64(so[2 * n], so[2 * n + 1]);
#pragma unroll
    for (int n = 5; n >= 0; --n) pc = pc * r2 + df64(ce[2 * n], ce[2 * n + 1]);
    const df64 sr = ps * r, cr = pc;
    // quadrant: sin(r + q pi/2), cos(r + q pi/2)
    if (q == 0) { *s_out = sr; *c_out = cr; }
    else if (q == 1) { *s_out = cr; *c_out = -sr; }
    else if (q == 2) { *s_out = -sr; *c_out = -cr; }
    else { *s_out = -cr; *c_out = sr; }
}

// sin and cos of theta in [0, pi] (the range of the geodesic's polar angle) from a table of
// the 65 nodes theta_i = i pi / 64 (float pairs, raptor::sincos_node) and the
// Taylor series of the offset d = theta - theta_i, |d| <= pi / 128: sin d to d^7 and cos d
// to d^6 (first omitted terms < 1e-20), the terms below ~2^-24 of the leading one summed in
// float; then the angle-addition formulas.  Outside [0, pi]: df_sincos.
RAPTOR_HD void df_sincos_tab(df64 x, df64* s_out, df64* c_out) {
    const float xf = x.hi + x.lo;
    if (!(xf >= 0.f && xf <= 3.14159265f)) {
        df_sincos(x, s_out, c_out);
        return;
    }
    // pi / 64 = Q1 + Q2 + Q3 (three floats)
    const float Q1 = 0.0490873866f, Q2 = -1.36598088e-09f, Q3 = -5.35976409e-17f;
    const int i = (int)rintf(xf * (::raptor::kSinTabN / 3.14159265358979f));
    const float fi = (float)i;
    df64 d = x - df_two_prod(fi, Q1);
    d = d - df_two_prod(fi, Q2);
    d = d - df64(fi * Q3, 0.f);
    const df64 d2 = d * d;
    const float d2f = d2.hi;
    // sin d = d (1 + d2 (-1/6 + d2 (1/120 + d2 (-1/5040)))): the last two terms in float
    const float ts = fmaf(-0.000198412701f, d2f, 0.00833333377f);
    df64 ps = df64(ts, 0.f) * d2 + df64(-0.166666672f, 4.96705388e-09f);
    ps = ps * d2 + df64(1.f, 0.f);
    const df64 sd = ps * d;
    // cos d = 1 + d2 (-1/2 + d2 (1/24 + d2 (-1/720))): the last two terms in float
    const float tc = fmaf(-0.00138888892f, d2f, 0.0416666679f);
    df64 pc = df64(tc, 0.f) * d2 + df64(-0.5f, 0.f);
    pc = pc * d2 + df64(1.f, 0.f);
    const float4 t = ::raptor::sincos_node(i);
    const df64 s0(t.x, t.y), c0(t.z, t.w);
    *s_out = s0 * pc + c0 * sd;
    *c_out = c0 * pc - s0 * sd;
}

RAPTOR_HD void sc(df64 v, df64* s, df64* c) { df_sincos_tab(v, s, c); }
// exact scalings by powers of two: two FP32 multiplies instead of a double-float product
RAPTOR_HD df64 twice(df64 v) { return df64(2.f * v.hi, 2.f * v.lo); }
RAPTOR_HD df64 halve(df64 v) { return df64(0.5f * v.hi, 0.5f * v.lo); }
RAPTOR_HD df64 rsq(df64 v) { return df64(1.0) / df_sqrt(v); }

}  // namespace dfns
using dfns::df64;
using dfns::df_fast_two_sum;
using dfns::df_sincos;
using dfns::df_sincos_tab;
using dfns::df_sqrt;
using dfns::df_two_prod;
using dfns::df_two_sum;

// one double-float division per force evaluation instead of two
template <>
struct JointInverse<df64> {
    static constexpr bool value = true;
};

template <>
struct Real<df64> {
    static RAPTOR_HD df64 sqrt_(df64 v) { return df_sqrt(v); }
    static RAPTOR_HD df64 rcp(df64 v) { return df64(1.0) / v; }
};

}  // namespace raptor
