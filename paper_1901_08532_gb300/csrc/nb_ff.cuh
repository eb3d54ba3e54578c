// Float-float ("EX") arithmetic for the extended-precision evaluation
// (paper, section 3 item 6: a number of about 48 mantissa bits with the
// single-precision exponent range, built from 32-bit operations only).
//
// A value is the unevaluated sum h + l of two FP32 numbers with |l| <= ulp(h)/2
// after normalisation.  The building blocks are the classical error-free
// transformations:
//   TwoSum (Knuth):         s + e == a + b exactly, any a, b;
//   Fast2Sum (Dekker):      s + e == a + b exactly when |a| >= |b| (or a == 0);
//   TwoProd (FMA form):     p + e == a * b exactly (barring underflow),
//                           e = fma(a, b, -p);
// and on top of them the "sloppy" and accurate double-word sums and the
// double-word product of Dekker (1971), whose error bounds are analysed by
// Joldes, Muller and Popescu (ACM TOMS 44, 2017): relative error of a
// product <= about 4 u^2, of a sloppy sum <= about 2 u^2 (|x| + |y|) /
// |x + y|, of an accurate sum <= about 3 u^2, u = 2^-24.
//
// Every helper is written for T = float (one value) or T = float2 (two
// independent values in the lanes of the packed f32x2 instructions).  The
// _rn intrinsics are never contracted or reassociated by the compiler, which
// the transformations rely on.
#pragma once

#include <cuda_runtime.h>

namespace nbk {
namespace ff {

__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float neg(float a) { return -a; }
__device__ __forceinline__ float splat(float, float v) { return v; }

__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 splat(float2, float v) { return make_float2(v, v); }

template <class T>
struct FF {
    T h, l;
};

template <class T>
__device__ __forceinline__ FF<T> two_sum(T a, T b)
{
    const T s = add(a, b);
    const T bb = sub(s, a);
    const T e = add(sub(a, sub(s, bb)), sub(b, bb));
    return {s, e};
}

template <class T>
__device__ __forceinline__ FF<T> fast_two_sum(T a, T b)
{
    const T s = add(a, b);
    return {s, sub(b, sub(s, a))};
}

template <class T>
__device__ __forceinline__ FF<T> two_prod(T a, T b)
{
    const T p = mul(a, b);
    return {p, fma(a, b, neg(p))};
}

// The operations below return UNNORMALISED double words: the high part is
// the FP32 rounding of the leading term and the low part gathers everything
// else, so |l| may exceed ulp(h)/2 by a few ulps.  Skipping the final
// Fast2Sum of the textbook forms saves three operations per call and does
// not change the value h + l; the products and sums that consume such a
// pair stay accurate to a few u^2 of their operands (a float32 emulation of
// the pair term below gives the same errors with and without it).

// x + y, the "sloppy" double-word sum: exact for the high parts, the low
// parts added in FP32; accurate unless x and y nearly cancel.
template <class T>
__device__ __forceinline__ FF<T> add(const FF<T> &x, const FF<T> &y)
{
    const FF<T> s = two_sum(x.h, y.h);
    return {s.h, add(s.l, add(x.l, y.l))};
}

// x + y with relative error of a few u^2 even under cancellation (the
// accurate double-word sum: both parts pass through TwoSum).
template <class T>
__device__ __forceinline__ FF<T> add_accurate(const FF<T> &x, const FF<T> &y)
{
    const FF<T> s = two_sum(x.h, y.h);
    const FF<T> t = two_sum(x.l, y.l);
    const FF<T> v = fast_two_sum(s.h, add(s.l, t.h));
    return {v.h, add(t.l, v.l)};
}

// x * y (the l * l term is below the format's resolution).
template <class T>
__device__ __forceinline__ FF<T> mul(const FF<T> &x, const FF<T> &y)
{
    const T p = mul(x.h, y.h);
    T e = fma(x.h, y.h, neg(p));
    e = fma(x.h, y.l, e);
    e = fma(x.l, y.h, e);
    return {p, e};
}

// x * c for an FP32 constant c.
template <class T>
__device__ __forceinline__ FF<T> mul(const FF<T> &x, T c)
{
    const T p = mul(x.h, c);
    return {p, fma(x.l, c, fma(x.h, c, neg(p)))};
}

// x * x.
template <class T>
__device__ __forceinline__ FF<T> sqr(const FF<T> &x)
{
    const T p = mul(x.h, x.h);
    return {p, fma(add(x.h, x.h), x.l, fma(x.h, x.h, neg(p)))};
}

// x * y + z in one pass: the exact product's high part meets z.h in a
// TwoSum and all lower-order terms are gathered in the low part.
template <class T>
__device__ __forceinline__ FF<T> mad(const FF<T> &x, const FF<T> &y, const FF<T> &z)
{
    const T p = mul(x.h, y.h);
    T e = fma(x.h, y.h, neg(p));
    e = fma(x.h, y.l, e);
    e = fma(x.l, y.h, e);
    const FF<T> s = two_sum(p, z.h);
    return {s.h, add(s.l, add(e, z.l))};
}

// R^(-1/2) for R > 0: the special-function estimate q0 (relative error
// below 2^-22) refined by one Newton step q = q0 + q0 (1 - R q0^2) / 2, with
// the residual 1 - R q0^2 formed from the exact square of q0 and a
// double-word product, so the result carries about 2^-45 relative error.
template <class T>
__device__ __forceinline__ FF<T> rsqrt(const FF<T> &R, T q0)
{
    const FF<T> q02 = two_prod(q0, q0);
    const FF<T> t = mul(R, q02);
    const T one = splat(q0, 1.0f);
    const T d = sub(sub(one, t.h), t.l);
    return fast_two_sum(q0, mul(mul(q0, d), splat(q0, 0.5f)));
}

// Unnormalised running sum (the cascaded summation "Sum2" of Ogita, Rump
// and Oishi): acc.h is the FP32 sum of the high parts, acc.l gathers every
// rounding error and every low part.  Normalise before the l part grows
// with the number of terms (once per tile).
template <class T>
__device__ __forceinline__ void accumulate(FF<T> &acc, const FF<T> &t)
{
    const FF<T> s = two_sum(acc.h, t.h);
    acc.h = s.h;
    acc.l = add(acc.l, add(s.l, t.l));
}

// acc += x * y (the product's low part goes straight into acc.l).
template <class T>
__device__ __forceinline__ void accumulate_mul(FF<T> &acc, const FF<T> &x, const FF<T> &y)
{
    accumulate(acc, mul(x, y));
}

}  // namespace ff
}  // namespace nbk

namespace nbk {

// FP32 rows of the EX j-buffer: x_h[3] x_l[3] v_h[3] v_l[3] a_h[3] a_l[3] m_h m_l.
constexpr int NCX = 20;

__device__ __forceinline__ float rsqrt_est_v(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 rsqrt_est_v(float2 x) { return make_float2(rsqrt_est_v(x.x), rsqrt_est_v(x.y)); }

// The i-particle of an EX evaluation, negated: -x, -v, -a as double words.
template <class T>
struct ExI {
    ff::FF<T> x[3], v[3], a[3];
};

// One pair term (two in the lanes of T = float2) in double-word arithmetic,
// the same formula as the FP64 pair: with r, v, a the differences j - i,
// R = r.r + eps^2, q = R^(-1/2), mu = m_j q^3, alpha = (r.v) q^2,
// beta = (v.v + r.a) q^2 + alpha^2, u = v - 3 alpha r and
// w = a - 6 alpha u - 3 beta r:  acc += mu r, jerk += mu u, snap += mu w
// into the unnormalised running sums p[0..8].  c[] are the 20 j-rows.
template <class T>
__device__ __forceinline__ void pair_ex(const T (&c)[NCX], const ExI<T> &ni, const ff::FF<T> &eps2,
                                        ff::FF<T> (&p)[9])
{
    using ff::FF;
    FF<T> r[3], dv[3], da[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r[k] = ff::add_accurate(FF<T>{c[k], c[3 + k]}, ni.x[k]);   // close pairs cancel
        dv[k] = ff::add(FF<T>{c[6 + k], c[9 + k]}, ni.v[k]);
        da[k] = ff::add(FF<T>{c[12 + k], c[15 + k]}, ni.a[k]);
    }
    const FF<T> R = ff::mad(r[0], r[0], ff::mad(r[1], r[1], ff::mad(r[2], r[2], eps2)));
    const FF<T> rv = ff::mad(r[0], dv[0], ff::mad(r[1], dv[1], ff::mul(r[2], dv[2])));
    const FF<T> sv = ff::mad(r[0], da[0], ff::mad(r[1], da[1], ff::mad(r[2], da[2],
                     ff::mad(dv[0], dv[0], ff::mad(dv[1], dv[1], ff::sqr(dv[2]))))));
    const FF<T> q = ff::rsqrt(R, rsqrt_est_v(R.h));
    const FF<T> q2 = ff::sqr(q);
    const FF<T> mu = ff::mul(ff::mul(FF<T>{c[18], c[19]}, q), q2);
    const FF<T> al = ff::mul(rv, q2);
    const FF<T> be = ff::mad(al, al, ff::mul(sv, q2));
    const T m3 = ff::splat(c[0], -3.0f), two = ff::splat(c[0], 2.0f);
    const FF<T> na3 = ff::mul(al, m3);
    const FF<T> na6 = {ff::mul(na3.h, two), ff::mul(na3.l, two)};   // exact doubling
    const FF<T> nb3 = ff::mul(be, m3);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const FF<T> u = ff::mad(na3, r[k], dv[k]);
        const FF<T> w = ff::mad(na6, u, ff::mad(nb3, r[k], da[k]));
        ff::accumulate_mul(p[k], mu, r[k]);
        ff::accumulate_mul(p[3 + k], mu, u);
        ff::accumulate_mul(p[6 + k], mu, w);
    }
}

}  // namespace nbk
