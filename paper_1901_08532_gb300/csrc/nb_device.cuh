// Device arithmetic shared by the kernels: the softened pair terms (FP64 and
// packed FP32), the Taylor predictor and the power-of-two step
// quantisation.  Each function states the formula it implements; the
// kernels that use them cite the paper's passages.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nb_internal.cuh"

namespace nbk {

// ------------------------------------------------------------ pair, FP64

// One softened pair term in FP64, accumulated into p[0..8]
// (acc, jerk, snap).  With r, v, a the differences j - i, R = r.r + eps^2,
// q = R^(-1/2), mu = m_j q^3, alpha = (r.v) q^2, beta = (v.v + r.a) q^2 +
// alpha^2, u = v - 3 alpha r and w = a - 6 alpha u - 3 beta r:
//   acc += mu r,  jerk += mu u,  snap += mu w.
// (jerk = mu v - 3 alpha A and snap = mu a - 6 alpha J - 3 beta A rewritten
// so that every step is one fused multiply-add.)
__device__ __forceinline__ void pair_fp64(const double2 &p0, const double2 &p1, const double2 &p2,
                                          const double2 &p3, const double2 &p4, double xi,
                                          double yi, double zi, double vxi, double vyi, double vzi,
                                          double axi, double ayi, double azi, double eps2,
                                          double *p)
{
    const double dx = p0.x - xi, dy = p0.y - yi, dz = p1.x - zi;
    const double mj = p1.y;
    const double dvx = p2.x - vxi, dvy = p2.y - vyi, dvz = p3.x - vzi;
    const double dax = p3.y - axi, day = p4.x - ayi, daz = p4.y - azi;
    const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    const double rv = fma(dx, dvx, fma(dy, dvy, dz * dvz));
    const double sv = fma(dx, dax, fma(dy, day, fma(dz, daz, fma(dvx, dvx, fma(dvy, dvy, dvz * dvz)))));
    const double q = nbk::rsqrt_fp64(r2);
    const double q2 = q * q;
    const double mu = mj * q * q2;
    const double al = rv * q2;
    const double be = fma(al, al, sv * q2);
    const double a3 = 3.0 * al, a6 = 6.0 * al, b3 = 3.0 * be;
    const double ux = fma(-a3, dx, dvx), uy = fma(-a3, dy, dvy), uz = fma(-a3, dz, dvz);
    const double wx = fma(-a6, ux, fma(-b3, dx, dax));
    const double wy = fma(-a6, uy, fma(-b3, dy, day));
    const double wz = fma(-a6, uz, fma(-b3, dz, daz));
    p[0] = fma(mu, dx, p[0]);
    p[1] = fma(mu, dy, p[1]);
    p[2] = fma(mu, dz, p[2]);
    p[3] = fma(mu, ux, p[3]);
    p[4] = fma(mu, uy, p[4]);
    p[5] = fma(mu, uz, p[5]);
    p[6] = fma(mu, wx, p[6]);
    p[7] = fma(mu, wy, p[7]);
    p[8] = fma(mu, wz, p[8]);
}

// ------------------------------------------------ pair, packed FP32 (mixed)

constexpr int NCF = 13;  // FP32 rows of the mixed j-buffer

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Special-function estimates of R^(-1/2) and 1/R in their flush-to-zero
// forms.  The non-flushing forms add a subnormal-input path around every
// estimate (about 10 % of the packed FMA rate in the throughput probes of
// k_peaks.cu); here R >= eps^2 >= 2^-80 is always a normal number, so the
// two forms give the same result (1/R would differ only for R > 2^126).
__device__ __forceinline__ float rsqrt_est(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_est(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// j per lane summed in FP32 (kMixedFoldJ / 2 terms in each half of a packed
// pair) before each fold into the compensated sums.  The FP32 rounding of a
// running sum grows with its length: over all 2^20 particles of the
// Plummer/Salpeter model, 256 j per fold left 32 snaps above 1e-6 of their
// condition number sum_j |S_ij| and whole 512-j tiles 369; 128 j leaves 9
// (at most 1.11e-6, the rest of that error being the pair terms' own FP32
// rounding), for 1.4 % more time than 256.
constexpr int kMixedFoldJ = 128;

// Two pair terms (j, j+1) for one i.  c[] are the 13 j-rows (as pairs), ni[]
// the negated i-values (-xh,-yh,-zh,-xl,-yl,-zl,-vx,-vy,-vz,-ax,-ay,-az).
// With r, v, a = j - i, R = r.r + eps^2, q = R^(-1/2), mu = m_j q^3,
// alpha = (r.v) q^2, beta = (v.v + r.a) q^2 + alpha^2, u = v - 3 alpha r and
// w = a - 6 alpha u - 3 beta r:  acc += mu r, jerk += mu u, snap += mu w.
__device__ __forceinline__ void pair_mixed2(const float2 (&c)[NCF], const float2 (&ni)[12],
                                            float2 eps2, float2 (&p)[9])
{
    const float2 dx = add2(add2(c[0], ni[0]), add2(c[4], ni[3]));
    const float2 dy = add2(add2(c[1], ni[1]), add2(c[5], ni[4]));
    const float2 dz = add2(add2(c[2], ni[2]), add2(c[6], ni[5]));
    const float2 dvx = add2(c[7], ni[6]), dvy = add2(c[8], ni[7]), dvz = add2(c[9], ni[8]);
    const float2 dax = add2(c[10], ni[9]), day = add2(c[11], ni[10]), daz = add2(c[12], ni[11]);
    const float2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
    const float2 rv = fma2(dx, dvx, fma2(dy, dvy, mul2(dz, dvz)));
    const float2 sv = fma2(dx, dax, fma2(dy, day, fma2(dz, daz, fma2(dvx, dvx, fma2(dvy, dvy, mul2(dvz, dvz))))));
    // q = R^(-1/2) and q^2 = 1/R both from the special-function unit, so the
    // squaring error of an estimate does not enter mu = m q^3 and alpha/beta
    const float2 q = make_float2(rsqrt_est(r2.x), rsqrt_est(r2.y));
    const float2 q2 = make_float2(rcp_est(r2.x), rcp_est(r2.y));
    const float2 mu = mul2(mul2(c[3], q), q2);
    const float2 al = mul2(rv, q2);
    const float2 be = fma2(al, al, mul2(sv, q2));
    const float2 na3 = mul2(al, f2(-3.0f)), na6 = mul2(al, f2(-6.0f)), nb3 = mul2(be, f2(-3.0f));
    const float2 ux = fma2(na3, dx, dvx), uy = fma2(na3, dy, dvy), uz = fma2(na3, dz, dvz);
    const float2 wx = fma2(na6, ux, fma2(nb3, dx, dax));
    const float2 wy = fma2(na6, uy, fma2(nb3, dy, day));
    const float2 wz = fma2(na6, uz, fma2(nb3, dz, daz));
    p[0] = fma2(mu, dx, p[0]);
    p[1] = fma2(mu, dy, p[1]);
    p[2] = fma2(mu, dz, p[2]);
    p[3] = fma2(mu, ux, p[3]);
    p[4] = fma2(mu, uy, p[4]);
    p[5] = fma2(mu, uz, p[5]);
    p[6] = fma2(mu, wx, p[6]);
    p[7] = fma2(mu, wy, p[7]);
    p[8] = fma2(mu, wz, p[8]);
}

// --------------------------------------------------------------- predictor

struct Taylor {
    double x, v, a;
};

// Horner form of x + v d + a d^2/2 + j d^3/6 + s d^4/24 + c d^5/120 and its
// first two derivatives.
__device__ __forceinline__ Taylor taylor(double x, double v, double a, double j, double s, double c,
                                         double d)
{
    const double d2 = 0.5 * d, d3 = d * (1.0 / 3.0), d4 = 0.25 * d, d5 = 0.2 * d;
    Taylor r;
    r.x = fma(d, fma(d2, fma(d3, fma(d4, fma(d5, c, s), j), a), v), x);
    r.v = fma(d, fma(d2, fma(d3, fma(d4, c, s), j), a), v);
    r.a = fma(d, fma(d2, fma(d3, c, s), j), a);
    return r;
}

// ------------------------------------------------------- step quantisation

// Largest power of two <= x for positive normal x (clears the mantissa).
__device__ __forceinline__ double pow2_floor(double x)
{
    return __hiloint2double(__double2hiint(x) & 0x7ff00000, 0);
}

__device__ __forceinline__ double quantise(double crit, double dt_old, double t1, double dt_min, double dt_max,
                           bool *floor_hit)
{
    double p;
    *floor_hit = false;
    if (!(crit >= dt_min)) {
        *floor_hit = true;
        p = dt_min;
    } else {
        p = isinf(crit) ? dt_max : fmin(pow2_floor(crit), dt_max);
    }
    if (dt_old > 0.0 && p > dt_old) {
        const double d2 = 2.0 * dt_old;
        const double q = t1 * (1.0 / d2);  // exact: d2 is a power of two
        p = (q == trunc(q)) ? d2 : dt_old;
    }
    return p;
}

// -------------------------------------------------------------- corrector

// One component of the 6th-order Hermite corrector over a step h (ih = 1/h,
// exact for power-of-two steps): the velocity change is the two-point
// Hermite quadrature of a(t) with a, a', a'' at both ends,
//   h/2 (a0 + a1) - h^2/10 (j1 - j0) + h^3/120 (s0 + s1),
// and the position change the same quadrature of v(t) with the corrected v1.
// c1, d1, e1 are the 3rd, 4th and 5th derivatives of a at the end of the
// step from the quintic through (a, j, s) at both ends: with the residuals
// R1 = a1 - a0 - j0 h - s0 h^2/2, R2 = h (j1 - j0 - s0 h), R3 = h^2 (s1 - s0),
//   c1 h^3 = 60 R1 - 36 R2 + 9 R3,  d1 h^4 = 360 R1 - 192 R2 + 36 R3,
//   e1 h^5 = 720 R1 - 360 R2 + 60 R3.
struct Corrected {
    double x1, v1, c1, d1, e1;
};

__device__ __forceinline__ Corrected hermite_correct(double h, double ih, double x0, double v0,
                                                     double a0, double j0, double s0, double a1,
                                                     double j1, double s1)
{
    Corrected r;
    r.v1 = fma(h, fma(h, fma(h, (s0 + s1) * (1.0 / 120.0), -(j1 - j0) * 0.1), 0.5 * (a0 + a1)), v0);
    r.x1 = fma(h, fma(h, fma(h, (j0 + j1) * (1.0 / 120.0), -(a1 - a0) * 0.1), 0.5 * (v0 + r.v1)), x0);
    const double R1 = a1 - fma(h, fma(0.5 * h, s0, j0), a0);
    const double R2 = h * (j1 - fma(h, s0, j0));
    const double R3 = h * h * (s1 - s0);
    const double ih3 = ih * ih * ih;
    r.c1 = (60.0 * R1 - 36.0 * R2 + 9.0 * R3) * ih3;
    r.d1 = (360.0 * R1 - 192.0 * R2 + 36.0 * R3) * ih3 * ih;
    r.e1 = (720.0 * R1 - 360.0 * R2 + 60.0 * R3) * ih3 * ih * ih;
    return r;
}

// Generalised Aarseth criterion in the 6th-order form from the squared
// norms n2 = |a|^2, |j|^2, |s|^2, |c|^2, |d|^2, |e|^2:
// eta (A1 / A4)^(1/3), A1 = sqrt(|a| |s|) + |j|, A4 = sqrt(|c| |e|) + |d|.
// A1 = A4 = 0 (a particle under no force, e.g. a lone one) sets no bound:
// +infinity, which quantise() maps to dt_max.
__device__ __forceinline__ double aarseth_dt(const double (&n2)[6], double eta)
{
    const double A1 = sqrt(sqrt(n2[0]) * sqrt(n2[2])) + sqrt(n2[1]);
    const double A4 = sqrt(sqrt(n2[3]) * sqrt(n2[5])) + sqrt(n2[4]);
    if (A1 == 0.0 && A4 == 0.0)
        return INFINITY;
    return eta * cbrt(A1 / A4);
}

// Starting step eta_s min(|a|/|j|, sqrt(|a|/|s|)) from |a| and the squared
// norms of j and s; a ratio 0/0 sets no bound (+infinity).
__device__ __forceinline__ double initial_dt(double na, double nj2, double ns2, double eta_s)
{
    const double c1 = (na == 0.0 && nj2 == 0.0) ? INFINITY : na / sqrt(nj2);
    const double c2 = (na == 0.0 && ns2 == 0.0) ? INFINITY : sqrt(na / sqrt(ns2));
    return eta_s * fmin(c1, c2);
}

}  // namespace nbk
