// The FP64 corrector of one particle, shared by the corrector kernel and the
// device-resident block stepper so that both take identical decisions.
#pragma once

#include "nb_device.cuh"

namespace nbk {

// ------------------------------------------- corrector of one particle, FP64

// Corrector, interpolation and new step of particle i at time t1 with its
// new acceleration, jerk and snap f[0..8] (section 3, section 3 item 3):
// the Hermite corrector above, the quintic's crackle, pop and a^(5), the
// generalised Aarseth criterion quantised to a power of two.  State rows
// st[(F * 3 + d) * N + i].  Sets the control block's error flag for a
// non-finite value and counts floor hits.
//
// noise > 0 (nb_config.step_noise): the relative rounding level of the
// evaluated a, jerk and snap.  The quintic's residuals R1, R2, R3 then carry
// a rounding floor (noise times the magnitudes they are formed from), which
// the interpolation divides by h^3, h^4, h^5; the criterion uses the
// magnitudes of crackle, pop and a^(5) less their floors (at least 0), so it
// responds only to resolved derivatives.  noise = 0 is the criterion as is.
__device__ __forceinline__ void correct_particle_fp64(double *st, double *t, double *dt, size_t N, int i,
                                                      double t1, const double (&f)[9], double eta,
                                                      double dt_min, double dt_max, double dt_shared,
                                                      nb_ctl *ctl, double noise = 0.0)
{
    const double h = t1 - t[i];
    const double ih = 1.0 / h;  // exact: h is a power of two (the particle's step)
    double n2[6] = {0, 0, 0, 0, 0, 0};  // squared norms of a1, j1, s1, c1, d1, e1
    double m2[3] = {0, 0, 0};  // squared norms of a0, j0, s0 (their rounding floor)
    bool finite = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double *px = st + (F_X * 3 + d) * N + i;
        double *pv = st + (F_V * 3 + d) * N + i;
        double *pa = st + (F_A * 3 + d) * N + i;
        double *pj = st + (F_J * 3 + d) * N + i;
        double *ps = st + (F_S * 3 + d) * N + i;
        double *pc = st + (F_C * 3 + d) * N + i;
        const double a0 = *pa, j0 = *pj, s0 = *ps;
        const double a1 = f[d], j1 = f[3 + d], s1 = f[6 + d];
        const Corrected r = hermite_correct(h, ih, *px, *pv, a0, j0, s0, a1, j1, s1);
        finite = finite && isfinite(r.x1) && isfinite(r.v1) && isfinite(a1) && isfinite(j1) &&
                 isfinite(s1) && isfinite(r.c1);
        *px = r.x1;
        *pv = r.v1;
        *pa = a1;
        *pj = j1;
        *ps = s1;
        *pc = r.c1;
        n2[0] = fma(a1, a1, n2[0]);
        n2[1] = fma(j1, j1, n2[1]);
        n2[2] = fma(s1, s1, n2[2]);
        n2[3] = fma(r.c1, r.c1, n2[3]);
        n2[4] = fma(r.d1, r.d1, n2[4]);
        n2[5] = fma(r.e1, r.e1, n2[5]);
        m2[0] = fma(a0, a0, m2[0]);
        m2[1] = fma(j0, j0, m2[1]);
        m2[2] = fma(s0, s0, m2[2]);
    }
    t[i] = t1;
    bool hit = false;
    if (noise > 0.0 && dt_shared <= 0.0) {
        // rounding floors of R1, R2, R3 and of crackle, pop and a^(5)
        const double na0 = sqrt(m2[0]), nj0 = sqrt(m2[1]), ns0 = sqrt(m2[2]);
        const double na1 = sqrt(n2[0]), nj1 = sqrt(n2[1]), ns1 = sqrt(n2[2]);
        const double s1f = noise * (na1 + na0 + h * (nj0 + 0.5 * h * ns0));
        const double s2f = noise * h * (nj1 + nj0 + h * ns0);
        const double s3f = noise * h * h * (ns1 + ns0);
        const double ih3 = ih * ih * ih;
        const double fc = (60.0 * s1f + 36.0 * s2f + 9.0 * s3f) * ih3;
        const double fd = (360.0 * s1f + 192.0 * s2f + 36.0 * s3f) * ih3 * ih;
        const double fe = (720.0 * s1f + 360.0 * s2f + 60.0 * s3f) * ih3 * ih * ih;
        const double c = fmax(sqrt(n2[3]) - fc, 0.0), dd = fmax(sqrt(n2[4]) - fd, 0.0);
        const double e = fmax(sqrt(n2[5]) - fe, 0.0);
        n2[3] = c * c;
        n2[4] = dd * dd;
        n2[5] = e * e;
    }
    const double dtn =
        dt_shared > 0.0 ? dt_shared : quantise(aarseth_dt(n2, eta), dt[i], t1, dt_min, dt_max, &hit);
    dt[i] = dtn;
    if (hit)
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->floor_hits), 1ull);
    if (!finite)
        atomicOr(&ctl->err, NB_ERR_NONFINITE);
}

}  // namespace nbk
