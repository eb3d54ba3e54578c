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
__device__ __forceinline__ void correct_particle_fp64(double *st, double *t, double *dt, size_t N, int i,
                                                      double t1, const double (&f)[9], double eta,
                                                      double dt_min, double dt_max, double dt_shared,
                                                      nb_ctl *ctl)
{
    const double h = t1 - t[i];
    const double ih = 1.0 / h;  // exact: h is a power of two (the particle's step)
    double n2[6] = {0, 0, 0, 0, 0, 0};  // squared norms of a1, j1, s1, c1, d1, e1
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
    }
    t[i] = t1;
    bool hit = false;
    const double dtn =
        dt_shared > 0.0 ? dt_shared : quantise(aarseth_dt(n2, eta), dt[i], t1, dt_min, dt_max, &hit);
    dt[i] = dtn;
    if (hit)
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->floor_hits), 1ull);
    if (!finite)
        atomicOr(&ctl->err, NB_ERR_NONFINITE);
}

}  // namespace nbk
