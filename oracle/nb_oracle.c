/*
 * FP64 CPU oracle for the 6th-order Hermite block-time-step direct N-body
 * method described in section 3 of Goz et al. (arXiv:1901.08532), which
 * takes its integrator from Nitadori & Makino 2008.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the CUDA library.  Plain, slow,
 * single-threaded C99, IEEE double precision, compiled with
 * -ffp-contract=off so that x86 and Arm hosts round identically.
 * Each function states the passage it follows.
 */
#include "nb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ----------------------------------------------------------------- helpers */

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

/* Neumaier's improved Kahan summation (Neumaier 1974): running sum plus a
 * separate correction term; the value is sum + comp. */
typedef struct { double sum, comp; } nsum;

static void nsum_add(nsum *s, double x)
{
    double t = s->sum + x;
    if (fabs(s->sum) >= fabs(x))
        s->comp += (s->sum - t) + x;
    else
        s->comp += (x - t) + s->sum;
    s->sum = t;
}

static double nsum_value(const nsum *s) { return s->sum + s->comp; }

/* ----------------------------------------------------------- pair formula */

/* One term of the evaluation sum for Plummer-softened gravity (G = 1).
 * With r = x_j - x_i, v = v_j - v_i, a = a_j - a_i and R = |r|^2 + eps^2:
 *   A = m_j r / R^(3/2)                       (acceleration)
 *   J = m_j v / R^(3/2) - 3 alpha A           (jerk, dA/dt)
 *   S = m_j a / R^(3/2) - 6 alpha J - 3 beta A (snap, d2A/dt2)
 * where alpha = (r.v)/R and beta = (|v|^2 + r.a)/R + alpha^2.  These are the
 * successive time derivatives of A along the trajectories (section 3: the
 * evaluation stage yields acceleration, jerk and snap). */
void orc_pair(const double xi[3], const double vi[3], const double ai[3],
              const double xj[3], const double vj[3], const double aj[3],
              double mj, double eps, double acc[3], double jrk[3], double snp[3])
{
    double r[3], v[3], a[3];
    for (int k = 0; k < 3; k++) {
        r[k] = xj[k] - xi[k];
        v[k] = vj[k] - vi[k];
        a[k] = aj[k] - ai[k];
    }
    double R = dot3(r, r) + eps * eps;
    double mr3 = mj / (R * sqrt(R));
    double alpha = dot3(r, v) / R;
    double beta = (dot3(v, v) + dot3(r, a)) / R + alpha * alpha;
    for (int k = 0; k < 3; k++) {
        acc[k] = mr3 * r[k];
        jrk[k] = mr3 * v[k] - 3.0 * alpha * acc[k];
        snp[k] = mr3 * a[k] - 6.0 * alpha * jrk[k] - 3.0 * beta * acc[k];
    }
}

/* Evaluation kernel semantics (section 3, item 4, steps i-iv): every active
 * particle accumulates the pair terms of all other particles; the self term
 * is skipped (step iii).  Sums are compensated so that the result is within
 * about one rounding of the exact sum of the computed terms. */
void orc_evaluate(int64_t n, const double *m, const double *x, const double *v,
                  const double *a, double eps, int64_t n_act, const int32_t *act,
                  double *acc, double *jrk, double *snp)
{
    for (int64_t k = 0; k < n_act; k++) {
        int64_t i = act[k];
        nsum sa[3] = {{0, 0}, {0, 0}, {0, 0}};
        nsum sj[3] = {{0, 0}, {0, 0}, {0, 0}};
        nsum ss[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (int64_t j = 0; j < n; j++) {
            if (j == i)
                continue;
            double A[3], J[3], S[3];
            orc_pair(&x[3 * i], &v[3 * i], &a[3 * i], &x[3 * j], &v[3 * j],
                     &a[3 * j], m[j], eps, A, J, S);
            for (int c = 0; c < 3; c++) {
                nsum_add(&sa[c], A[c]);
                nsum_add(&sj[c], J[c]);
                nsum_add(&ss[c], S[c]);
            }
        }
        for (int c = 0; c < 3; c++) {
            acc[3 * k + c] = nsum_value(&sa[c]);
            jrk[3 * k + c] = nsum_value(&sj[c]);
            snp[3 * k + c] = nsum_value(&ss[c]);
        }
    }
}

void orc_evaluate_kappa(int64_t n, const double *m, const double *x,
                        const double *v, const double *a, double eps,
                        int64_t n_act, const int32_t *act, double *ka,
                        double *kj, double *ks)
{
    for (int64_t k = 0; k < n_act; k++) {
        int64_t i = act[k];
        nsum sa = {0, 0}, sj = {0, 0}, ss = {0, 0};
        for (int64_t j = 0; j < n; j++) {
            if (j == i)
                continue;
            double A[3], J[3], S[3];
            orc_pair(&x[3 * i], &v[3 * i], &a[3 * i], &x[3 * j], &v[3 * j],
                     &a[3 * j], m[j], eps, A, J, S);
            nsum_add(&sa, norm3(A));
            nsum_add(&sj, norm3(J));
            nsum_add(&ss, norm3(S));
        }
        ka[k] = nsum_value(&sa);
        kj[k] = nsum_value(&sj);
        ks[k] = nsum_value(&ss);
    }
}

/* ---------------------------------------------------------------- predictor */

/* Predictor stage (section 3): Taylor expansion of each particle from its own
 * time t_i to t, using everything the 6th-order scheme stores (a, jerk, snap
 * and the interpolated crackle). */
void orc_predict(int64_t n, double t, const double *ti, const double *x,
                 const double *v, const double *a, const double *j,
                 const double *s, const double *c, double *xp, double *vp,
                 double *ap)
{
    for (int64_t i = 0; i < n; i++) {
        double d = t - ti[i];
        double d2 = d * d, d3 = d2 * d, d4 = d3 * d, d5 = d4 * d;
        for (int k = 0; k < 3; k++) {
            int64_t q = 3 * i + k;
            xp[q] = x[q] + v[q] * d + a[q] * d2 / 2.0 + j[q] * d3 / 6.0 +
                    s[q] * d4 / 24.0 + c[q] * d5 / 120.0;
            vp[q] = v[q] + a[q] * d + j[q] * d2 / 2.0 + s[q] * d3 / 6.0 +
                    c[q] * d4 / 24.0;
            ap[q] = a[q] + j[q] * d + s[q] * d2 / 2.0 + c[q] * d3 / 6.0;
        }
    }
}

/* ---------------------------------------------------------------- corrector */

/* Corrector stage (section 3).  The velocity change is the integral of a(t)
 * over the step, taken with the two-point Hermite quadrature that uses a, a'
 * and a'' at both ends (exact for a(t) of degree <= 5):
 *   int_0^h f = h/2 (f0 + f1) - h^2/10 (f1' - f0') + h^3/120 (f0'' + f1'').
 * The position change is the same quadrature applied to v(t), with the
 * corrected v1 at the end of the step. */
void orc_correct(double h, const double x0[3], const double v0[3],
                 const double a0[3], const double j0[3], const double s0[3],
                 const double a1[3], const double j1[3], const double s1[3],
                 double x1[3], double v1[3])
{
    for (int k = 0; k < 3; k++) {
        v1[k] = v0[k] + h / 2.0 * (a0[k] + a1[k]) - h * h / 10.0 * (j1[k] - j0[k]) +
                h * h * h / 120.0 * (s0[k] + s1[k]);
        x1[k] = x0[k] + h / 2.0 * (v0[k] + v1[k]) - h * h / 10.0 * (a1[k] - a0[k]) +
                h * h * h / 120.0 * (j0[k] + j1[k]);
    }
}

/* Solve the 3x3 system M y = r by Gaussian elimination with partial
 * pivoting (plain textbook form). */
static void solve3(double M[3][3], double r[3], double y[3])
{
    for (int col = 0; col < 3; col++) {
        int piv = col;
        for (int row = col + 1; row < 3; row++)
            if (fabs(M[row][col]) > fabs(M[piv][col]))
                piv = row;
        if (piv != col) {
            for (int k = 0; k < 3; k++) {
                double t = M[col][k];
                M[col][k] = M[piv][k];
                M[piv][k] = t;
            }
            double t = r[col];
            r[col] = r[piv];
            r[piv] = t;
        }
        for (int row = col + 1; row < 3; row++) {
            double f = M[row][col] / M[col][col];
            for (int k = col; k < 3; k++)
                M[row][k] -= f * M[col][k];
            r[row] -= f * r[col];
        }
    }
    for (int row = 2; row >= 0; row--) {
        double acc = r[row];
        for (int k = row + 1; k < 3; k++)
            acc -= M[row][k] * y[k];
        y[row] = acc / M[row][row];
    }
}

/* Higher derivatives for the 6th-order scheme: the unique quintic p(tau) on
 * [0, h] with p, p', p'' equal to (a, jerk, snap) at both ends.  Writing
 * p(tau) = a0 + j0 tau + s0 tau^2/2 + c0 tau^3/6 + d0 tau^4/24 + e0 tau^5/120,
 * the unknowns u = c0 h^3, w = d0 h^4, z = e0 h^5 satisfy
 *   a1 - a0 - j0 h - s0 h^2/2 = u/6 + w/24 + z/120
 *   h (j1 - j0 - s0 h)        = u/2 + w/6  + z/24
 *   h^2 (s1 - s0)             = u   + w/2  + z/6
 * and at the end of the step c1 = (u + w + z/2)/h^3, d1 = (w + z)/h^4,
 * e1 = z/h^5 (crackle, and the 4th and 5th derivatives of a). */
void orc_interpolate(double h, const double a0[3], const double j0[3],
                     const double s0[3], const double a1[3], const double j1[3],
                     const double s1[3], double c1[3], double d1[3], double e1[3])
{
    for (int k = 0; k < 3; k++) {
        double M[3][3] = {{1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0},
                          {1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0},
                          {1.0, 1.0 / 2.0, 1.0 / 6.0}};
        double r[3];
        r[0] = a1[k] - a0[k] - j0[k] * h - s0[k] * h * h / 2.0;
        r[1] = h * (j1[k] - j0[k] - s0[k] * h);
        r[2] = h * h * (s1[k] - s0[k]);
        double y[3];
        solve3(M, r, y);
        double h3 = h * h * h, h4 = h3 * h, h5 = h4 * h;
        c1[k] = (y[0] + y[1] + y[2] / 2.0) / h3;
        d1[k] = (y[1] + y[2]) / h4;
        e1[k] = y[2] / h5;
    }
}

/* --------------------------------------------------------------- time step */

/* Generalised Aarseth criterion (section 3 item 3) in the 6th-order form.
 * A particle under no force at all (every derivative exactly zero, as for a
 * lone particle) gives A1 = A4 = 0: the ratio then carries no information
 * and sets no bound (+infinity, which the quantiser maps to dt_max). */
double orc_dt_crit(double eta, const double a[3], const double j[3],
                   const double s[3], const double c[3], const double d[3],
                   const double e[3])
{
    double A1 = sqrt(norm3(a) * norm3(s)) + norm3(j);
    double A4 = sqrt(norm3(c) * norm3(e)) + norm3(d);
    if (A1 == 0.0 && A4 == 0.0)
        return INFINITY;
    return eta * cbrt(A1 / A4);
}

/* Rounding floors of the interpolated crackle, pop and a^(5), for the step
 * criterion read under rounding (section 3 item 3's criterion assumes those
 * derivatives are resolved).  Each input a0, j0, s0, a1, j1, s1 is taken to
 * carry an error of at most `noise` times its norm.  The three residuals of
 * the interpolation's system (orc_interpolate) are linear in the inputs, so
 * each residual's error is at most noise times the sum of |coefficient| x
 * |input| over its own terms:
 *   rho_1 = noise (|a1| + |a0| + h |j0| + h^2/2 |s0|)    (a1 - a0 - j0 h - s0 h^2/2)
 *   rho_2 = noise h (|j1| + |j0| + h |s0|)               (h (j1 - j0 - s0 h))
 *   rho_3 = noise h^2 (|s1| + |s0|)                      (h^2 (s1 - s0))
 * The end-of-step derivatives are linear in the residuals, (c1 h^3, d1 h^4,
 * e1 h^5) = G (R1, R2, R3); taking each residual's error as independent,
 * floor_q = sum_k |G_qk| rho_k / h^(3+q).  G is formed here column by
 * column, as the interpolation's response to a unit residual, by the same
 * elimination as orc_interpolate. */
void orc_interp_floor(double noise, double h, const double a0[3], const double j0[3],
                      const double s0[3], const double a1[3], const double j1[3],
                      const double s1[3], double floor[3])
{
    double rho[3];
    rho[0] = noise * (norm3(a1) + norm3(a0) + h * norm3(j0) + h * h / 2.0 * norm3(s0));
    rho[1] = noise * h * (norm3(j1) + norm3(j0) + h * norm3(s0));
    rho[2] = noise * h * h * (norm3(s1) + norm3(s0));
    double G[3][3];
    for (int k = 0; k < 3; k++) {
        double M[3][3] = {{1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0},
                          {1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0},
                          {1.0, 1.0 / 2.0, 1.0 / 6.0}};
        double r[3] = {0.0, 0.0, 0.0};
        r[k] = 1.0;
        double y[3];
        solve3(M, r, y);
        G[0][k] = y[0] + y[1] + y[2] / 2.0;
        G[1][k] = y[1] + y[2];
        G[2][k] = y[2];
    }
    double hk = h * h * h;
    for (int q = 0; q < 3; q++) {
        floor[q] = (fabs(G[q][0]) * rho[0] + fabs(G[q][1]) * rho[1] + fabs(G[q][2]) * rho[2]) / hk;
        hk *= h;
    }
}

/* The criterion of orc_dt_crit with |c|, |d|, |e| replaced by the parts
 * above their rounding floors, max(|c| - floor[0], 0) and so on: only
 * resolved derivatives bound the step. */
double orc_dt_crit_floored(double eta, const double a[3], const double j[3],
                           const double s[3], const double c[3], const double d[3],
                           const double e[3], const double floor[3])
{
    double nc = fmax(norm3(c) - floor[0], 0.0);
    double nd = fmax(norm3(d) - floor[1], 0.0);
    double ne = fmax(norm3(e) - floor[2], 0.0);
    double A1 = sqrt(norm3(a) * norm3(s)) + norm3(j);
    double A4 = sqrt(nc * ne) + nd;
    if (A1 == 0.0 && A4 == 0.0)
        return INFINITY;
    return eta * cbrt(A1 / A4);
}

double orc_dt_initial(double eta_s, const double a[3], const double j[3],
                      const double s[3])
{
    double na = norm3(a), nj = norm3(j), ns = norm3(s);
    /* a ratio 0/0 sets no bound; fmin takes the bound that exists */
    double t1 = (na == 0.0 && nj == 0.0) ? INFINITY : na / nj;
    double t2 = (na == 0.0 && ns == 0.0) ? INFINITY : sqrt(na / ns);
    return eta_s * fmin(t1, t2);
}

double orc_dt_quantise(double dt_crit, double dt_old, double t1, double dt_min,
                       double dt_max, int *floor_hit)
{
    double p;
    *floor_hit = 0;
    if (!(dt_crit >= dt_min)) {         /* also catches NaN */
        *floor_hit = 1;
        p = dt_min;
    } else if (isinf(dt_crit)) {        /* no bound from the criterion */
        p = dt_max;
    } else {
        int ex;
        frexp(dt_crit, &ex);            /* dt_crit = f 2^ex, 0.5 <= f < 1 */
        p = ldexp(1.0, ex - 1);         /* largest power of two <= dt_crit */
        if (p > dt_max)
            p = dt_max;
    }
    if (dt_old > 0.0 && p > dt_old) {
        double d2 = 2.0 * dt_old;
        p = (fmod(t1, d2) == 0.0) ? d2 : dt_old;
    }
    return p;
}

/* ------------------------------------------------------------- diagnostics */

/* Energy of section 3 item 6 (used in Eq. 1). */
void orc_energy(int64_t n, const double *m, const double *x, const double *v,
                double eps, double *ekin, double *epot)
{
    nsum k = {0, 0}, p = {0, 0};
    for (int64_t i = 0; i < n; i++)
        nsum_add(&k, 0.5 * m[i] * dot3(&v[3 * i], &v[3 * i]));
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++) {
            double r[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1],
                           x[3 * j + 2] - x[3 * i + 2]};
            nsum_add(&p, -m[i] * m[j] / sqrt(dot3(r, r) + eps * eps));
        }
    *ekin = nsum_value(&k);
    *epot = nsum_value(&p);
}

void orc_angmom(int64_t n, const double *m, const double *x, const double *v,
                double L[3], double *Labs)
{
    nsum s[3] = {{0, 0}, {0, 0}, {0, 0}}, sa = {0, 0};
    for (int64_t i = 0; i < n; i++) {
        const double *r = &x[3 * i], *u = &v[3 * i];
        double l[3] = {r[1] * u[2] - r[2] * u[1], r[2] * u[0] - r[0] * u[2],
                       r[0] * u[1] - r[1] * u[0]};
        for (int k = 0; k < 3; k++)
            nsum_add(&s[k], m[i] * l[k]);
        nsum_add(&sa, m[i] * norm3(l));
    }
    for (int k = 0; k < 3; k++)
        L[k] = nsum_value(&s[k]);
    *Labs = nsum_value(&sa);
}

/* -------------------------------------------------------------- integrator */

struct orc_sys {
    int64_t n;
    double eps;
    orc_params p;
    double *m, *x, *v, *a, *j, *s, *c, *t, *dt;
    double *xp, *vp, *ap, *a1, *j1, *s1;
    int32_t *act;
    int64_t floor_hits;
};

uint64_t orc_hash_index(int64_t i)
{
    /* SplitMix64 finaliser of (i + 1) * golden gamma. */
    uint64_t z = (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double *dalloc(int64_t n) { return (double *)calloc((size_t)n, sizeof(double)); }

orc_sys *orc_create(int64_t n, const double *m, const double *x,
                    const double *v, double eps, const orc_params *p)
{
    orc_sys *s = (orc_sys *)calloc(1, sizeof(orc_sys));
    s->n = n;
    s->eps = eps;
    s->p = *p;
    s->m = dalloc(n);
    s->x = dalloc(3 * n); s->v = dalloc(3 * n); s->a = dalloc(3 * n);
    s->j = dalloc(3 * n); s->s = dalloc(3 * n); s->c = dalloc(3 * n);
    s->t = dalloc(n); s->dt = dalloc(n);
    s->xp = dalloc(3 * n); s->vp = dalloc(3 * n); s->ap = dalloc(3 * n);
    s->a1 = dalloc(3 * n); s->j1 = dalloc(3 * n); s->s1 = dalloc(3 * n);
    s->act = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    memcpy(s->m, m, (size_t)n * sizeof(double));
    memcpy(s->x, x, (size_t)(3 * n) * sizeof(double));
    memcpy(s->v, v, (size_t)(3 * n) * sizeof(double));

    for (int64_t i = 0; i < n; i++)
        s->act[i] = (int32_t)i;
    /* pass 1: a and jerk need only x and v (a_j - a_i = 0 here) */
    double *zero = dalloc(3 * n);
    orc_evaluate(n, s->m, s->x, s->v, zero, eps, n, s->act, s->a, s->j, s->s1);
    /* pass 2: snap with the pass-1 accelerations */
    orc_evaluate(n, s->m, s->x, s->v, s->a, eps, n, s->act, s->a1, s->j1, s->s);
    free(zero);
    for (int64_t i = 0; i < n; i++) {
        int hit = 0;
        if (p->dt_shared > 0.0)
            s->dt[i] = p->dt_shared;
        else
            s->dt[i] = orc_dt_quantise(orc_dt_initial(p->eta_s, &s->a[3 * i],
                                                      &s->j[3 * i], &s->s[3 * i]),
                                       -1.0, 0.0, p->dt_min, p->dt_max, &hit);
        s->floor_hits += hit;
    }
    return s;
}

void orc_destroy(orc_sys *s)
{
    if (!s)
        return;
    free(s->m); free(s->x); free(s->v); free(s->a); free(s->j); free(s->s);
    free(s->c); free(s->t); free(s->dt); free(s->xp); free(s->vp); free(s->ap);
    free(s->a1); free(s->j1); free(s->s1); free(s->act);
    free(s);
}

/* Predict everything to tn, evaluate the n_act listed particles, then
 * correct them, interpolate their higher derivatives and (unless keep_dt)
 * choose their next steps. */
static void advance_active(orc_sys *s, double tn, int64_t n_act, int keep_dt)
{
    int64_t n = s->n;
    orc_predict(n, tn, s->t, s->x, s->v, s->a, s->j, s->s, s->c, s->xp, s->vp, s->ap);
    orc_evaluate(n, s->m, s->xp, s->vp, s->ap, s->eps, n_act, s->act, s->a1,
                 s->j1, s->s1);
    for (int64_t k = 0; k < n_act; k++) {
        int64_t i = s->act[k];
        double h = tn - s->t[i];
        double x1[3], v1[3], c1[3], d1[3], e1[3];
        orc_correct(h, &s->x[3 * i], &s->v[3 * i], &s->a[3 * i], &s->j[3 * i],
                    &s->s[3 * i], &s->a1[3 * k], &s->j1[3 * k], &s->s1[3 * k], x1, v1);
        orc_interpolate(h, &s->a[3 * i], &s->j[3 * i], &s->s[3 * i], &s->a1[3 * k],
                        &s->j1[3 * k], &s->s1[3 * k], c1, d1, e1);
        double fl[3] = {0.0, 0.0, 0.0};
        if (s->p.step_noise > 0.0)
            orc_interp_floor(s->p.step_noise, h, &s->a[3 * i], &s->j[3 * i], &s->s[3 * i],
                             &s->a1[3 * k], &s->j1[3 * k], &s->s1[3 * k], fl);
        for (int q = 0; q < 3; q++) {
            s->x[3 * i + q] = x1[q];
            s->v[3 * i + q] = v1[q];
            s->a[3 * i + q] = s->a1[3 * k + q];
            s->j[3 * i + q] = s->j1[3 * k + q];
            s->s[3 * i + q] = s->s1[3 * k + q];
            s->c[3 * i + q] = c1[q];
        }
        s->t[i] = tn;
        if (keep_dt)
            continue;
        if (s->p.dt_shared > 0.0) {
            s->dt[i] = s->p.dt_shared;
        } else {
            int hit = 0;
            double crit = s->p.step_noise > 0.0
                              ? orc_dt_crit_floored(s->p.eta, &s->a[3 * i], &s->j[3 * i],
                                                    &s->s[3 * i], c1, d1, e1, fl)
                              : orc_dt_crit(s->p.eta, &s->a[3 * i], &s->j[3 * i],
                                            &s->s[3 * i], c1, d1, e1);
            s->dt[i] = orc_dt_quantise(crit, s->dt[i], tn, s->p.dt_min, s->p.dt_max, &hit);
            s->floor_hits += hit;
        }
    }
}

/* Block time steps (section 2 names them; the scheduler picks the particles
 * whose own step ends earliest).  All times are dyadic, so t_i + dt_i and the
 * equality test are exact. */
int64_t orc_step(orc_sys *s, double *t_out, uint64_t *set_hash)
{
    int64_t n = s->n;
    double tn = INFINITY;
    for (int64_t i = 0; i < n; i++)
        if (s->t[i] + s->dt[i] < tn)
            tn = s->t[i] + s->dt[i];
    int64_t n_act = 0;
    uint64_t h = 0;
    for (int64_t i = 0; i < n; i++)
        if (s->t[i] + s->dt[i] == tn) {
            s->act[n_act++] = (int32_t)i;
            h += orc_hash_index(i);
        }
    advance_active(s, tn, n_act, 0);
    if (t_out)
        *t_out = tn;
    if (set_hash)
        *set_hash = h;
    return n_act;
}

int64_t orc_run_until(orc_sys *s, double t_end, int64_t log_cap, double *log_t,
                      int64_t *log_n, uint64_t *log_hash)
{
    int64_t steps = 0;
    for (;;) {
        double tmin = INFINITY;
        for (int64_t i = 0; i < s->n; i++)
            if (s->t[i] < tmin)
                tmin = s->t[i];
        if (tmin >= t_end)
            break;
        double tn;
        uint64_t h;
        int64_t na = orc_step(s, &tn, &h);
        if (steps < log_cap) {
            log_t[steps] = tn;
            log_n[steps] = na;
            log_hash[steps] = h;
        }
        steps++;
    }
    return steps;
}

int64_t orc_replay(orc_sys *s, int64_t n_steps, const double *t_next,
                   const int64_t *act_offsets, const int32_t *act_idx)
{
    for (int64_t k = 0; k < n_steps; k++) {
        int64_t na = act_offsets[k + 1] - act_offsets[k];
        memcpy(s->act, &act_idx[act_offsets[k]], (size_t)na * sizeof(int32_t));
        double tn = t_next[k];
        advance_active(s, tn, na, 1);
    }
    return n_steps;
}

void orc_get_state(const orc_sys *s, double *x, double *v, double *a,
                   double *j, double *sn, double *c, double *t, double *dt)
{
    size_t b3 = (size_t)(3 * s->n) * sizeof(double), b1 = (size_t)s->n * sizeof(double);
    if (x) memcpy(x, s->x, b3);
    if (v) memcpy(v, s->v, b3);
    if (a) memcpy(a, s->a, b3);
    if (j) memcpy(j, s->j, b3);
    if (sn) memcpy(sn, s->s, b3);
    if (c) memcpy(c, s->c, b3);
    if (t) memcpy(t, s->t, b1);
    if (dt) memcpy(dt, s->dt, b1);
}

void orc_set_state(orc_sys *s, const double *x, const double *v,
                   const double *a, const double *j, const double *sn,
                   const double *c, const double *t, const double *dt)
{
    size_t b3 = (size_t)(3 * s->n) * sizeof(double), b1 = (size_t)s->n * sizeof(double);
    if (x) memcpy(s->x, x, b3);
    if (v) memcpy(s->v, v, b3);
    if (a) memcpy(s->a, a, b3);
    if (j) memcpy(s->j, j, b3);
    if (sn) memcpy(s->s, sn, b3);
    if (c) memcpy(s->c, c, b3);
    if (t) memcpy(s->t, t, b1);
    if (dt) memcpy(s->dt, dt, b1);
}

int64_t orc_floor_hits(const orc_sys *s) { return s->floor_hits; }
