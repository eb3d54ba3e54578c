/*
 * FP64 CPU oracle for the 6th-order Hermite block-time-step direct N-body
 * method (Goz et al., "Direct N-body code on low-power embedded ARM GPUs",
 * section 3; the integrator itself is Nitadori & Makino 2008, New Astronomy
 * 13, 498, which the paper cites for all of its formulas).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded C99 in IEEE double
 * precision, with no blocking, fusion or reordering.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may call it; the
 * CUDA library never links it and shares no code with it.
 *
 * Array layout: vectors are [n][3] row-major doubles (x, y, z per particle).
 */
#ifndef NB_ORACLE_H
#define NB_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Softened acceleration, jerk and snap of particle i from particle j
 * (one term of the evaluation sum, section 3 item 4). */
void orc_pair(const double xi[3], const double vi[3], const double ai[3],
              const double xj[3], const double vj[3], const double aj[3],
              double mj, double eps, double acc[3], double jrk[3], double snp[3]);

/* Evaluation step (section 3, item 4 steps i-iv): for each listed i, sum the
 * pair terms over all j != i with Neumaier-compensated summation. */
void orc_evaluate(int64_t n, const double *m, const double *x, const double *v,
                  const double *a, double eps, int64_t n_act, const int32_t *act,
                  double *acc, double *jrk, double *snp);

/* Condition numbers of the evaluation sums: for each listed i, the sums over
 * j != i of |A_ij|, |J_ij| and |S_ij| (Euclidean norms of the pair terms).
 * A computed sum carries rounding errors of each term, so its error is
 * bounded relative to these sums, not to the (possibly cancelling) result. */
void orc_evaluate_kappa(int64_t n, const double *m, const double *x,
                        const double *v, const double *a, double eps,
                        int64_t n_act, const int32_t *act, double *ka,
                        double *kj, double *ks);

/* Predictor (section 3): Taylor series of x, v, a of every particle from its
 * own time t_i to t, through crackle c. */
void orc_predict(int64_t n, double t, const double *ti, const double *x,
                 const double *v, const double *a, const double *j,
                 const double *s, const double *c, double *xp, double *vp,
                 double *ap);

/* Corrector (section 3): 6th-order Hermite corrector of one particle over
 * step h; v1 first, then x1 using v1. */
void orc_correct(double h, const double x0[3], const double v0[3],
                 const double a0[3], const double j0[3], const double s0[3],
                 const double a1[3], const double j1[3], const double s1[3],
                 double x1[3], double v1[3]);

/* Quintic Hermite interpolation of a(t) on [0, h] through (a, j, s) at both
 * ends; returns the 3rd, 4th and 5th derivatives of a at the END of the step. */
void orc_interpolate(double h, const double a0[3], const double j0[3],
                     const double s0[3], const double a1[3], const double j1[3],
                     const double s1[3], double c1[3], double d1[3], double e1[3]);

/* Generalised Aarseth criterion for a 6th-order scheme (section 3 item 3):
 * eta * (A1 / A4)^(1/3), A_k = sqrt(|a^(k-1)| |a^(k+1)|) + |a^(k)|;
 * +infinity (no bound) when A1 = A4 = 0, a particle under no force. */
double orc_dt_crit(double eta, const double a[3], const double j[3],
                   const double s[3], const double c[3], const double d[3],
                   const double e[3]);

/* Rounding floors of the interpolated crackle, pop and a^(5) when every
 * input vector carries a relative error up to `noise`: the residuals'
 * error bounds rho_1..rho_3 (noise times the sum of |coefficient| x |input|
 * of each residual) propagated through the absolute values of the
 * interpolation's linear map; floor[0..2] for |c1|, |d1|, |e1|. */
void orc_interp_floor(double noise, double h, const double a0[3], const double j0[3],
                      const double s0[3], const double a1[3], const double j1[3],
                      const double s1[3], double floor[3]);

/* orc_dt_crit with |c|, |d|, |e| less their floors (at least 0). */
double orc_dt_crit_floored(double eta, const double a[3], const double j[3],
                           const double s[3], const double c[3], const double d[3],
                           const double e[3], const double floor[3]);

/* Starting step before any interpolation exists:
 * eta_s * min(|a|/|j|, sqrt(|a|/|s|)), a ratio 0/0 counting as no bound. */
double orc_dt_initial(double eta_s, const double a[3], const double j[3],
                      const double s[3]);

/* Power-of-two block step: largest 2^k <= dt_crit, clamped to
 * [dt_min, dt_max]; at most twice dt_old, and doubling only when t1 is a
 * multiple of the doubled step.  dt_old <= 0 means "no previous step".
 * *floor_hit is set to 1 when dt_crit < dt_min. */
double orc_dt_quantise(double dt_crit, double dt_old, double t1, double dt_min,
                       double dt_max, int *floor_hit);

/* Energy (section 3 item 6): kinetic sum 1/2 m v^2 and softened potential
 * -sum_{i<j} m_i m_j / sqrt(r^2 + eps^2), compensated sums. */
void orc_energy(int64_t n, const double *m, const double *x, const double *v,
                double eps, double *ekin, double *epot);

/* Angular momentum L = sum m x cross v, and sum m |x cross v| (for a
 * well-conditioned relative error). */
void orc_angmom(int64_t n, const double *m, const double *x, const double *v,
                double L[3], double *Labs);

/* --------------------------------------------------------------------------
 * Whole integrator.  The system owns copies of all arrays.
 * -------------------------------------------------------------------------- */
typedef struct orc_sys orc_sys;

typedef struct {
    double eta;      /* Aarseth accuracy parameter                */
    double eta_s;    /* starting-step parameter                   */
    double dt_min;   /* smallest allowed block step               */
    double dt_max;   /* largest allowed block step                */
    double dt_shared;/* > 0: every particle steps with this dt    */
    double step_noise;/* > 0: criterion with rounding floors of    */
                      /* this relative level (orc_interp_floor)    */
} orc_params;

/* Copies m, x, v; evaluates a, j (pass 1, a_j = 0) then s (pass 2, with
 * the pass-1 accelerations as a_j); crackle starts at 0; sets starting steps. */
orc_sys *orc_create(int64_t n, const double *m, const double *x,
                    const double *v, double eps, const orc_params *p);
void orc_destroy(orc_sys *s);

/* One block step: t_next = min(t_i + dt_i); active = {i : t_i + dt_i ==
 * t_next}; predict all, evaluate active, correct, interpolate, new dt.
 * Returns n_act; *t_out = t_next; *set_hash = order-independent hash of the
 * active set (sum over i of a 64-bit mix of i). */
int64_t orc_step(orc_sys *s, double *t_out, uint64_t *set_hash);

/* Step until every particle reaches t_end (t_end must be a multiple of
 * dt_max so that all particles synchronise there).  When log_cap > 0 the
 * first log_cap steps are recorded as (t_next, n_act, set_hash).  Returns the
 * number of block steps. */
int64_t orc_run_until(orc_sys *s, double t_end, int64_t log_cap, double *log_t,
                      int64_t *log_n, uint64_t *log_hash);

/* Replay: take the block steps given by a log of (t_next, active sets) from
 * another integrator instead of the oracle's own dt decisions.  Only the
 * state update is computed.  act_offsets has n_steps + 1 entries. */
int64_t orc_replay(orc_sys *s, int64_t n_steps, const double *t_next,
                   const int64_t *act_offsets, const int32_t *act_idx);

void orc_get_state(const orc_sys *s, double *x, double *v, double *a,
                   double *j, double *sn, double *c, double *t, double *dt);
void orc_set_state(orc_sys *s, const double *x, const double *v,
                   const double *a, const double *j, const double *sn,
                   const double *c, const double *t, const double *dt);
int64_t orc_floor_hits(const orc_sys *s);
uint64_t orc_hash_index(int64_t i);

#ifdef __cplusplus
}
#endif
#endif
