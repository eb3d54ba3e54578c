/*
 * libnb -- GB300 (sm_103a) direct N-body hot path: the 6th-order Hermite
 * predictor / evaluation / corrector with power-of-two block time steps.
 *
 * The operations follow the paper's statement of the method (Goz et al.,
 * "Direct N-body code on low-power embedded ARM GPUs", arXiv:1901.08532):
 *   - section 2: the device is fed coordinates, velocities and masses and
 *     returns forces; block time steps with a high-order Hermite scheme;
 *   - section 3, opening paragraph: predictor, evaluation (acceleration,
 *     jerk, snap) and corrector stages of the 6th-order Hermite integrator;
 *   - section 3 item 3: time step by the generalised Aarseth criterion,
 *     energy and angular momentum evaluated on the device;
 *   - section 3 item 4 (steps i-iv): the evaluation kernel, j-particles
 *     cached in on-chip memory, partial sums in registers, self term
 *     excluded;
 *   - section 3 item 6 and Eq. 1: precision choice and the energy error.
 *
 * Conventions for every entry point
 *   - Return value: NB_OK (0) or a negative nb_status.  A context whose call
 *     returned NB_ECUDA must only be passed to nb_last_error and nb_free.
 *   - Host arrays passed in are read (or written) during the call only; the
 *     caller keeps ownership.  Vectors are [n][3] row-major doubles.
 *   - Device pointers passed in are borrowed for the call only and must be
 *     device memory of the context's device.
 *   - The context owns all of its device memory (allocated in nb_init,
 *     released in nb_free) and runs all work on the stream given in
 *     nb_config.stream (a cudaStream_t; NULL = the legacy default stream).
 *     Entry points that return host data synchronise that stream.
 *   - Softened gravity with G = 1: pair term from particle j on particle i
 *     with r = x_j - x_i, R = |r|^2 + eps^2, A = m_j r / R^(3/2); jerk and
 *     snap are its first and second time derivatives.  eps > 0 is required,
 *     which makes the i = j term exactly zero.
 *   - Times are double; block steps are powers of two, so every time the
 *     library produces is a dyadic rational computed exactly.
 */
#ifndef NB_H
#define NB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NB_VERSION 1

typedef struct nb_ctx nb_ctx;

typedef enum {
    NB_OK = 0,
    NB_EINVAL = -1,     /* bad argument; message in nb_last_error        */
    NB_ECUDA = -2,      /* CUDA error; the context is no longer usable   */
    NB_ENOMEM = -3,     /* device or host allocation failed              */
    NB_ENONFINITE = -4, /* non-finite input, or a non-finite result       */
    NB_ETIMEOUT = -5,   /* a bounded device-side wait gave up             */
    NB_ESTATE = -6      /* call out of order (e.g. correct before eval)   */
} nb_status;

/* Arithmetic of the evaluation step (section 3 item 6).  Prediction,
 * correction, time steps and energy are FP64 in every mode, for contexts
 * (nb_init) and ensembles, except the ensemble-only NB_MIXED32. */
typedef enum {
    NB_FP64 = 0,  /* every operation of the pair sum in IEEE double          */
    NB_MIXED = 1, /* FP64 positions and accumulation; pair differences
                     rounded to FP32 (positions as hi + lo FP32 pairs), FP32
                     pair arithmetic with R^(-1/2) and 1/R from the special-
                     function unit, FP32 sums within a j-tile folded into a
                     compensated (TwoSum) accumulator                       */
    NB_SP = 2,    /* single precision control (section 3 item 6): as NB_MIXED
                     but positions rounded to FP32 (no lo part), so pair
                     differences carry the rounding of the positions; not
                     available for ensembles                                 */
    NB_EX = 3,    /* extended precision (section 3 item 6): every predicted
                     position, velocity, acceleration and mass held as a
                     double word hi + lo of FP32 numbers (about 48 mantissa
                     bits, FP32 exponent range) and the whole pair term
                     computed in double-word arithmetic from FP32
                     operations; per-tile sums added in FP64              */
    NB_MIXED32 = 4 /* ensembles only: the NB_MIXED pair arithmetic with the
                     predictor, the corrector's increments and the step
                     criterion in FP32, from an FP32 copy of the state (x
                     and v as double words); the increments are added to
                     the FP64 state.  Faster per block step than NB_MIXED,
                     not the form in which prediction and correction stay
                     FP64                                                  */
} nb_precision;

/* Shape of the evaluation launch.  0 in any field means "choose
 * automatically". */
typedef struct {
    int32_t ki;       /* i-particles per thread: FP64 1, 2 or 4; mixed and
                         SP 1, 2 or 3 (3 with junroll 4); EX 1               */
    int32_t threads;  /* threads per block: 32..512, multiple of 32 (EX:
                         at most 128)                                         */
    int32_t jtile;    /* j-particles per shared-memory stage: multiple of lanes */
    int32_t lanes;    /* threads sharing one i (j split inside a warp): 1..32  */
    int32_t split;    /* blocks sharing one i-tile (j split across blocks)     */
    int32_t junroll;  /* mixed path: j per inner iteration, 2 or 4; EX: 2
                         (two j in the lanes of packed f32x2 operations) or 1
                         (scalar FP32 operations)                             */
} nb_tiles;

typedef struct {
    int32_t precision; /* nb_precision                                        */
    double eta;        /* Aarseth accuracy parameter (0.4)                    */
    double eta_s;      /* starting-step parameter (0.01)                      */
    double dt_min;     /* smallest block step (2^-20), a power of two         */
    double dt_max;     /* largest block step (2^-3), a power of two           */
    double dt_shared;  /* 0: block steps; > 0: every particle uses this fixed
                          power-of-two step (the paper's shared step, sec. 3
                          item 3)                                             */
    nb_tiles tiles;    /* evaluation launch shape (0 = automatic)             */
    int32_t start_forces; /* 1: nb_init computes the starting a, jerk, snap and
                          steps; 0: they start at zero with dt = dt_max and
                          the caller supplies them with nb_set_state
                          (checkpoint resume, benchmarks)                     */
    void *stream;      /* cudaStream_t for all work; NULL = legacy default    */
    int32_t device_steps; /* 1: nb_run_until and nb_run_diag run block steps
                          whose active set holds at most 128 particles inside
                          one cooperative launch (device-resident scheduling,
                          evaluation and correction; larger steps return to
                          the host-driven path, and after a launch that took
                          no step the host tries again only after 1, 3, 7 ...
                          host steps); 0: every step host-driven            */
    double step_noise;  /* 0: the generalised Aarseth criterion as is.  > 0:
                          the relative rounding level of the evaluated a,
                          jerk and snap (about 4e-7 = 2^-21 for NB_MIXED,
                          the error of m q q^2 from its two hardware
                          estimates); the parts
                          of the interpolated crackle, pop and a^(5) below
                          their rounding floor (the residuals' rounding
                          divided by h^3 .. h^5) are discounted before the
                          criterion.  For mixed contexts and ensembles,
                          whose FP32 rounding otherwise drives close pairs
                          to dt_min (ensembles use it as well).  [0, 1e-3] */
} nb_config;

/* Fill cfg with the defaults listed above (FP64, automatic tiles,
 * start_forces = 1, device_steps = 1, step_noise = 0). */
void nb_config_default(nb_config *cfg);

/* Create a context on the current CUDA device for n particles with masses
 * m[n], positions x[n][3] and velocities v[n][3] (host arrays, copied) and
 * softening eps > 0: the inputs the paper's device receives (section 2:
 * the host feeds the device coordinates, velocities and masses, and the
 * device computes the forces).  The start-up below is
 * the initialisation of the 6th-order Hermite scheme of section 3 (opening
 * paragraph), which needs a, jerk and snap before the first predictor.  Computes the starting acceleration and jerk (one
 * evaluation pass with a_j = 0), then the snap (a second pass using those
 * accelerations), sets crackle to zero, t_i = 0 and the starting steps
 * (eta_s * min(|a|/|j|, sqrt(|a|/|s|)), rounded down to a power of two and
 * clamped to [dt_min, dt_max]; a ratio 0/0, as for a particle under no force,
 * sets no bound, so such a particle starts at dt_max).
 * Errors: NB_EINVAL (n < 1, n > 2^29, eps <= 0, bad config), NB_ENONFINITE
 * (non-finite m, x or v, or m < 0), NB_ENOMEM, NB_ECUDA.  *out is NULL on error. */
nb_status nb_init(nb_ctx **out, int64_t n, const double *m, const double *x,
                  const double *v, double eps, const nb_config *cfg);

/* Predictor (section 3): Taylor-expand x, v and a of EVERY particle from its
 * own time t_i to t through crackle, into the evaluation buffer.  Does not
 * change the integrator state.  Errors: NB_EINVAL (non-finite t). */
nb_status nb_predict(nb_ctx *ctx, double t);

/* Read back the evaluation buffer written by the last nb_predict: predicted
 * positions, velocities and accelerations ([n][3] host arrays; NULL skips).
 * NB_FP64 contexts return the FP64 values; NB_MIXED and NB_SP contexts
 * return the FP32 values the packed FP32 kernel uses (position = hi + lo,
 * evaluated in FP64; lo = 0 for NB_SP); NB_EX contexts return hi + lo of
 * every double word.
 * Errors: NB_ESTATE (no prediction yet). */
nb_status nb_get_predicted(nb_ctx *ctx, double *xp, double *vp, double *ap);

/* Evaluation (section 3 item 4): acceleration, jerk and snap of the n_act
 * particles listed in active[] (int32 indices in [0, n); NULL means all n in
 * order, then n_act must equal n) against all n predicted particles from
 * the last nb_predict, self term excluded.  active is a host pointer, or a
 * device pointer when active_on_device != 0.  acc, jerk and snap receive
 * [n_act][3] doubles; they are host pointers, or device pointers when
 * out_on_device != 0; any of them may be NULL (results are then only kept
 * for nb_correct).  Indices are checked on the host when active is a host
 * pointer; device lists are trusted.
 * Errors: NB_EINVAL (n_act < 0 or > n, bad index), NB_ESTATE (no prediction yet). */
nb_status nb_evaluate(nb_ctx *ctx, const int32_t *active, int64_t n_act,
                      int active_on_device, double *acc, double *jerk,
                      double *snap, int out_on_device);

/* Block-step scheduler alone (section 2): t_next = min_i(t_i + dt_i) and the
 * active set {i : t_i + dt_i == t_next}, ascending (every particle in shared
 * mode), without predicting or evaluating.  *t_next and *n_act (may be
 * NULL) receive them; nb_get_active copies the set out.  Together with
 * nb_predict, nb_evaluate_partial, nb_set_forces and nb_correct this is
 * nb_step taken apart, for a caller that sums the evaluation over several
 * devices. */
nb_status nb_schedule(nb_ctx *ctx, double *t_next, int64_t *n_act);

/* Evaluation of the active set (as in nb_evaluate) against the predicted
 * j-particles of [j_lo, j_hi) only: one device's share of the paper's
 * multi-device evaluation (section 3 item 3: with n devices each evaluates
 * N (N/n) interactions, and the results are collected and reduced).  The
 * self term needs no special care (eps > 0 makes it exactly 0 wherever i
 * falls).  part receives the FP64 partial sums [9][n_act] (row q * n_act + k:
 * acc x, y, z, jerk x, y, z, snap x, y, z of active[k]), a device pointer
 * when part_on_device != 0, else a host pointer (the call then
 * synchronises).  The partial sums are not kept for nb_correct: add the
 * shares of all j-ranges and load the totals with nb_set_forces.  Shares
 * that cover [0, n) add up, to rounding, to nb_evaluate's sums.
 * Errors: NB_EINVAL (not 0 <= j_lo <= j_hi <= n; for NB_MIXED, NB_SP and
 * NB_EX j_lo and j_hi must be multiples of 4, or j_hi == n; as nb_evaluate),
 * NB_ESTATE (no prediction yet). */
nb_status nb_evaluate_partial(nb_ctx *ctx, const int32_t *active, int64_t n_act, int active_on_device,
                              int64_t j_lo, int64_t j_hi, double *part, int part_on_device);

/* Load the acceleration, jerk and snap of the active set (f: [9][n_act]
 * doubles in the layout of nb_evaluate_partial, device or host per
 * f_on_device) as the evaluation at the last prediction time, so that
 * nb_correct can follow.  Errors: NB_EINVAL, NB_ENONFINITE (a non-finite
 * host value), NB_ESTATE (no prediction yet). */
nb_status nb_set_forces(nb_ctx *ctx, const int32_t *active, int64_t n_act, int active_on_device,
                        const double *f, int f_on_device);

/* Condition numbers of the evaluation's sums (section 3 item 4: a, jerk and
 * snap are sums over j of pair terms A_ij, J_ij, S_ij) for the n_act
 * particles listed in active[] (as in nb_evaluate; NULL means all n):
 * kappa[q * n_act + k] = sum_j |T_ij| for T = A, J, S (q = 0, 1, 2; vector
 * norms) against the predicted j-particles of the last nb_predict.  They
 * scale the error bound of each sum (the mixed path's bound is 1e-6 kappa).
 * A diagnostic: one thread per listed particle, FP32 pair terms with
 * two-part position differences, relative accuracy about 1e-6; any
 * precision.  kappa is a host pointer (the call then synchronises) or a
 * device pointer when out_on_device != 0.  Indices are checked on the host
 * when active is a host pointer; device lists are trusted.  Does not touch
 * the context's evaluation results or active set.
 * Errors: NB_EINVAL (n_act < 0 or > n, bad index, NULL kappa), NB_ESTATE
 * (no prediction yet), NB_ECUDA. */
nb_status nb_evaluate_kappa(nb_ctx *ctx, const int32_t *active, int64_t n_act, int active_on_device,
                            double *kappa, int out_on_device);

/* Corrector (section 3) for the particles of the last nb_evaluate (or
 * nb_set_forces), whose prediction time must equal t: corrected x and v, the
 * new a/jerk/snap,
 * crackle from quintic interpolation, t_i = t and a new step (generalised
 * Aarseth criterion, section 3 item 3, which sets no bound when every
 * derivative is zero; shared step when dt_shared > 0).
 * Errors: NB_ESTATE (no matching evaluation), NB_ENONFINITE (a corrected
 * value is not finite). */
nb_status nb_correct(nb_ctx *ctx, double t);

/* One block step (section 2: individual power-of-two block time steps;
 * section 3, opening paragraph: the predictor, evaluation and corrector
 * stages, in that order), entirely on the device: t_next = min_i(t_i + dt_i),
 * the active set {i : t_i + dt_i == t_next} (ascending indices), predict all,
 * evaluate the active set, correct it.  *t_out and *n_act_out (either may
 * be NULL) receive the step's time and active count. */
nb_status nb_step(nb_ctx *ctx, double *t_out, int64_t *n_act_out);

/* Block steps (section 2; the stages of section 3, and the time-step
 * selection of section 3 item 3 after every corrector) until every particle
 * has reached t_end (a multiple of dt_max, so that all particles synchronise
 * there).  *steps_out may be NULL.
 * When log_cap > 0, the first log_cap steps are recorded in log_t[] (time)
 * and log_n[] (active count). */
nb_status nb_run_until(nb_ctx *ctx, double t_end, int64_t *steps_out,
                       int64_t log_cap, double *log_t, int64_t *log_n);

/* Integrate like nb_run_until and record a diagnostics stream on the device
 * (section 3 item 3: energy and angular momentum are computed on the device;
 * Eq. 1 defines their relative errors).  A sample is taken at the starting
 * time and at every multiple of dt_diag up to t_end, when all particles are
 * synchronised; samples stay in device memory during the run and are copied
 * to the host once at the end.
 *   dt_diag  > 0, a multiple of dt_max (dt_shared in shared mode); t_end a
 *            multiple of dt_diag; the current time must be a multiple of
 *            dt_max (true after nb_init and after any nb_run_until /
 *            nb_run_diag).
 *   cap      capacity of out in samples; samples beyond cap are computed but
 *            not returned (*n_samples still counts them).
 *   out      host array [cap][8], per sample: t, E_kin, E_pot, L_x, L_y, L_z,
 *            sum m |x cross v|, number of block steps taken so far.
 *   n_samples, steps_out  may be NULL.
 * Errors: NB_EINVAL for the conditions above, then as nb_run_until. */
nb_status nb_run_diag(nb_ctx *ctx, double t_end, double dt_diag, int64_t cap, double *out,
                      int64_t *n_samples, int64_t *steps_out);

/* Kinetic energy sum 1/2 m v^2 and softened potential
 * -sum_{i<j} m_i m_j / sqrt(r^2 + eps^2) of the current state (section 3
 * item 3 and Eq. 1); meaningful when all t_i are equal.  FP64, deterministic. */
nb_status nb_energy(nb_ctx *ctx, double *ekin, double *epot);

/* Angular momentum L = sum m x cross v (L[3]) and sum m |x cross v| (*labs,
 * may be NULL) of the current state (section 3 item 3, Eq. 1). */
nb_status nb_angmom(nb_ctx *ctx, double L[3], double *labs);

/* Copy the integrator state to host arrays ([n][3] for vectors, [n] for t
 * and dt); any pointer may be NULL to skip that field.  c is the crackle.
 * This is the state of the Hermite scheme of section 3 (positions,
 * velocities, a, jerk, snap, crackle, own time and block step, section 2).
 * In section 3 item 3 particle data crosses between host and device at
 * every shared step; here the state stays in device memory and this call
 * copies it out on request.
 * nb_get_state followed by nb_set_state on a fresh context (start_forces =
 * 0) resumes an integration bit for bit. */
nb_status nb_get_state(nb_ctx *ctx, double *x, double *v, double *a, double *j,
                       double *s, double *c, double *t, double *dt);

/* Overwrite the integrator state from host arrays (checkpoint resume of the
 * section 3 Hermite state, see nb_get_state); NULL skips a field.  Errors: NB_ENONFINITE, NB_EINVAL (dt not a power of
 * two in [dt_min, dt_max], or t_i not a multiple of dt_i). */
nb_status nb_set_state(nb_ctx *ctx, const double *x, const double *v,
                       const double *a, const double *j, const double *s,
                       const double *c, const double *t, const double *dt);

/* Indices of the last evaluated active set: up to cap entries into idx[],
 * the full count in *n_act. */
nb_status nb_get_active(nb_ctx *ctx, int32_t *idx, int64_t cap, int64_t *n_act);

/* Test hook for failure detection: kind 1 makes the first shared-memory tile
 * copy of the NEXT evaluation expect 16 bytes more than the copy delivers,
 * so that block's bounded wait (1 s of wall clock) runs out; the block
 * waits, again bounded, for its copies in flight, flags the error and
 * returns.  The evaluation then reports NB_ETIMEOUT at its next host
 * synchronisation and the context stays usable.  kind 0 clears it.  The
 * injection is one-shot. */
nb_status nb_inject_fault(nb_ctx *ctx, int32_t kind);

/* Replace the evaluation launch shape (zero fields = automatic). */
nb_status nb_set_tiles(nb_ctx *ctx, const nb_tiles *tiles);

/* The launch shape the library would use for n_act active particles under
 * the current setting (automatic fields resolved). */
nb_status nb_resolve_tiles(nb_ctx *ctx, int64_t n_act, nb_tiles *out);

/* Counters since nb_init: kernels launched by this context and pair
 * interactions evaluated (n_act * n per evaluation, self term included). */
nb_status nb_counters(nb_ctx *ctx, int64_t *launches, double *interactions);

/* ---------------------------------------------------------------------------
 * Ensembles: many independent systems, each on its own block time steps,
 * advanced together in ONE persistent GPU launch (captured in a CUDA graph).
 * The paper integrates one system; this is the batched form of the same
 * predictor / evaluation / corrector cycle (sections 2-3).  Each system is
 * owned by a cluster of ctas_per_system thread blocks that pull systems from
 * a device queue, largest first.
 * ------------------------------------------------------------------------- */
typedef struct nb_ensemble nb_ensemble;

/* n_systems systems of sizes[] particles; m, x ([.][3]) and v ([.][3]) are
 * the systems' particles concatenated in order (host, copied).  Same config
 * fields as nb_init (tiles and start_forces are ignored; the starting forces
 * and steps are always computed, in one launch).  The ensemble runs on
 * cfg->stream, or on a stream of its own when that is NULL (graph capture
 * needs a stream other than the legacy default stream).  Precision NB_FP64,
 * NB_MIXED, NB_EX or NB_MIXED32 (NB_SP is rejected).  NB_FP64, NB_MIXED and
 * NB_EX use the FP64 predictor and corrector, as a context does; NB_MIXED32
 * runs the predictor (from an FP32 copy of the state, x and v as double
 * words) and the corrector's increments and step criterion in FP32.
 * Errors: NB_EINVAL, NB_ENONFINITE, NB_ENOMEM, NB_ECUDA. */
nb_status nb_ensemble_init(nb_ensemble **out, int32_t n_systems, const int64_t *sizes,
                           const double *m, const double *x, const double *v, double eps,
                           const nb_config *cfg);

/* Launch shape: thread blocks per system (1..16, one hardware cluster; above
 * 8 the non-portable cluster size, NB_EINVAL from nb_ensemble_run where the
 * device cannot co-schedule it), threads per block (64..256, multiple of 32),
 * j-tile length (multiple of 4, at most 1024).  0 in a field selects the
 * default: NB_MIXED and NB_MIXED32 4 blocks, j-tile 1024; NB_FP64 8 blocks, NB_EX 16 blocks
 * where the device co-schedules clusters of 16, else 8, j-tile 256; 128 threads. */
nb_status nb_ensemble_set_shape(nb_ensemble *e, int32_t ctas_per_system, int32_t threads,
                                int32_t jtile);

/* The launch shape in use (after defaults are resolved); NULL skips a field. */
nb_status nb_ensemble_get_shape(nb_ensemble *e, int32_t *ctas_per_system, int32_t *threads,
                                int32_t *jtile);

/* Advance every system with block steps until all of its particles reach
 * t_end (a multiple of dt_max, or of dt_shared in shared mode), in one
 * persistent launch; with use_graph != 0 the launch is captured once in a
 * CUDA graph and replayed on later calls with the same t_end.  Synchronises. */
nb_status nb_ensemble_run(nb_ensemble *e, double t_end, int use_graph);

/* State of all particles, systems concatenated as at nb_ensemble_init. */
nb_status nb_ensemble_get_state(nb_ensemble *e, double *x, double *v, double *a, double *j,
                                double *s, double *c, double *t, double *dt);

/* Block steps of each system in the last run (steps[n_systems], may be
 * NULL), pair interactions evaluated since creation, and launches issued. */
nb_status nb_ensemble_stats(nb_ensemble *e, int64_t *steps, double *interactions,
                            int64_t *launches);

/* Record every block step the ensemble takes from now on (in this and later
 * nb_ensemble_run calls), the ensemble form of nb_run_until's log (section 2
 * block steps): per step its system, time and active count, and the active
 * particles' indices within their system, ascending.  step_cap steps and
 * idx_cap indices are kept in device memory allocated here; steps beyond
 * either capacity are counted but not kept.  step_cap = idx_cap = 0 turns
 * the log off and frees it.  Calling this resets the log.
 * Errors: NB_EINVAL (a capacity < 0, step_cap > 2^32, idx_cap > 2^34),
 * NB_ENOMEM, NB_ECUDA. */
nb_status nb_ensemble_set_log(nb_ensemble *e, int64_t step_cap, int64_t idx_cap);

/* Copy the step log out.  Host arrays with room for the capacities given to
 * nb_ensemble_set_log (any may be NULL): sys[k], t[k], n_act[k] and
 * idx_off[k] per kept step k (idx_off: where step k's indices start in
 * idx[], -1 where they were not kept), the steps of each system in the
 * order taken (steps of different systems interleave).  *n_steps and *n_idx
 * (may be NULL) receive the totals recorded, kept or not. */
nb_status nb_ensemble_get_log(nb_ensemble *e, int32_t *sys, double *t, int32_t *n_act,
                              int64_t *idx_off, int32_t *idx, int64_t *n_steps, int64_t *n_idx);

/* Message for the last error of e (NULL: the last failed nb_ensemble_init
 * on this thread). */
const char *nb_ensemble_last_error(const nb_ensemble *e);

/* Release the ensemble and all of its device memory.  NULL is allowed. */
void nb_ensemble_free(nb_ensemble *e);

/* ---------------------------------------------------------------------------
 * Differentiable all-pairs evaluation (FP64, every particle active), for
 * gradients of fixed-step Hermite trajectories.  All pointers are device
 * memory; vectors are [n][3] rows, m is [n]; work runs on `stream` (a
 * cudaStream_t, NULL = legacy default) and is only enqueued.
 * ------------------------------------------------------------------------- */

/* Bytes of device workspace nb_pairs_fp64 needs for n particles (caller
 * allocated, 256-byte aligned, reusable between calls on one stream). */
size_t nb_pairs_workspace_bytes(int64_t n);

/* acc, jerk, snap [n][3] of every particle from all others (section 3
 * item 4) at the given positions x, velocities v and accelerations a.
 * Errors: NB_EINVAL (n < 1, n > 2^26, NULL pointer, eps out of range), NB_ECUDA. */
nb_status nb_pairs_fp64(int64_t n, const double *m, const double *x, const double *v,
                        const double *a, double eps, double *acc, double *jerk, double *snap,
                        void *work, void *stream);

/* Adjoint of nb_pairs_fp64: given the cotangents gacc, gjerk, gsnap [n][3]
 * of its outputs, the gradients gx, gv, ga [n][3] and gm [n] of
 * sum(gacc.acc + gjerk.jerk + gsnap.snap) with respect to x, v, a and m
 * (hand-written reverse mode of the pair terms, one pass, no atomics).
 * Errors: NB_EINVAL, NB_ECUDA. */
nb_status nb_pairs_fp64_adjoint(int64_t n, const double *m, const double *x, const double *v,
                                const double *a, double eps, const double *gacc,
                                const double *gjerk, const double *gsnap, double *gx, double *gv,
                                double *ga, double *gm, void *stream);

/* The O(N) stages of a fixed-step Hermite trajectory (section 3: predictor
 * and corrector around the evaluation; every particle on the shared step of
 * section 3 item 3) and their adjoints, for differentiating trajectories.
 * All arrays are device [n][3] doubles; work is only enqueued on `stream`;
 * h > 0 is the step (in [1e-12, 1e6]).  Errors: NB_EINVAL (n outside
 * [1, 2^40], bad h, a required pointer NULL), NB_ECUDA.
 *
 * Predictor: xp, vp, ap of every particle from x, v, a, jerk j, snap s and
 * crackle c over the step h (Taylor series through crackle). */
nb_status nb_traj_predict(int64_t n, double h, const double *x, const double *v, const double *a,
                          const double *j, const double *s, const double *c, double *xp, double *vp,
                          double *ap, void *stream);

/* Adjoint of nb_traj_predict: cotangents gxp, gvp, gap of its outputs (NULL
 * = zero) are ADDED to gx, gv, ga, gj, gs, and gc is WRITTEN (the crackle
 * enters the step only through the predictor). */
nb_status nb_traj_predict_adjoint(int64_t n, double h, const double *gxp, const double *gvp,
                                  const double *gap, double *gx, double *gv, double *ga, double *gj,
                                  double *gs, double *gc, void *stream);

/* Corrector: from the start-of-step x, v, a, j, s and the new acceleration,
 * jerk and snap A, J, S (the evaluation at the predicted state) the
 * corrected x1, v1 (two-point Hermite quadrature, v first) and the crackle
 * c1 of the quintic through (a, j, s) and (A, J, S), exactly as nb_correct
 * applies them. */
nb_status nb_traj_correct(int64_t n, double h, const double *x, const double *v, const double *a,
                          const double *j, const double *s, const double *A, const double *J,
                          const double *S, double *x1, double *v1, double *c1, void *stream);

/* Adjoint of nb_traj_correct: from the cotangents gx1, gv1, gc1 of its
 * outputs and gA_in, gJ_in, gS_in of A, J, S's other uses (any may be NULL
 * = zero) it WRITES the gradients gx, gv, ga, gj, gs of the start-of-step
 * state and the total cotangents gA, gJ, gS of the evaluation's outputs
 * (the input of nb_pairs_fp64_adjoint). */
nb_status nb_traj_correct_adjoint(int64_t n, double h, const double *gx1, const double *gv1,
                                  const double *gc1, const double *gA_in, const double *gJ_in,
                                  const double *gS_in, double *gx, double *gv, double *ga, double *gj,
                                  double *gs, double *gA, double *gJ, double *gS, void *stream);

/* Allocation-free FP64 evaluation.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory: a host
 * application that owns all GPU memory through its own pool or caching
 * allocator and forbids raw cudaMalloc (which would bypass the pool's
 * accounting); a latency-critical loop where cudaMalloc/cudaFree, which can
 * synchronise the device, are not acceptable; a deployment whose memory
 * must all be reserved before it starts.  It evaluates the same sums as
 * nb_evaluate on an NB_FP64 context and calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *   jrec    device, 5 arrays of n 16-byte records: jrec[c * n + i] holds
 *           (x, y), (z, m), (vx, vy), (vz, ax), (ay, az) for c = 0..4 (the
 *           predicted particles; 16-byte aligned)
 *   active  device, n_act int32 indices in [0, n) (not checked)
 *   out     device, [9][n_act] doubles: row q * n_act + k holds acc x, y, z,
 *           jerk x, y, z, snap x, y, z (q = 0..8) of particle active[k]
 *   split   0: automatic; > 0: that many blocks share each i-tile
 *   stream  cudaStream_t (NULL: legacy default stream); the call only
 *           enqueues work and does not synchronise
 * Scratch: the j-split partial sums and counters use a fixed 16 MiB array
 * inside the library, reserved on every GPU that loads it until the
 * library is unloaded.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Every call clears the counters it
 * uses and otherwise reuses the array, so calls whose work overlaps on the
 * GPU (other streams, other threads) race on it and must be serialised.
 * A device-side wait that times out leaves out incomplete; this entry
 * point does not report it.
 * Errors (message via nb_last_error(NULL)): NB_EINVAL (bad argument; jrec
 * not 16-byte, active not 4-byte or out not 8-byte aligned; an explicit
 * split whose partials, split * 9 * n_act doubles, exceed the scratch, or
 * that needs more than 4096 i-tiles or 65535 j-chunks), NB_ECUDA.  Every
 * NB_EINVAL is returned before any CUDA call, so nothing is launched. */
nb_status nb_evaluate_fp64_static(const void *jrec, int64_t n, const int32_t *active,
                                  int64_t n_act, double eps, int32_t split, double *out,
                                  void *stream);

/* Throughput probe of one CUDA-core pipe on the current device, the
 * measured denominator of the evaluation kernels' roofline (the pair sum of
 * section 3 item 4 runs on these pipes, not on tensor cores).  kind:
 *   0 scalar FP32 FMA, 1 packed f32x2 FMA, 2 FP64 FMA, 3 R^(-1/2) estimate,
 *   4 1/R estimate, 5 packed FMAs with one R^(-1/2) estimate per 13 (the
 *   proportion of the mixed pair term), 6 the same with the estimate in its
 *   non-flushing form, 7 packed FMAs with one R^(-1/2) and one 1/R estimate
 *   per 13, 8 packed FMAs each reading three distinct register pairs (no
 *   loop constants).
 * The probe launches blocks_per_sm blocks of `threads` threads on every SM
 * (all resident at once), each thread running `iters` iterations of
 * independent dependency chains, once to warm up and once timed; it
 * allocates and frees a few KB and synchronises.  Outputs (any may be NULL):
 * operations per clock per SM from the blocks' own cycle counts (an FMA is
 * one operation, an f32x2 FMA two), estimates per clock per SM (kinds 5-7;
 * kinds 3-4 report theirs as operations), operations per second over the
 * GPU from CUDA events, and the SM clock in MHz the launch ran at.
 * Errors: NB_EINVAL (kind outside 0..8, blocks_per_sm outside 1..32,
 * threads not a multiple of 32 in 32..1024, iters outside 1..2^24),
 * NB_ECUDA (message via nb_last_error(NULL)). */
nb_status nb_peak_probe(int32_t kind, int32_t blocks_per_sm, int32_t threads, int32_t iters,
                        double *ops_per_clk_sm, double *ops_per_s, double *est_per_clk_sm,
                        double *sm_mhz);

/* Message for the last error of ctx ("" if none).  ctx may be NULL, then
 * the message of the last failed nb_init on this thread is returned. */
const char *nb_last_error(const nb_ctx *ctx);

/* Release the context and all of its device memory.  NULL is allowed. */
void nb_free(nb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* NB_H */
