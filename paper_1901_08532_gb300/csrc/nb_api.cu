// C-ABI of libnb (declared in include/nb.h): argument checking, device
// memory ownership, error reporting, and the order of kernel launches for
// the predictor -> evaluation -> corrector cycle of the paper's section 3.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "nb_internal.cuh"

namespace {

thread_local std::string g_init_err;

nb_status fail(nb_ctx *c, nb_status s, const std::string &msg)
{
    c->err = msg;
    return s;
}

nb_status cuda_fail(nb_ctx *c, cudaError_t e, const char *where)
{
    c->dead = true;
    c->err = std::string(where) + ": " + cudaGetErrorString(e);
    return NB_ECUDA;
}

#define CU(c, call)                                       \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess)                            \
            return cuda_fail((c), e_, #call);             \
    } while (0)

#define CHECK_CTX(c)              \
    do {                          \
        if (!(c))                 \
            return NB_EINVAL;     \
        if ((c)->dead)            \
            return NB_ECUDA;      \
    } while (0)

bool is_pow2_double(double x)
{
    if (!(x > 0.0) || !std::isfinite(x))
        return false;
    int e;
    return std::frexp(x, &e) == 0.5;
}

bool finite_all(const double *p, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i]))
            return false;
    return true;
}

std::string check_config(const nb_config &c)
{
    if (c.precision != NB_FP64 && c.precision != NB_MIXED && c.precision != NB_SP && c.precision != NB_EX)
        return "precision must be NB_FP64, NB_MIXED, NB_SP or NB_EX";
    if (!(c.eta > 0.0) || !std::isfinite(c.eta))
        return "eta must be positive";
    if (!(c.eta_s > 0.0) || !std::isfinite(c.eta_s))
        return "eta_s must be positive";
    if (!is_pow2_double(c.dt_min) || !is_pow2_double(c.dt_max) || c.dt_min > c.dt_max)
        return "dt_min and dt_max must be powers of two with dt_min <= dt_max";
    if (c.dt_shared != 0.0 && !is_pow2_double(c.dt_shared))
        return "dt_shared must be 0 or a power of two";
    if (!(c.step_noise >= 0.0) || !(c.step_noise <= 1e-3))
        return "step_noise must be in [0, 1e-3]";
    const nb_tiles &t = c.tiles;
    if (t.ki < 0 || t.threads < 0 || t.jtile < 0 || t.lanes < 0 || t.split < 0 || t.junroll < 0)
        return "tile fields must be >= 0";
    return "";
}

std::string check_tiles(const nb_tiles &t)
{
    if (t.ki < 0 || t.ki > 4)
        return "tiles.ki must be 0, 1, 2, 3 or 4";
    if (t.threads != 0 && (t.threads < 32 || t.threads > 512 || t.threads % 32))
        return "tiles.threads must be 0 or a multiple of 32 in [32, 512]";
    if (t.lanes != 0 && (t.lanes > 32 || (t.lanes & (t.lanes - 1))))
        return "tiles.lanes must be 0 or a power of two <= 32";
    if (t.jtile < 0 || t.jtile > 4096)
        return "tiles.jtile must be in [0, 4096]";
    if (t.split < 0 || t.split > 4096)
        return "tiles.split must be in [0, 4096]";
    if (t.junroll != 0 && t.junroll != 1 && t.junroll != 2 && t.junroll != 4)
        return "tiles.junroll must be 0, 1, 2 or 4";
    return "";
}

// Read the device control block (synchronises the stream) and turn its
// error flags into a status.
nb_status sync_ctl(nb_ctx *c)
{
    CU(c, cudaMemcpyAsync(c->ctl_h, c->ctl, sizeof(nb_ctl), cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    const int err = c->ctl_h->err;
    if (err) {
        CU(c, cudaMemsetAsync(&c->ctl->err, 0, sizeof(int32_t), c->stream));
        if (err & NB_ERR_TIMEOUT) {
            if (c->tile_cnt)
                CU(c, cudaMemsetAsync(c->tile_cnt, 0, c->tile_cnt_cap * sizeof(unsigned), c->stream));
            CU(c, cudaStreamSynchronize(c->stream));
            return fail(c, NB_ETIMEOUT, "a device-side wait timed out; results are incomplete");
        }
        CU(c, cudaStreamSynchronize(c->stream));
        return fail(c, NB_ENONFINITE, "non-finite value produced on the device");
    }
    return NB_OK;
}

nb_status eval_on_device(nb_ctx *c, const int32_t *act_dev, int64_t n_act)
{
    EvalLaunch L;
    L.act = act_dev;
    L.n_act = static_cast<int>(n_act);
    L.out = c->anew;
    L.ostride = static_cast<int>(c->n);
    L.tiles = nb_auto_tiles(c, n_act, c->cfg.tiles);
    cudaError_t e = nb_launch_eval(c, L);
    if (e == cudaErrorInvalidValue)
        return fail(c, NB_EINVAL, "evaluation launch shape is not valid for this size");
    CU(c, e);
    return NB_OK;
}

// predict -> evaluate -> correct for the active list the scheduler left in
// c->act_next, which becomes c->act (the last step's set, for nb_get_active).
nb_status advance(nb_ctx *c, double tn, int64_t n_act)
{
    std::swap(c->act, c->act_next);
    CU(c, nb_launch_predict(c, tn));
    nb_status s = eval_on_device(c, c->act, n_act);
    if (s != NB_OK)
        return s;
    CU(c, nb_launch_correct(c, tn, static_cast<int>(n_act)));
    c->n_act = n_act;
    c->have_pred = false;
    c->have_eval = false;
    return NB_OK;
}

// Next block time and active set (into c->act_next); returns status.
nb_status schedule(nb_ctx *c, double *tn, int64_t *n_act)
{
    if (c->cfg.dt_shared > 0.0) {
        *tn = c->t_sys + c->cfg.dt_shared;
        *n_act = c->n;
        CU(c, nb_launch_iota(c, static_cast<int>(c->n), c->act_next));
        return NB_OK;
    }
    CU(c, nb_launch_schedule(c));
    nb_status s = sync_ctl(c);
    if (s != NB_OK)
        return s;
    unsigned long long b = c->ctl_h->tnext_bits;
    double t;
    std::memcpy(&t, &b, sizeof t);
    *tn = t;
    *n_act = c->ctl_h->n_act;
    return NB_OK;
}

// Block steps until the next block time passes t_end; steps with small
// active sets run in the device-resident stepper (one cooperative launch for
// a whole run of them), a step with a larger set runs here through the tuned
// kernels.  Shared steps make every particle active, so they always take the
// host path.  Appends to the step log (log_t, log_n, capacity log_cap) and
// counts into *steps.
nb_status integrate_to(nb_ctx *c, double t_end, int64_t log_cap, double *log_t, int64_t *log_n,
                       int64_t *steps_io)
{
    const bool device = c->cfg.device_steps != 0 && c->cfg.dt_shared == 0.0;
    int64_t steps = *steps_io;
    if (device && log_cap > steps) {
        CU(c, cudaMalloc(&c->stp_log_t, static_cast<size_t>(log_cap) * sizeof(double)));
        CU(c, cudaMalloc(&c->stp_log_n, static_cast<size_t>(log_cap) * sizeof(int64_t)));
    }
    auto release_log = [&]() {
        cudaFree(c->stp_log_t);
        cudaFree(c->stp_log_n);
        c->stp_log_t = nullptr;
        c->stp_log_n = nullptr;
    };
    nb_status s = NB_OK;
    int backoff = 0, skip = 0;  // host steps before the stepper is tried again
    for (;;) {
        if (device && skip > 0) {
            --skip;
        } else if (device) {
            int64_t ds = 0, acts = 0;
            int reason = 0, na_last = 0;
            double t_last = 0.0;
            cudaError_t e = nb_run_stepper(c, t_end, log_cap, steps, &ds, &acts, &reason, &na_last, &t_last);
            if (e != cudaSuccess) {
                release_log();
                return cuda_fail(c, e, "device-resident block steps");
            }
            if (ds > 0) {
                if (log_cap > steps) {
                    const int64_t k = std::min(ds, log_cap - steps);
                    e = cudaMemcpyAsync(log_t + steps, c->stp_log_t + steps, k * sizeof(double),
                                        cudaMemcpyDeviceToHost, c->stream);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(log_n + steps, c->stp_log_n + steps, k * sizeof(int64_t),
                                            cudaMemcpyDeviceToHost, c->stream);
                    if (e == cudaSuccess)
                        e = cudaStreamSynchronize(c->stream);
                    if (e != cudaSuccess) {
                        release_log();
                        return cuda_fail(c, e, "step log copy");
                    }
                }
                steps += ds;
                c->t_sys = t_last;
                c->n_act = na_last;
                c->interactions += static_cast<double>(acts) * static_cast<double>(c->n);
            }
            if (reason != 1)
                break;  // t_end reached, or an error flag (reported by sync_ctl)
            // the next active set is too large: a launch that took no step at
            // all doubles the number of host steps before the next attempt
            backoff = ds > 0 ? 0 : std::min(2 * backoff + 1, 255);
            skip = backoff;
        }
        double tn;
        int64_t na;
        s = schedule(c, &tn, &na);
        if (s != NB_OK)
            break;
        if (tn > t_end)
            break;
        if (na < 1) {
            s = fail(c, NB_ESTATE, "scheduler found no active particle");
            break;
        }
        s = advance(c, tn, na);
        if (s != NB_OK)
            break;
        c->t_sys = tn;
        if (steps < log_cap) {
            log_t[steps] = tn;
            log_n[steps] = na;
        }
        ++steps;
    }
    release_log();
    c->have_pred = false;
    c->have_eval = false;
    *steps_io = steps;
    return s;
}

void free_all(nb_ctx *c)
{
    cudaFree(c->m);
    cudaFree(c->st);
    cudaFree(c->t);
    cudaFree(c->dt);
    cudaFree(c->jb64);
    cudaFree(c->jf32);
    cudaFree(c->act);
    cudaFree(c->act_next);
    cudaFree(c->anew);
    cudaFree(c->stage);
    cudaFree(c->part);
    cudaFree(c->tile_cnt);
    cudaFree(c->blk);
    cudaFree(c->red);
    cudaFree(c->ctl);
    cudaFree(c->diag);
    cudaFree(c->ring);
    cudaFree(c->stp_bmin);
    cudaFree(c->stp_bcnt);
    cudaFree(c->stp_cand);
    cudaFree(c->stp_part);
    cudaFree(c->stp_out);
    if (c->stp_out_h)
        cudaFreeHost(c->stp_out_h);
    if (c->ctl_h)
        cudaFreeHost(c->ctl_h);
    if (c->diag_h)
        cudaFreeHost(c->diag_h);
}

}  // namespace

void nb_set_thread_error(const char *msg)
{
    g_init_err = msg ? msg : "";
}

extern "C" {

void nb_config_default(nb_config *cfg)
{
    if (!cfg)
        return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->precision = NB_FP64;
    cfg->eta = 0.4;
    cfg->eta_s = 0.01;
    cfg->dt_min = std::ldexp(1.0, -20);
    cfg->dt_max = std::ldexp(1.0, -3);
    cfg->dt_shared = 0.0;
    cfg->start_forces = 1;
    cfg->stream = nullptr;
    cfg->device_steps = 1;
    cfg->step_noise = 0.0;
}

nb_status nb_init(nb_ctx **out, int64_t n, const double *m, const double *x, const double *v,
                  double eps, const nb_config *cfg)
{
    if (!out) {
        g_init_err = "out must not be NULL";
        return NB_EINVAL;
    }
    *out = nullptr;
    nb_config cf;
    if (cfg)
        cf = *cfg;
    else
        nb_config_default(&cf);
    // 2^29 particles take about 190 GB in any precision; the cap keeps every
    // per-component index (3 n, and the padded rows) within 32 bits
    if (n < 1 || n > (int64_t(1) << 29)) {
        g_init_err = "n must be in [1, 2^29]";
        return NB_EINVAL;
    }
    if (!m || !x || !v) {
        g_init_err = "m, x and v must not be NULL";
        return NB_EINVAL;
    }
    std::string msg = check_config(cf);
    if (msg.empty())
        msg = check_tiles(cf.tiles);
    if (!msg.empty()) {
        g_init_err = msg;
        return NB_EINVAL;
    }
    // eps^2 must be an FP32 normal number (FP64 rsqrt estimate); the mixed
    // path also needs m / eps^3 to stay below the FP32 range.
    const bool fp32_range = nb_jrows(cf.precision) > 0;
    const double eps_min = fp32_range ? std::ldexp(1.0, -40) : std::ldexp(1.0, -60);
    if (!(eps >= eps_min) || !(eps <= 1e18)) {
        g_init_err = fp32_range ? "eps must be in [2^-40, 1e18] for FP32 pair arithmetic"
                                : "eps must be in [2^-60, 1e18]";
        return NB_EINVAL;
    }
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(m[i]) || m[i] < 0.0) {
            g_init_err = "masses must be finite and >= 0";
            return NB_ENONFINITE;
        }
    if (!finite_all(x, 3 * n) || !finite_all(v, 3 * n)) {
        g_init_err = "positions and velocities must be finite";
        return NB_ENONFINITE;
    }

    nb_ctx *c = new nb_ctx();
    c->cfg = cf;
    c->n = n;
    c->eps = eps;
    c->stream = static_cast<cudaStream_t>(cf.stream);
    auto bail = [&](nb_status s) {
        g_init_err = c->err;
        free_all(c);
        delete c;
        return s;
    };
#define CUI(call)                                          \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) {                           \
            cuda_fail(c, e_, #call);                       \
            return bail(e_ == cudaErrorMemoryAllocation ? NB_ENOMEM : NB_ECUDA); \
        }                                                  \
    } while (0)

    CUI(cudaGetDevice(&c->dev));
    CUI(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev));
    CUI(nb_eval_smem_setup());
    const size_t N = static_cast<size_t>(n);
    CUI(cudaMalloc(&c->m, N * sizeof(double)));
    CUI(cudaMalloc(&c->st, 18 * N * sizeof(double)));
    CUI(cudaMalloc(&c->t, N * sizeof(double)));
    CUI(cudaMalloc(&c->dt, N * sizeof(double)));
    c->npad = (n + 3) / 4 * 4;
    if (const int rows = nb_jrows(cf.precision)) {
        CUI(cudaMalloc(&c->jf32, rows * static_cast<size_t>(c->npad) * sizeof(float)));
        CUI(cudaMemsetAsync(c->jf32, 0, rows * static_cast<size_t>(c->npad) * sizeof(float), c->stream));
    } else
        CUI(cudaMalloc(&c->jb64, 5 * N * sizeof(double2)));
    CUI(cudaMalloc(&c->act, N * sizeof(int32_t)));
    CUI(cudaMalloc(&c->act_next, N * sizeof(int32_t)));
    CUI(cudaMalloc(&c->anew, 9 * N * sizeof(double)));
    CUI(cudaMalloc(&c->stage, 3 * N * sizeof(double)));
    CUI(cudaMalloc(&c->blk, ((N + 1023) / 1024 + 1) * sizeof(int32_t)));
    CUI(cudaMalloc(&c->ctl, sizeof(nb_ctl)));
    CUI(cudaMalloc(&c->diag, 8 * sizeof(double)));
    CUI(cudaMallocHost(&c->ctl_h, sizeof(nb_ctl)));
    CUI(cudaMallocHost(&c->diag_h, 8 * sizeof(double)));

    // upload: positions and velocities [n][3] -> component rows
    std::vector<double> h(18 * N, 0.0);
    for (size_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) {
            h[(F_X * 3 + d) * N + i] = x[3 * i + d];
            h[(F_V * 3 + d) * N + i] = v[3 * i + d];
        }
    CUI(cudaMemcpyAsync(c->st, h.data(), 18 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUI(cudaMemcpyAsync(c->m, m, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUI(cudaMemsetAsync(c->t, 0, N * sizeof(double), c->stream));
    CUI(cudaMemsetAsync(c->dt, 0, N * sizeof(double), c->stream));
    CUI(cudaMemsetAsync(c->ctl, 0, sizeof(nb_ctl), c->stream));

    // start-up: pass 0 (a_j = 0) gives a and jerk, pass 1 gives snap
    CUI(nb_launch_iota(c, static_cast<int>(n), c->act));
    if (!cf.start_forces) {
        std::vector<double> d(N, cf.dt_shared > 0.0 ? cf.dt_shared : cf.dt_max);
        CUI(cudaMemcpyAsync(c->dt, d.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CUI(cudaStreamSynchronize(c->stream));
        c->t_sys = 0.0;
        *out = c;
        return NB_OK;
    }
    for (int pass = 0; pass < 2; ++pass) {
        CUI(nb_launch_predict(c, 0.0));
        nb_status s = eval_on_device(c, c->act, n);
        if (s != NB_OK)
            return bail(s);
        CUI(nb_launch_init_state(c, pass));
    }
    nb_status s = sync_ctl(c);
    if (s != NB_OK)
        return bail(s);
    c->t_sys = 0.0;
    *out = c;
    return NB_OK;
#undef CUI
}

nb_status nb_predict(nb_ctx *c, double t)
{
    CHECK_CTX(c);
    if (!std::isfinite(t))
        return fail(c, NB_EINVAL, "t must be finite");
    CU(c, nb_launch_predict(c, t));
    c->have_pred = true;
    c->t_pred = t;
    c->have_eval = false;
    return NB_OK;
}

nb_status nb_get_predicted(nb_ctx *c, double *xp, double *vp, double *ap)
{
    CHECK_CTX(c);
    if (!c->have_pred)
        return fail(c, NB_ESTATE, "nb_get_predicted needs a prediction (nb_predict) first");
    const size_t N = static_cast<size_t>(c->n);
    if (c->cfg.precision == NB_EX) {
        const size_t P = static_cast<size_t>(c->npad);
        std::vector<float> h(20 * P);
        CU(c, cudaMemcpyAsync(h.data(), c->jf32, 20 * P * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CU(c, cudaStreamSynchronize(c->stream));
        double *dst[3] = {xp, vp, ap};
        for (size_t i = 0; i < N; ++i)
            for (int g = 0; g < 3; ++g)
                if (dst[g])
                    for (int d = 0; d < 3; ++d)
                        dst[g][3 * i + d] = (double)h[(6 * g + d) * P + i] + (double)h[(6 * g + 3 + d) * P + i];
        return NB_OK;
    }
    if (nb_fp32_eval(c->cfg.precision)) {
        const size_t P = static_cast<size_t>(c->npad);
        std::vector<float> h(13 * P);
        CU(c, cudaMemcpyAsync(h.data(), c->jf32, 13 * P * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CU(c, cudaStreamSynchronize(c->stream));
        for (size_t i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) {
                if (xp) xp[3 * i + d] = (double)h[d * P + i] + (double)h[(4 + d) * P + i];
                if (vp) vp[3 * i + d] = h[(7 + d) * P + i];
                if (ap) ap[3 * i + d] = h[(10 + d) * P + i];
            }
        return NB_OK;
    }
    std::vector<double2> h(5 * N);
    CU(c, cudaMemcpyAsync(h.data(), c->jb64, 5 * N * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < N; ++i) {
        const double2 r0 = h[i], r1 = h[N + i], r2 = h[2 * N + i], r3 = h[3 * N + i], r4 = h[4 * N + i];
        const double px[3] = {r0.x, r0.y, r1.x}, pv[3] = {r2.x, r2.y, r3.x}, pa[3] = {r3.y, r4.x, r4.y};
        for (int d = 0; d < 3; ++d) {
            if (xp) xp[3 * i + d] = px[d];
            if (vp) vp[3 * i + d] = pv[d];
            if (ap) ap[3 * i + d] = pa[d];
        }
    }
    return NB_OK;
}

nb_status nb_evaluate(nb_ctx *c, const int32_t *active, int64_t n_act, int active_on_device,
                      double *acc, double *jerk, double *snap, int out_on_device)
{
    CHECK_CTX(c);
    if (!c->have_pred)
        return fail(c, NB_ESTATE, "nb_evaluate needs a prediction (nb_predict) first");
    if (n_act < 0 || n_act > c->n)
        return fail(c, NB_EINVAL, "n_act must be in [0, n]");
    if (!active && n_act != c->n)
        return fail(c, NB_EINVAL, "active == NULL requires n_act == n");
    if (active && !active_on_device)
        for (int64_t k = 0; k < n_act; ++k)
            if (active[k] < 0 || active[k] >= c->n)
                return fail(c, NB_EINVAL, "active index out of range");
    if (n_act > 0) {
        if (!active)
            CU(c, nb_launch_iota(c, static_cast<int>(c->n), c->act));
        else if (active != c->act)
            CU(c, cudaMemcpyAsync(c->act, active, static_cast<size_t>(n_act) * sizeof(int32_t),
                                  active_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  c->stream));
        nb_status s = eval_on_device(c, c->act, n_act);
        if (s != NB_OK)
            return s;
    }
    c->n_act = n_act;
    c->have_eval = true;
    c->t_eval = c->t_pred;
    double *outs[3] = {acc, jerk, snap};
    bool host_copy = false;
    for (int q = 0; q < 3; ++q) {
        if (!outs[q] || n_act == 0)
            continue;
        if (out_on_device) {
            CU(c, nb_launch_transpose_out(c, static_cast<int>(n_act), 3 * q, outs[q]));
        } else {
            CU(c, nb_launch_transpose_out(c, static_cast<int>(n_act), 3 * q, c->stage));
            CU(c, cudaMemcpyAsync(outs[q], c->stage, static_cast<size_t>(3 * n_act) * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream));
            CU(c, cudaStreamSynchronize(c->stream));
            host_copy = true;
        }
    }
    if (host_copy)
        return sync_ctl(c);
    return NB_OK;
}

nb_status nb_schedule(nb_ctx *c, double *t_next, int64_t *n_act)
{
    CHECK_CTX(c);
    double tn;
    int64_t na;
    nb_status s = schedule(c, &tn, &na);
    if (s != NB_OK)
        return s;
    std::swap(c->act, c->act_next);
    c->n_act = na;
    c->have_eval = false;
    if (t_next)
        *t_next = tn;
    if (n_act)
        *n_act = na;
    return NB_OK;
}

// Copy an active list into c->act (checked when it is a host list).
nb_status load_active(nb_ctx *c, const int32_t *active, int64_t n_act, int active_on_device)
{
    if (n_act < 0 || n_act > c->n)
        return fail(c, NB_EINVAL, "n_act must be in [0, n]");
    if (!active && n_act != c->n)
        return fail(c, NB_EINVAL, "active == NULL requires n_act == n");
    if (active && !active_on_device)
        for (int64_t k = 0; k < n_act; ++k)
            if (active[k] < 0 || active[k] >= c->n)
                return fail(c, NB_EINVAL, "active index out of range");
    if (n_act == 0)
        return NB_OK;
    if (!active)
        CU(c, nb_launch_iota(c, static_cast<int>(c->n), c->act));
    else if (active != c->act)
        CU(c, cudaMemcpyAsync(c->act, active, static_cast<size_t>(n_act) * sizeof(int32_t),
                              active_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
    return NB_OK;
}

nb_status nb_evaluate_partial(nb_ctx *c, const int32_t *active, int64_t n_act, int active_on_device,
                              int64_t j_lo, int64_t j_hi, double *part, int part_on_device)
{
    CHECK_CTX(c);
    if (!c->have_pred)
        return fail(c, NB_ESTATE, "nb_evaluate_partial needs a prediction (nb_predict) first");
    if (!part)
        return fail(c, NB_EINVAL, "part must not be NULL");
    const bool rows = nb_jrows(c->cfg.precision) > 0;
    if (j_lo < 0 || j_hi > c->n || j_lo > j_hi)
        return fail(c, NB_EINVAL, "j-range must satisfy 0 <= j_lo <= j_hi <= n");
    if (rows && (j_lo % 4 || (j_hi % 4 && j_hi != c->n)))
        return fail(c, NB_EINVAL, "FP32-row precisions need j_lo and j_hi multiples of 4 (or j_hi == n)");
    nb_status s = load_active(c, active, n_act, active_on_device);
    if (s != NB_OK)
        return s;
    // the partial sums overwrite the context's evaluation results
    c->have_eval = false;
    if (n_act == 0)
        return NB_OK;
    EvalLaunch L;
    L.act = c->act;
    L.n_act = static_cast<int>(n_act);
    L.ostride = static_cast<int>(n_act);
    L.out = part_on_device ? part : c->anew;
    L.j0 = j_lo;
    L.j1 = rows && j_hi == c->n ? c->npad : j_hi;
    L.tiles = nb_auto_tiles(c, n_act, c->cfg.tiles, L.j1 - L.j0);
    cudaError_t e = nb_launch_eval(c, L);
    if (e == cudaErrorInvalidValue)
        return fail(c, NB_EINVAL, "evaluation launch shape is not valid for this size");
    CU(c, e);
    if (!part_on_device) {
        CU(c, cudaMemcpyAsync(part, c->anew, static_cast<size_t>(9 * n_act) * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
        return sync_ctl(c);
    }
    return NB_OK;
}

nb_status nb_set_forces(nb_ctx *c, const int32_t *active, int64_t n_act, int active_on_device,
                        const double *f, int f_on_device)
{
    CHECK_CTX(c);
    if (!c->have_pred)
        return fail(c, NB_ESTATE, "nb_set_forces needs a prediction (nb_predict) first");
    if (!f && n_act > 0)
        return fail(c, NB_EINVAL, "f must not be NULL");
    if (f && !f_on_device && !finite_all(f, 9 * n_act))
        return fail(c, NB_ENONFINITE, "forces must be finite");
    nb_status s = load_active(c, active, n_act, active_on_device);
    if (s != NB_OK)
        return s;
    if (n_act > 0)
        CU(c, cudaMemcpy2DAsync(c->anew, static_cast<size_t>(c->n) * sizeof(double), f,
                                static_cast<size_t>(n_act) * sizeof(double),
                                static_cast<size_t>(n_act) * sizeof(double), 9,
                                f_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    c->n_act = n_act;
    c->have_eval = true;
    c->t_eval = c->t_pred;
    return NB_OK;
}

nb_status nb_evaluate_kappa(nb_ctx *c, const int32_t *active, int64_t n_act, int active_on_device,
                            double *kappa, int out_on_device)
{
    CHECK_CTX(c);
    if (!c->have_pred)
        return fail(c, NB_ESTATE, "nb_evaluate_kappa needs a prediction (nb_predict) first");
    if (n_act < 0 || n_act > c->n)
        return fail(c, NB_EINVAL, "n_act must be in [0, n]");
    if (!active && n_act != c->n)
        return fail(c, NB_EINVAL, "active == NULL requires n_act == n");
    if (!kappa && n_act > 0)
        return fail(c, NB_EINVAL, "kappa must not be NULL");
    if (active && !active_on_device)
        for (int64_t k = 0; k < n_act; ++k)
            if (active[k] < 0 || active[k] >= c->n)
                return fail(c, NB_EINVAL, "active index out of range");
    if (n_act == 0)
        return NB_OK;
    // stream-ordered scratch for a host (or implied) active list and for
    // results bound for the host; the context's own buffers stay untouched
    const bool own_act = !(active && active_on_device);
    const size_t act_bytes = own_act ? (static_cast<size_t>(n_act) * sizeof(int32_t) + 15) / 16 * 16 : 0;
    const size_t out_bytes = out_on_device ? 0 : static_cast<size_t>(3 * n_act) * sizeof(double);
    struct Scratch {  // released on every return path, in stream order
        void *p = nullptr;
        cudaStream_t s = nullptr;
        ~Scratch()
        {
            if (p)
                cudaFreeAsync(p, s);
        }
    } tmp;
    tmp.s = c->stream;
    if (act_bytes + out_bytes > 0)
        CU(c, cudaMallocAsync(&tmp.p, act_bytes + out_bytes, c->stream));
    const int32_t *act_d = active;
    if (own_act) {
        int32_t *a = static_cast<int32_t *>(tmp.p);
        if (active)
            CU(c, cudaMemcpyAsync(a, active, static_cast<size_t>(n_act) * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, c->stream));
        else
            CU(c, nb_launch_iota(c, static_cast<int>(c->n), a));
        act_d = a;
    }
    double *out_d = out_on_device ? kappa : reinterpret_cast<double *>(static_cast<char *>(tmp.p) + act_bytes);
    CU(c, nb_launch_kappa(c, act_d, static_cast<int>(n_act), out_d));
    if (!out_on_device) {
        CU(c, cudaMemcpyAsync(kappa, out_d, out_bytes, cudaMemcpyDeviceToHost, c->stream));
        CU(c, cudaStreamSynchronize(c->stream));
    }
    return NB_OK;
}

nb_status nb_correct(nb_ctx *c, double t)
{
    CHECK_CTX(c);
    if (!c->have_eval || c->t_eval != t)
        return fail(c, NB_ESTATE, "nb_correct(t) needs an evaluation of a prediction at the same t");
    CU(c, nb_launch_correct(c, t, static_cast<int>(c->n_act)));
    c->have_eval = false;
    c->have_pred = false;
    if (c->n_act == c->n)
        c->t_sys = t;
    return NB_OK;
}

nb_status nb_step(nb_ctx *c, double *t_out, int64_t *n_act_out)
{
    CHECK_CTX(c);
    double tn;
    int64_t na;
    nb_status s = schedule(c, &tn, &na);
    if (s != NB_OK)
        return s;
    if (na < 1)
        return fail(c, NB_ESTATE, "scheduler found no active particle");
    s = advance(c, tn, na);
    if (s != NB_OK)
        return s;
    c->t_sys = tn;
    if (t_out)
        *t_out = tn;
    if (n_act_out)
        *n_act_out = na;
    return NB_OK;
}

nb_status nb_run_until(nb_ctx *c, double t_end, int64_t *steps_out, int64_t log_cap, double *log_t,
                       int64_t *log_n)
{
    CHECK_CTX(c);
    if (!std::isfinite(t_end))
        return fail(c, NB_EINVAL, "t_end must be finite");
    if (std::fmod(t_end, c->cfg.dt_shared > 0.0 ? c->cfg.dt_shared : c->cfg.dt_max) != 0.0)
        return fail(c, NB_EINVAL, "t_end must be a multiple of dt_max (dt_shared in shared mode)");
    if (log_cap > 0 && (!log_t || !log_n))
        return fail(c, NB_EINVAL, "log buffers must not be NULL when log_cap > 0");
    int64_t steps = 0;
    nb_status s = integrate_to(c, t_end, log_cap, log_t, log_n, &steps);
    if (s != NB_OK)
        return s;
    if (steps_out)
        *steps_out = steps;
    return sync_ctl(c);
}

nb_status nb_run_diag(nb_ctx *c, double t_end, double dt_diag, int64_t cap, double *out,
                      int64_t *n_samples, int64_t *steps_out)
{
    CHECK_CTX(c);
    const double quantum = c->cfg.dt_shared > 0.0 ? c->cfg.dt_shared : c->cfg.dt_max;
    if (!std::isfinite(t_end) || !(dt_diag > 0.0) || !std::isfinite(dt_diag))
        return fail(c, NB_EINVAL, "t_end must be finite and dt_diag > 0");
    if (std::fmod(dt_diag, quantum) != 0.0)
        return fail(c, NB_EINVAL, "dt_diag must be a multiple of dt_max (dt_shared in shared mode)");
    if (std::fmod(t_end, dt_diag) != 0.0)
        return fail(c, NB_EINVAL, "t_end must be a multiple of dt_diag");
    if (std::fmod(c->t_sys, quantum) != 0.0)
        return fail(c, NB_ESTATE, "the current time is not a synchronisation time");
    if (cap < 0 || (cap > 0 && !out))
        return fail(c, NB_EINVAL, "out must not be NULL when cap > 0");
    if (t_end < c->t_sys)
        return fail(c, NB_EINVAL, "t_end is before the current time");
    const int64_t want = static_cast<int64_t>((t_end - c->t_sys) / dt_diag) + 1;
    const int64_t keep = std::min(cap, want);
    if (keep > c->ring_cap) {
        cudaFree(c->ring);
        c->ring = nullptr;
        c->ring_cap = 0;
        CU(c, cudaMalloc(&c->ring, static_cast<size_t>(keep) * 8 * sizeof(double)));
        c->ring_cap = keep;
    }
    // Per sample: energies and angular momentum into the ring slot, the time
    // and step count into pinned host memory (known on the host).
    std::vector<double> hdr;
    hdr.reserve(static_cast<size_t>(2 * keep));
    int64_t taken = 0, steps = 0;
    auto sample = [&](double t) -> nb_status {
        if (taken < keep) {
            double *slot = c->ring + 8 * taken;
            CU(c, nb_launch_energy(c, slot + 1));
            CU(c, nb_launch_angmom(c, slot + 3));
            hdr.push_back(t);
            hdr.push_back(static_cast<double>(steps));
        }
        ++taken;
        return NB_OK;
    };
    nb_status s = sample(c->t_sys);
    if (s != NB_OK)
        return s;
    double t_next = c->t_sys + dt_diag;
    while (t_next <= t_end) {
        s = integrate_to(c, t_next, 0, nullptr, nullptr, &steps);
        if (s != NB_OK)
            return s;
        s = sync_ctl(c);  // an error flag ends the run before the sample
        if (s != NB_OK)
            return s;
        s = sample(t_next);
        if (s != NB_OK)
            return s;
        t_next += dt_diag;
    }
    s = sync_ctl(c);
    if (s != NB_OK)
        return s;
    if (keep > 0) {
        CU(c, cudaMemcpyAsync(out, c->ring, static_cast<size_t>(keep) * 8 * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
        CU(c, cudaStreamSynchronize(c->stream));
        for (int64_t k = 0; k < keep; ++k) {
            out[8 * k + 0] = hdr[2 * k];
            out[8 * k + 7] = hdr[2 * k + 1];
        }
    }
    if (n_samples)
        *n_samples = taken;
    if (steps_out)
        *steps_out = steps;
    return NB_OK;
}

nb_status nb_energy(nb_ctx *c, double *ekin, double *epot)
{
    CHECK_CTX(c);
    CU(c, nb_launch_energy(c, c->diag));
    CU(c, cudaMemcpyAsync(c->diag_h, c->diag, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    nb_status s = sync_ctl(c);
    if (s != NB_OK)
        return s;
    if (ekin)
        *ekin = c->diag_h[0];
    if (epot)
        *epot = c->diag_h[1];
    return NB_OK;
}

nb_status nb_angmom(nb_ctx *c, double L[3], double *labs)
{
    CHECK_CTX(c);
    CU(c, nb_launch_angmom(c, c->diag));
    CU(c, cudaMemcpyAsync(c->diag_h, c->diag, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    nb_status s = sync_ctl(c);
    if (s != NB_OK)
        return s;
    if (L)
        for (int d = 0; d < 3; ++d)
            L[d] = c->diag_h[d];
    if (labs)
        *labs = c->diag_h[3];
    return NB_OK;
}

nb_status nb_get_state(nb_ctx *c, double *x, double *v, double *a, double *j, double *s, double *cr,
                       double *t, double *dt)
{
    CHECK_CTX(c);
    const size_t N = static_cast<size_t>(c->n);
    double *outs[NFIELD] = {x, v, a, j, s, cr};
    for (int f = 0; f < NFIELD; ++f) {
        if (!outs[f])
            continue;
        CU(c, nb_launch_soa_to_rows(c, f, c->stage));
        CU(c, cudaMemcpyAsync(outs[f], c->stage, 3 * N * sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
    }
    if (t)
        CU(c, cudaMemcpyAsync(t, c->t, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (dt)
        CU(c, cudaMemcpyAsync(dt, c->dt, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return sync_ctl(c);
}

nb_status nb_set_state(nb_ctx *c, const double *x, const double *v, const double *a, const double *j,
                       const double *s, const double *cr, const double *t, const double *dt)
{
    CHECK_CTX(c);
    const size_t N = static_cast<size_t>(c->n);
    const double *ins[NFIELD] = {x, v, a, j, s, cr};
    for (int f = 0; f < NFIELD; ++f)
        if (ins[f] && !finite_all(ins[f], 3 * c->n))
            return fail(c, NB_ENONFINITE, "state fields must be finite");
    // t and dt are checked together on the host: dt_i a power of two in
    // [dt_min, dt_max] that divides t_i (block steps stay commensurate)
    std::vector<double> tt, dd;
    const double *tp = t, *dp = dt;
    if (!t || !dt) {
        tt.resize(N);
        dd.resize(N);
        CU(c, cudaMemcpyAsync(tt.data(), c->t, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(c, cudaMemcpyAsync(dd.data(), c->dt, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(c, cudaStreamSynchronize(c->stream));
        if (!t)
            tp = tt.data();
        if (!dt)
            dp = dd.data();
    }
    double tmin = tp[0];
    for (size_t i = 0; i < N; ++i) {
        if (!std::isfinite(tp[i]) || !is_pow2_double(dp[i]) || dp[i] < c->cfg.dt_min ||
            dp[i] > c->cfg.dt_max || std::fmod(tp[i], dp[i]) != 0.0)
            return fail(c, NB_EINVAL, "each dt_i must be a power of two in [dt_min, dt_max] dividing t_i");
        tmin = tp[i] < tmin ? tp[i] : tmin;
    }
    for (int f = 0; f < NFIELD; ++f) {
        if (!ins[f])
            continue;
        CU(c, cudaMemcpyAsync(c->stage, ins[f], 3 * N * sizeof(double), cudaMemcpyHostToDevice,
                              c->stream));
        CU(c, nb_launch_rows_to_soa(c, c->stage, f));
    }
    if (t)
        CU(c, cudaMemcpyAsync(c->t, t, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (dt)
        CU(c, cudaMemcpyAsync(c->dt, dt, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    c->t_sys = tmin;
    c->have_pred = false;
    c->have_eval = false;
    return NB_OK;
}

nb_status nb_get_active(nb_ctx *c, int32_t *idx, int64_t cap, int64_t *n_act)
{
    CHECK_CTX(c);
    if (n_act)
        *n_act = c->n_act;
    const int64_t k = cap < c->n_act ? cap : c->n_act;
    if (idx && k > 0) {
        CU(c, cudaMemcpyAsync(idx, c->act, static_cast<size_t>(k) * sizeof(int32_t),
                              cudaMemcpyDeviceToHost, c->stream));
        CU(c, cudaStreamSynchronize(c->stream));
    }
    return NB_OK;
}

nb_status nb_inject_fault(nb_ctx *c, int32_t kind)
{
    CHECK_CTX(c);
    if (kind != 0 && kind != 1)
        return fail(c, NB_EINVAL, "fault kind must be 0 (none) or 1 (stalled tile copy)");
    c->inject = kind;
    return NB_OK;
}

nb_status nb_set_tiles(nb_ctx *c, const nb_tiles *tiles)
{
    CHECK_CTX(c);
    nb_tiles t{};
    if (tiles)
        t = *tiles;
    const std::string msg = check_tiles(t);
    if (!msg.empty())
        return fail(c, NB_EINVAL, msg);
    c->cfg.tiles = t;
    return NB_OK;
}

nb_status nb_resolve_tiles(nb_ctx *c, int64_t n_act, nb_tiles *out)
{
    CHECK_CTX(c);
    if (!out || n_act < 1 || n_act > c->n)
        return fail(c, NB_EINVAL, "out must not be NULL and n_act in [1, n]");
    *out = nb_auto_tiles(c, n_act, c->cfg.tiles);
    return NB_OK;
}

nb_status nb_counters(nb_ctx *c, int64_t *launches, double *interactions)
{
    CHECK_CTX(c);
    if (launches)
        *launches = c->launches;
    if (interactions)
        *interactions = c->interactions;
    return NB_OK;
}

const char *nb_last_error(const nb_ctx *c)
{
    return c ? c->err.c_str() : g_init_err.c_str();
}

void nb_free(nb_ctx *c)
{
    if (!c)
        return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
