// Corrector stage and time-step selection (paper, section 3 and section 3
// item 3), one thread per active particle, FP64:
//   * 6th-order Hermite corrector (the two-point quadrature with a, a', a''
//     at both ends, exact for a(t) of degree <= 5), v first, then x;
//   * crackle, pop and the 5th derivative of a at the end of the step from
//     the quintic through (a, jerk, snap) at both ends, in closed form;
//   * new block step from the generalised Aarseth criterion
//     eta (A1 / A4)^(1/3), A_k = sqrt(|a^(k-1)| |a^(k+1)|) + |a^(k)|,
//     rounded down to a power of two, clamped to [dt_min, dt_max], at most
//     doubled, and doubled only where t1 is a multiple of the doubled step.
#include "nb_correct.cuh"
#include "nb_device.cuh"
#include "nb_internal.cuh"

namespace {

using nbk::initial_dt;
using nbk::quantise;

struct CorrectArgs {
    double *st;
    double *t;
    double *dt;
    const int32_t *act;
    const double *anew;  // [9][ostride]
    int ostride;
    int n_act;
    int n;
    double t1, eta, dt_min, dt_max, dt_shared, noise;
    nb_ctl *ctl;
};

__global__ void __launch_bounds__(128) correct_kernel(CorrectArgs a)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n_act)
        return;
    double f[9];
#pragma unroll
    for (int q = 0; q < 9; ++q)
        f[q] = a.anew[q * (size_t)a.ostride + k];
    nbk::correct_particle_fp64(a.st, a.t, a.dt, static_cast<size_t>(a.n), a.act[k], a.t1, f, a.eta,
                               a.dt_min, a.dt_max, a.dt_shared, a.ctl, a.noise);
}

// Start-up (nb_init): pass 0 stores a and jerk of the first evaluation (made
// with a_j = 0); pass 1 stores the snap of the second evaluation and the
// starting steps eta_s min(|a|/|j|, sqrt(|a|/|s|)).
__global__ void init_state_kernel(double *st, double *dt, const double *anew, int n, int pass,
                                  double eta_s, double dt_min, double dt_max, double dt_shared,
                                  nb_ctl *ctl)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const size_t N = static_cast<size_t>(n);
    if (pass == 0) {
        for (int d = 0; d < 3; ++d) {
            st[(F_A * 3 + d) * N + i] = anew[(0 + d) * N + i];
            st[(F_J * 3 + d) * N + i] = anew[(3 + d) * N + i];
        }
        return;
    }
    double na = 0, nj = 0, ns = 0;
    bool finite = true;
    for (int d = 0; d < 3; ++d) {
        const double a = st[(F_A * 3 + d) * N + i], j = st[(F_J * 3 + d) * N + i];
        const double s = anew[(6 + d) * N + i];
        st[(F_S * 3 + d) * N + i] = s;
        st[(F_C * 3 + d) * N + i] = 0.0;
        na = fma(a, a, na);
        nj = fma(j, j, nj);
        ns = fma(s, s, ns);
        finite = finite && isfinite(a) && isfinite(j) && isfinite(s);
    }
    bool hit = false;
    double d0;
    if (dt_shared > 0.0) {
        d0 = dt_shared;
    } else {
        d0 = quantise(initial_dt(sqrt(na), nj, ns, eta_s), -1.0, 0.0, dt_min, dt_max, &hit);
    }
    dt[i] = d0;
    if (hit)
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->floor_hits), 1ull);
    if (!finite)
        atomicOr(&ctl->err, NB_ERR_NONFINITE);
}

// [3][ostride] component rows of anew starting at q0 -> [n_act][3] rows.
__global__ void transpose_kernel(const double *anew, int ostride, int n_act, int q0, double *dst)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * n_act)
        return;
    const int k = e / 3, d = e - 3 * k;
    dst[e] = anew[(q0 + d) * (size_t)ostride + k];
}

// State layout conversions: [n][3] rows (the C-ABI's vector layout) <->
// three component rows of the structure-of-arrays state.
__global__ void rows_to_soa_kernel(const double *rows, double *soa, int n)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * n)
        return;
    const int i = e / 3, d = e - 3 * i;
    soa[static_cast<size_t>(d) * n + i] = rows[e];
}

__global__ void soa_to_rows_kernel(const double *soa, double *rows, int n)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * n)
        return;
    const int i = e / 3, d = e - 3 * i;
    rows[e] = soa[static_cast<size_t>(d) * n + i];
}

}  // namespace

cudaError_t nb_launch_rows_to_soa(nb_ctx *c, const double *rows, int field)
{
    const int n = static_cast<int>(c->n);
    rows_to_soa_kernel<<<(3 * n + 255) / 256, 256, 0, c->stream>>>(
        rows, c->st + static_cast<size_t>(field) * 3 * n, n);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t nb_launch_soa_to_rows(nb_ctx *c, int field, double *rows)
{
    const int n = static_cast<int>(c->n);
    soa_to_rows_kernel<<<(3 * n + 255) / 256, 256, 0, c->stream>>>(
        c->st + static_cast<size_t>(field) * 3 * n, rows, n);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t nb_launch_correct(nb_ctx *c, double t1, int n_act)
{
    if (n_act <= 0)
        return cudaSuccess;
    CorrectArgs a;
    a.st = c->st;
    a.t = c->t;
    a.dt = c->dt;
    a.act = c->act;
    a.anew = c->anew;
    a.ostride = static_cast<int>(c->n);
    a.n_act = n_act;
    a.n = static_cast<int>(c->n);
    a.t1 = t1;
    a.eta = c->cfg.eta;
    a.noise = c->cfg.step_noise;
    a.dt_min = c->cfg.dt_min;
    a.dt_max = c->cfg.dt_max;
    a.dt_shared = c->cfg.dt_shared;
    a.ctl = c->ctl;
    correct_kernel<<<(n_act + 127) / 128, 128, 0, c->stream>>>(a);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t nb_launch_init_state(nb_ctx *c, int pass)
{
    const int n = static_cast<int>(c->n);
    init_state_kernel<<<(n + 127) / 128, 128, 0, c->stream>>>(c->st, c->dt, c->anew, n, pass,
                                                               c->cfg.eta_s, c->cfg.dt_min,
                                                               c->cfg.dt_max, c->cfg.dt_shared, c->ctl);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t nb_launch_transpose_out(nb_ctx *c, int n_act, int q0, double *dst)
{
    if (n_act <= 0)
        return cudaSuccess;
    const int total = 3 * n_act;
    transpose_kernel<<<(total + 255) / 256, 256, 0, c->stream>>>(c->anew, static_cast<int>(c->n), n_act,
                                                                 q0, dst);
    c->launches += 1;
    return cudaGetLastError();
}
