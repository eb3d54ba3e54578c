// Condition numbers of the evaluation's sums (section 3 item 4: a, jerk and
// snap of particle i are sums over j of pair terms A_ij, J_ij, S_ij): for
// each listed particle, kappa = (sum_j |A_ij|, sum_j |J_ij|, sum_j |S_ij|)
// with vector norms, against the predicted j-particles of the last
// nb_predict.  A summation whose terms each carry a few units of rounding
// errs by at most that many units of kappa, so kappa is the scale of the
// mixed path's error bound.
//
// A diagnostic, not a hot kernel: one thread per listed particle, every
// thread of a warp reading the same j (broadcast loads), FP32 pair terms on
// positions differenced in two parts (hi and lo), FP32 sums of 64 terms
// folded into FP64.  Relative accuracy about 1e-6, ample for a condition
// number.  Reads whichever evaluation buffer the context's precision keeps.
#include <string>

#include "nb_internal.cuh"

namespace {

constexpr int kKappaThreads = 128;

// j-buffer layouts: FP64 records, 13 FP32 rows (mixed / single precision),
// 20 FP32 rows of double words (EX).
enum { kLayout64 = 0, kLayout13 = 1, kLayout20 = 2 };

struct Part {
    float xh[3], xl[3], v[3], a[3], m;
};

template <int L>
__device__ __forceinline__ Part fetch(const void *jb, size_t stride, int j)
{
    Part p;
    if (L == kLayout64) {
        const double2 *r = static_cast<const double2 *>(jb);
        const double2 r0 = r[j], r1 = r[stride + j], r2 = r[2 * stride + j];
        const double2 r3 = r[3 * stride + j], r4 = r[4 * stride + j];
        const double x[3] = {r0.x, r0.y, r1.x};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            p.xh[d] = __double2float_rn(x[d]);
            p.xl[d] = __double2float_rn(x[d] - static_cast<double>(p.xh[d]));
        }
        p.m = __double2float_rn(r1.y);
        p.v[0] = __double2float_rn(r2.x);
        p.v[1] = __double2float_rn(r2.y);
        p.v[2] = __double2float_rn(r3.x);
        p.a[0] = __double2float_rn(r3.y);
        p.a[1] = __double2float_rn(r4.x);
        p.a[2] = __double2float_rn(r4.y);
    } else if (L == kLayout13) {
        const float *f = static_cast<const float *>(jb);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            p.xh[d] = f[d * stride + j];
            p.xl[d] = f[(4 + d) * stride + j];
            p.v[d] = f[(7 + d) * stride + j];
            p.a[d] = f[(10 + d) * stride + j];
        }
        p.m = f[3 * stride + j];
    } else {
        const float *f = static_cast<const float *>(jb);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            p.xh[d] = f[d * stride + j];
            p.xl[d] = f[(3 + d) * stride + j];
            p.v[d] = f[(6 + d) * stride + j] + f[(9 + d) * stride + j];
            p.a[d] = f[(12 + d) * stride + j] + f[(15 + d) * stride + j];
        }
        p.m = f[18 * stride + j] + f[19 * stride + j];
    }
    return p;
}

__device__ __forceinline__ float norm3f(float x, float y, float z) { return sqrtf(x * x + y * y + z * z); }

// With r, v, a = j - i, R = r.r + eps^2, q = R^(-1/2), mu = m_j q^3,
// alpha = (r.v) q^2, beta = (v.v + r.a) q^2 + alpha^2: A = mu r,
// J = mu (v - 3 alpha r), S = mu (a - 6 alpha u - 3 beta r) with u = v - 3 alpha r.
template <int L>
__global__ void __launch_bounds__(kKappaThreads) kappa_kernel(const void *jb, size_t stride, int n,
                                                              const int32_t *act, int n_act, float eps2,
                                                              double *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_act)
        return;
    const Part pi = fetch<L>(jb, stride, act[k]);
    double kap[3] = {0.0, 0.0, 0.0};
    float run[3] = {0.0f, 0.0f, 0.0f};
    for (int j = 0; j < n; ++j) {
        const Part pj = fetch<L>(jb, stride, j);
        float r[3], dv[3], da[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            r[d] = (pj.xh[d] - pi.xh[d]) + (pj.xl[d] - pi.xl[d]);
            dv[d] = pj.v[d] - pi.v[d];
            da[d] = pj.a[d] - pi.a[d];
        }
        const float rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const float q = rsqrtf(rr + eps2);
        const float q2 = q * q;
        const float mu = pj.m * q * q2;
        const float al = (r[0] * dv[0] + r[1] * dv[1] + r[2] * dv[2]) * q2;
        const float be = (dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2] + r[0] * da[0] + r[1] * da[1] +
                          r[2] * da[2]) * q2 + al * al;
        float u[3], w[3];
#pragma unroll
        for (int d = 0; d < 3; ++d)
            u[d] = dv[d] - 3.0f * al * r[d];
#pragma unroll
        for (int d = 0; d < 3; ++d)
            w[d] = da[d] - 6.0f * al * u[d] - 3.0f * be * r[d];
        run[0] += mu * sqrtf(rr);
        run[1] += mu * norm3f(u[0], u[1], u[2]);
        run[2] += mu * norm3f(w[0], w[1], w[2]);
        if ((j & 63) == 63) {
#pragma unroll
            for (int q3 = 0; q3 < 3; ++q3) {
                kap[q3] += run[q3];
                run[q3] = 0.0f;
            }
        }
    }
#pragma unroll
    for (int q3 = 0; q3 < 3; ++q3)
        out[static_cast<size_t>(q3) * n_act + k] = kap[q3] + run[q3];
}

}  // namespace

cudaError_t nb_launch_kappa(nb_ctx *c, const int32_t *act_dev, int n_act, double *out_dev)
{
    if (n_act <= 0)
        return cudaSuccess;
    const int grid = (n_act + kKappaThreads - 1) / kKappaThreads;
    const float eps2 = static_cast<float>(c->eps * c->eps);
    const int n = static_cast<int>(c->n);
    if (c->cfg.precision == NB_EX)
        kappa_kernel<kLayout20><<<grid, kKappaThreads, 0, c->stream>>>(
            c->jf32, static_cast<size_t>(c->npad), n, act_dev, n_act, eps2, out_dev);
    else if (nb_fp32_eval(c->cfg.precision))
        kappa_kernel<kLayout13><<<grid, kKappaThreads, 0, c->stream>>>(
            c->jf32, static_cast<size_t>(c->npad), n, act_dev, n_act, eps2, out_dev);
    else
        kappa_kernel<kLayout64><<<grid, kKappaThreads, 0, c->stream>>>(
            c->jb64, static_cast<size_t>(c->n), n, act_dev, n_act, eps2, out_dev);
    c->launches += 1;
    return cudaGetLastError();
}
