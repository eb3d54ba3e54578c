// All-pairs evaluation and its hand-written adjoint, FP64, stateless (every
// particle active), for differentiating fixed-step Hermite trajectories.
//
// Forward: the caller's rows x, v, a [n][3] and m [n] are packed into the
// evaluation records and the FP64 evaluation kernel runs with every particle
// active (paper, section 3 item 4).
//
// Adjoint: for a pair term (i <- j) with r = x_j - x_i, v = v_j - v_i,
// a = a_j - a_i, R = r.r + eps^2, q = R^(-1/2), mu = m_j q^3,
// alpha = (r.v) q^2, beta = (v.v + r.a) q^2 + alpha^2, u = v - 3 alpha r,
// w = a - 6 alpha u - 3 beta r and A = mu r, J = mu u, S = mu w, the
// cotangents (Ab, Jb, Sb) of particle i give L = Ab.A + Jb.J + Sb.S = mu Phi,
//   Phi = Pr.r + (Jb - 6 alpha Sb).v + Sb.a,
//   Pr  = Ab - 3 alpha Jb + (18 alpha^2 - 3 beta) Sb.
// With Pa = dPhi/dalpha = -3 Jb.r - 6 Sb.v + 36 alpha Sb.r and
// Pb = dPhi/dbeta = -3 Sb.r (alpha and beta held fixed in Phi):
//   dL/dr = mu [Pr + q^2 ((Pa + 2 alpha Pb) v + Pb a
//                         - (3 Phi + 2 alpha Pa + 2 (beta + alpha^2) Pb) r)]
//   dL/dv = mu [Jb - 6 alpha Sb + q^2 ((Pa + 2 alpha Pb) r + 2 Pb v)]
//   dL/da = mu [Sb + q^2 Pb r]
//   dL/dm_j = q^3 Phi,
// from dmu/dr = -3 mu q^2 r, dalpha/dr = q^2 (v - 2 alpha r),
// dalpha/dv = q^2 r, dbeta/dr = q^2 (a + 2 alpha v - 2 (beta + alpha^2) r),
// dbeta/dv = 2 q^2 (v + alpha r), dbeta/da = q^2 r.
// Particle k receives -dL/d(r, v, a) of every pair where it is i (with its
// own cotangents) and +dL/d(r, v, a) and dL/dm of every pair where it is j
// (with the other particle's cotangents).  `lanes` consecutive threads own
// k and visit every l once between them (every lanes-th l of each tile);
// their sums are combined by a fixed-order butterfly of warp shuffles, so
// no atomics are needed and the result does not depend on scheduling.  The
// lanes keep small systems from leaving most SMs idle (one thread per k
// would give 64 blocks for 8192 particles).
#include <algorithm>

#include "nb_device.cuh"
#include "nb_internal.cuh"

namespace {

constexpr int kAdjThreads = 128;
constexpr int kAdjTile = 64;

// The bracket B(g) of dL/d(r, v, a) = q^3 B(g) for a pair with unit source
// mass (mu = m_j q^3 factored out), linear in the cotangents g.
__device__ __forceinline__ void pair_bracket(const double (&r)[3], const double (&v)[3], const double (&a)[3],
                                             const double (&u)[3], const double (&w)[3], double q2, double al,
                                             double be, const double *g, double (&br)[3], double (&bv)[3],
                                             double (&ba)[3])
{
    const double *Ab = g, *Jb = g + 3, *Sb = g + 6;
    const double c18 = 18.0 * al * al - 3.0 * be;
    double phi = 0, sr = 0, sv = 0, jr = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        phi = fma(Ab[d], r[d], fma(Jb[d], u[d], fma(Sb[d], w[d], phi)));
        sr = fma(Sb[d], r[d], sr);
        sv = fma(Sb[d], v[d], sv);
        jr = fma(Jb[d], r[d], jr);
    }
    const double Pa = -3.0 * jr - 6.0 * sv + 36.0 * al * sr;
    const double Pb = -3.0 * sr;
    const double cv = fma(2.0 * al, Pb, Pa);
    const double cr = fma(3.0, phi, fma(2.0 * al, Pa, 2.0 * (be + al * al) * Pb));
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double Pr = fma(c18, Sb[d], fma(-3.0 * al, Jb[d], Ab[d]));
        br[d] = fma(q2, fma(cv, v[d], fma(Pb, a[d], -cr * r[d])), Pr);
        bv[d] = fma(q2, fma(cv, r[d], 2.0 * Pb * v[d]), fma(-6.0 * al, Sb[d], Jb[d]));
        ba[d] = fma(q2 * Pb, r[d], Sb[d]);
    }
}

// For particle k and every l: the pair (i = k, j = l) with k's cotangents and
// source mass m_l, and the pair (i = l, j = k) with l's cotangents and source
// mass m_k.  Negating r, v, a negates u, w, Phi and the bracket's
// coefficients, so the second pair's gradient with respect to x_k equals the
// first pair's form evaluated at (r, v, a) with l's cotangents; by linearity
// both roles need one bracket with g* = m_k g_l - m_l g_k, times q^3.  The mass
// gradient of m_k is -q^3 Phi(g_l).  For l = k, g* = 0 and Phi = 0 exactly.
__global__ void __launch_bounds__(kAdjThreads) adjoint_kernel(int n, int lanes, const double *__restrict__ m,
                                                              const double *__restrict__ x,
                                                              const double *__restrict__ v,
                                                              const double *__restrict__ a,
                                                              const double *__restrict__ gA,
                                                              const double *__restrict__ gJ,
                                                              const double *__restrict__ gS, double eps2,
                                                              double *__restrict__ gx, double *__restrict__ gv,
                                                              double *__restrict__ ga, double *__restrict__ gm)
{
    __shared__ double s_st[kAdjTile][10];  // x, v, a, m
    __shared__ double s_g[kAdjTile][9];    // cotangents
    const int slot = threadIdx.x / lanes, lj = threadIdx.x - slot * lanes;
    const int k = blockIdx.x * (blockDim.x / lanes) + slot;
    const bool valid = k < n;
    const int kk = valid ? k : 0;
    double xk[3], vk[3], ak[3], gk[9];
    for (int d = 0; d < 3; ++d) {
        xk[d] = x[3 * kk + d];
        vk[d] = v[3 * kk + d];
        ak[d] = a[3 * kk + d];
        gk[d] = gA[3 * kk + d];
        gk[3 + d] = gJ[3 * kk + d];
        gk[6 + d] = gS[3 * kk + d];
    }
    const double mk = m[kk];
    double ox[3] = {0, 0, 0}, ov[3] = {0, 0, 0}, oa[3] = {0, 0, 0}, om = 0.0;
    for (int l0 = 0; l0 < n; l0 += kAdjTile) {
        __syncthreads();
        for (int e = threadIdx.x; e < kAdjTile; e += blockDim.x) {
            const int l = l0 + e;
            const bool ok = l < n;
            const int ll = ok ? l : 0;
            for (int d = 0; d < 3; ++d) {
                s_st[e][d] = x[3 * ll + d];
                s_st[e][3 + d] = v[3 * ll + d];
                s_st[e][6 + d] = a[3 * ll + d];
                s_g[e][d] = ok ? gA[3 * ll + d] : 0.0;
                s_g[e][3 + d] = ok ? gJ[3 * ll + d] : 0.0;
                s_g[e][6 + d] = ok ? gS[3 * ll + d] : 0.0;
            }
            s_st[e][9] = ok ? m[ll] : 0.0;
        }
        __syncthreads();
        const int len = min(kAdjTile, n - l0);
        for (int e = lj; e < len; e += lanes) {
            double r[3], vr[3], ar[3];
            for (int d = 0; d < 3; ++d) {
                r[d] = s_st[e][d] - xk[d];
                vr[d] = s_st[e][3 + d] - vk[d];
                ar[d] = s_st[e][6 + d] - ak[d];
            }
            const double R = fma(r[0], r[0], fma(r[1], r[1], fma(r[2], r[2], eps2)));
            const double q = nbk::rsqrt_fp64(R);
            const double q2 = q * q, q3 = q * q2;
            const double al = fma(r[0], vr[0], fma(r[1], vr[1], r[2] * vr[2])) * q2;
            const double be = fma(fma(vr[0], vr[0], fma(vr[1], vr[1], vr[2] * vr[2])) +
                                      fma(r[0], ar[0], fma(r[1], ar[1], r[2] * ar[2])),
                                  q2, al * al);
            double u[3], w[3];
            for (int d = 0; d < 3; ++d) {
                u[d] = fma(-3.0 * al, r[d], vr[d]);
                w[d] = fma(-6.0 * al, u[d], fma(-3.0 * be, r[d], ar[d]));
            }
            const double ml = s_st[e][9];
            double gs[9];
            double phil = 0.0;
            for (int q9 = 0; q9 < 9; ++q9)
                gs[q9] = fma(mk, s_g[e][q9], -ml * gk[q9]);
            for (int d = 0; d < 3; ++d)
                phil = fma(s_g[e][d], r[d], fma(s_g[e][3 + d], u[d], fma(s_g[e][6 + d], w[d], phil)));
            double br[3], bv[3], ba[3];
            pair_bracket(r, vr, ar, u, w, q2, al, be, gs, br, bv, ba);
            for (int d = 0; d < 3; ++d) {
                ox[d] = fma(q3, br[d], ox[d]);
                ov[d] = fma(q3, bv[d], ov[d]);
                oa[d] = fma(q3, ba[d], oa[d]);
            }
            om = fma(-q3, phil, om);
        }
    }
    for (int off = lanes >> 1; off > 0; off >>= 1) {
        for (int d = 0; d < 3; ++d) {
            ox[d] += __shfl_xor_sync(0xffffffffu, ox[d], off);
            ov[d] += __shfl_xor_sync(0xffffffffu, ov[d], off);
            oa[d] += __shfl_xor_sync(0xffffffffu, oa[d], off);
        }
        om += __shfl_xor_sync(0xffffffffu, om, off);
    }
    if (valid && lj == 0) {
        for (int d = 0; d < 3; ++d) {
            gx[3 * k + d] = ox[d];
            gv[3 * k + d] = ov[d];
            ga[3 * k + d] = oa[d];
        }
        gm[k] = om;
    }
}

__global__ void pack_records(int n, const double *m, const double *x, const double *v, const double *a,
                             double2 *rec, int32_t *iota)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const size_t N = static_cast<size_t>(n);
    rec[i] = make_double2(x[3 * i], x[3 * i + 1]);
    rec[N + i] = make_double2(x[3 * i + 2], m[i]);
    rec[2 * N + i] = make_double2(v[3 * i], v[3 * i + 1]);
    rec[3 * N + i] = make_double2(v[3 * i + 2], a[3 * i]);
    rec[4 * N + i] = make_double2(a[3 * i + 1], a[3 * i + 2]);
    iota[i] = i;
}

__global__ void unpack_rows(int n, const double *sums, double *acc, double *jerk, double *snap)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * n)
        return;
    const int i = e / 3, d = e - 3 * i;
    const size_t N = static_cast<size_t>(n);
    acc[e] = sums[(0 + d) * N + i];
    jerk[e] = sums[(3 + d) * N + i];
    snap[e] = sums[(6 + d) * N + i];
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

// FP64 evaluation kernel entry for the stateless path (k_eval.cu).
cudaError_t nb_launch_eval_fp64_rows(const double2 *rec, int n, const int32_t *act, double *out,
                                     double eps2, nb_ctl *ctl, cudaStream_t stream, int sm_count);

extern "C" {

size_t nb_pairs_workspace_bytes(int64_t n)
{
    if (n < 1)
        return 0;
    const size_t N = static_cast<size_t>(n);
    return align256(5 * N * sizeof(double2)) + align256(N * sizeof(int32_t)) +
           align256(9 * N * sizeof(double)) + align256(sizeof(nb_ctl));
}

nb_status nb_pairs_fp64(int64_t n, const double *m, const double *x, const double *v, const double *a,
                        double eps, double *acc, double *jerk, double *snap, void *work, void *stream)
{
    if (n < 1 || n > (1LL << 26) || !m || !x || !v || !a || !acc || !jerk || !snap || !work ||
        !(eps >= 0x1p-60) || !(eps <= 1e18)) {
        nb_set_thread_error("nb_pairs_fp64: invalid argument");
        return NB_EINVAL;
    }
    const int nn = static_cast<int>(n);
    const size_t N = static_cast<size_t>(n);
    unsigned char *w = static_cast<unsigned char *>(work);
    double2 *rec = reinterpret_cast<double2 *>(w);
    int32_t *iota = reinterpret_cast<int32_t *>(w + align256(5 * N * sizeof(double2)));
    double *sums = reinterpret_cast<double *>(w + align256(5 * N * sizeof(double2)) + align256(N * sizeof(int32_t)));
    nb_ctl *ctl = reinterpret_cast<nb_ctl *>(reinterpret_cast<unsigned char *>(sums) + align256(9 * N * sizeof(double)));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctl, 0, sizeof(nb_ctl), s);
    if (e == cudaSuccess) {
        pack_records<<<(nn + 255) / 256, 256, 0, s>>>(nn, m, x, v, a, rec, iota);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = nb_launch_eval_fp64_rows(rec, nn, iota, sums, eps * eps, ctl, s, sms);
    if (e == cudaSuccess) {
        unpack_rows<<<(3 * nn + 255) / 256, 256, 0, s>>>(nn, sums, acc, jerk, snap);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        nb_set_thread_error(cudaGetErrorString(e));
        return NB_ECUDA;
    }
    return NB_OK;
}

nb_status nb_pairs_fp64_adjoint(int64_t n, const double *m, const double *x, const double *v,
                                const double *a, double eps, const double *gacc, const double *gjerk,
                                const double *gsnap, double *gx, double *gv, double *ga, double *gm,
                                void *stream)
{
    if (n < 1 || n > (1LL << 26) || !m || !x || !v || !a || !gacc || !gjerk || !gsnap || !gx || !gv ||
        !ga || !gm || !(eps >= 0x1p-60) || !(eps <= 1e18)) {
        nb_set_thread_error("nb_pairs_fp64_adjoint: invalid argument");
        return NB_EINVAL;
    }
    const int nn = static_cast<int>(n);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        nb_set_thread_error(cudaGetErrorString(e));
        return NB_ECUDA;
    }
    // lanes per particle: the fewest that give every SM at least four blocks
    int lanes = 1;
    while (lanes < 32 && (static_cast<int64_t>(nn) * lanes + kAdjThreads - 1) / kAdjThreads < 4 * sms)
        lanes *= 2;
    const int per_block = kAdjThreads / lanes;
    adjoint_kernel<<<(nn + per_block - 1) / per_block, kAdjThreads, 0, s>>>(
        nn, lanes, m, x, v, a, gacc, gjerk, gsnap, eps * eps, gx, gv, ga, gm);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        nb_set_thread_error(cudaGetErrorString(e));
        return NB_ECUDA;
    }
    return NB_OK;
}

}  // extern "C"
