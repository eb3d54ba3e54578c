// The O(N) stages of a fixed-step 6th-order Hermite trajectory (paper,
// section 3: predictor and corrector around the evaluation, every particle
// on the shared step of section 3 item 3) and their hand-written adjoints,
// for differentiating trajectories.  Arrays are [n][3] rows of doubles
// (row-major, the layout of torch tensors), read and written once each:
// the kernels are bound by HBM bandwidth.
//
// With a fixed step h every stage is linear in its inputs, so each adjoint
// is the transposed coefficient matrix applied to the cotangents:
//   predictor  xp = x + h v + h^2/2 a + h^3/6 j + h^4/24 s + h^5/120 c
//              vp = v + h a + h^2/2 j + h^3/6 s + h^4/24 c
//              ap = a + h j + h^2/2 s + h^3/6 c
//   corrector  v1 = v + h/2 (a + A) - h^2/10 (J - j) + h^3/120 (s + S)
//              x1 = x + h/2 (v + v1) - h^2/10 (A - a) + h^3/120 (j + J)
//   crackle    c1 = (60 R1 - 36 R2 + 9 R3) / h^3 with R1 = A - a - h j -
//              h^2/2 s, R2 = h (J - j - h s), R3 = h^2 (S - s), i.e.
//              c1 = 60/h^3 (A - a) - 24/h^2 j - 36/h^2 J - 3/h s + 9/h S
// (A, J, S: the new acceleration, jerk and snap from the evaluation).
#include <algorithm>
#include <string>

#include "nb_device.cuh"
#include "nb_internal.cuh"

namespace {

constexpr int kTrajThreads = 256;

__device__ __forceinline__ double ld(const double *p, size_t e) { return p ? p[e] : 0.0; }

__global__ void __launch_bounds__(kTrajThreads) traj_predict_kernel(size_t ne, double h, const double *x,
                                                                    const double *v, const double *a,
                                                                    const double *j, const double *s,
                                                                    const double *c, double *xp,
                                                                    double *vp, double *ap)
{
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < ne;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const nbk::Taylor p = nbk::taylor(x[e], v[e], a[e], j[e], s[e], c[e], h);
        xp[e] = p.x;
        vp[e] = p.v;
        ap[e] = p.a;
    }
}

// gx += gxp, gv += h gxp + gvp, ga += h^2/2 gxp + h gvp + gap,
// gj += h^3/6 gxp + h^2/2 gvp + h gap, gs += h^4/24 gxp + h^3/6 gvp + h^2/2 gap,
// gc = h^5/120 gxp + h^4/24 gvp + h^3/6 gap.
__global__ void __launch_bounds__(kTrajThreads) traj_predict_adj_kernel(size_t ne, double h,
                                                                        const double *gxp,
                                                                        const double *gvp,
                                                                        const double *gap, double *gx,
                                                                        double *gv, double *ga, double *gj,
                                                                        double *gs, double *gc)
{
    const double h2 = h * h / 2.0, h3 = h * h * h / 6.0, h4 = h * h * h * h / 24.0;
    const double h5 = h * h * h * h * h / 120.0;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < ne;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const double X = ld(gxp, e), V = ld(gvp, e), A = ld(gap, e);
        gx[e] += X;
        gv[e] += fma(h, X, V);
        ga[e] += fma(h2, X, fma(h, V, A));
        gj[e] += fma(h3, X, fma(h2, V, h * A));
        gs[e] += fma(h4, X, fma(h3, V, h2 * A));
        gc[e] = fma(h5, X, fma(h4, V, h3 * A));
    }
}

__global__ void __launch_bounds__(kTrajThreads) traj_correct_kernel(size_t ne, double h, const double *x,
                                                                    const double *v, const double *a,
                                                                    const double *j, const double *s,
                                                                    const double *A, const double *J,
                                                                    const double *S, double *x1,
                                                                    double *v1, double *c1)
{
    const double ih = 1.0 / h;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < ne;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const nbk::Corrected r = nbk::hermite_correct(h, ih, x[e], v[e], a[e], j[e], s[e], A[e], J[e], S[e]);
        x1[e] = r.x1;
        v1[e] = r.v1;
        c1[e] = r.c1;
    }
}

// Cotangents gx1, gv1, gc1 of (x1, v1, c1) and gA_in, gJ_in, gS_in of the
// new A, J, S (their other uses) give the gradients of the old x, v, a, j,
// s (written) and the total cotangents gA, gJ, gS of the evaluation's
// outputs (written).  x1 depends on v1, so v1's total cotangent is
// gv1 + h/2 gx1.
__global__ void __launch_bounds__(kTrajThreads) traj_correct_adj_kernel(
    size_t ne, double h, const double *gx1, const double *gv1, const double *gc1, const double *gA_in,
    const double *gJ_in, const double *gS_in, double *gx, double *gv, double *ga, double *gj, double *gs,
    double *gA, double *gJ, double *gS)
{
    const double hh = 0.5 * h, h10 = h * h / 10.0, h120 = h * h * h / 120.0;
    const double k60 = 60.0 / (h * h * h), k24 = 24.0 / (h * h), k36 = 36.0 / (h * h);
    const double k3 = 3.0 / h, k9 = 9.0 / h;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < ne;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const double X = ld(gx1, e), C = ld(gc1, e);
        const double V = fma(hh, X, ld(gv1, e));
        gx[e] = X;
        gv[e] = fma(hh, X, V);
        ga[e] = fma(hh, V, fma(h10, X, -k60 * C));
        gj[e] = fma(h10, V, fma(h120, X, -k24 * C));
        gs[e] = fma(h120, V, -k3 * C);
        gA[e] = ld(gA_in, e) + fma(hh, V, fma(-h10, X, k60 * C));
        gJ[e] = ld(gJ_in, e) + fma(-h10, V, fma(h120, X, -k36 * C));
        gS[e] = ld(gS_in, e) + fma(h120, V, k9 * C);
    }
}

bool traj_args_ok(int64_t n, double h)
{
    return n >= 1 && n <= (int64_t(1) << 40) && h > 0.0 && h <= 1e6 && h >= 1e-12;
}

// Blocks for ne elements: one element per thread up to 4096 blocks, then
// grid-stride loops (enough to keep every SM of a large GPU busy).
int traj_grid(size_t ne)
{
    return static_cast<int>(std::min<size_t>((ne + kTrajThreads - 1) / kTrajThreads, 4096));
}

nb_status launched(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        nb_set_thread_error((std::string(what) + ": " + cudaGetErrorString(e)).c_str());
        return NB_ECUDA;
    }
    return NB_OK;
}

}  // namespace

extern "C" {

nb_status nb_traj_predict(int64_t n, double h, const double *x, const double *v, const double *a,
                          const double *j, const double *s, const double *c, double *xp, double *vp,
                          double *ap, void *stream)
{
    if (!traj_args_ok(n, h) || !x || !v || !a || !j || !s || !c || !xp || !vp || !ap) {
        nb_set_thread_error("nb_traj_predict: invalid argument");
        return NB_EINVAL;
    }
    const size_t ne = static_cast<size_t>(3 * n);
    traj_predict_kernel<<<traj_grid(ne), kTrajThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        ne, h, x, v, a, j, s, c, xp, vp, ap);
    return launched("nb_traj_predict");
}

nb_status nb_traj_predict_adjoint(int64_t n, double h, const double *gxp, const double *gvp,
                                  const double *gap, double *gx, double *gv, double *ga, double *gj,
                                  double *gs, double *gc, void *stream)
{
    if (!traj_args_ok(n, h) || !gx || !gv || !ga || !gj || !gs || !gc) {
        nb_set_thread_error("nb_traj_predict_adjoint: invalid argument");
        return NB_EINVAL;
    }
    const size_t ne = static_cast<size_t>(3 * n);
    traj_predict_adj_kernel<<<traj_grid(ne), kTrajThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        ne, h, gxp, gvp, gap, gx, gv, ga, gj, gs, gc);
    return launched("nb_traj_predict_adjoint");
}

nb_status nb_traj_correct(int64_t n, double h, const double *x, const double *v, const double *a,
                          const double *j, const double *s, const double *A, const double *J,
                          const double *S, double *x1, double *v1, double *c1, void *stream)
{
    if (!traj_args_ok(n, h) || !x || !v || !a || !j || !s || !A || !J || !S || !x1 || !v1 || !c1) {
        nb_set_thread_error("nb_traj_correct: invalid argument");
        return NB_EINVAL;
    }
    const size_t ne = static_cast<size_t>(3 * n);
    traj_correct_kernel<<<traj_grid(ne), kTrajThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        ne, h, x, v, a, j, s, A, J, S, x1, v1, c1);
    return launched("nb_traj_correct");
}

nb_status nb_traj_correct_adjoint(int64_t n, double h, const double *gx1, const double *gv1,
                                  const double *gc1, const double *gA_in, const double *gJ_in,
                                  const double *gS_in, double *gx, double *gv, double *ga, double *gj,
                                  double *gs, double *gA, double *gJ, double *gS, void *stream)
{
    if (!traj_args_ok(n, h) || !gx || !gv || !ga || !gj || !gs || !gA || !gJ || !gS) {
        nb_set_thread_error("nb_traj_correct_adjoint: invalid argument");
        return NB_EINVAL;
    }
    const size_t ne = static_cast<size_t>(3 * n);
    traj_correct_adj_kernel<<<traj_grid(ne), kTrajThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        ne, h, gx1, gv1, gc1, gA_in, gJ_in, gS_in, gx, gv, ga, gj, gs, gA, gJ, gS);
    return launched("nb_traj_correct_adjoint");
}

}  // extern "C"
