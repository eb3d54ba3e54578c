// Predictor stage of the 6th-order Hermite scheme (paper, section 3): every
// particle's x, v and a are Taylor-expanded from its own time t_i to the
// common time t through crackle, in FP64, and written into the layout the
// evaluation kernel streams (one coalesced pass): FP64 records, or for the
// mixed path 13 FP32 rows with positions split into hi + lo.
#include "nb_device.cuh"
#include "nb_internal.cuh"

namespace {

using nbk::Taylor;
using nbk::taylor;

__global__ void __launch_bounds__(256) predict_kernel(const double *__restrict__ st,
                                                      const double *__restrict__ ti,
                                                      const double *__restrict__ m, int n, double t,
                                                      double2 *__restrict__ jb64,
                                                      float *__restrict__ jf32, size_t npad)
{
    const size_t N = static_cast<size_t>(n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = t - ti[i];
        Taylor p[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            p[k] = taylor(st[(F_X * 3 + k) * N + i], st[(F_V * 3 + k) * N + i],
                          st[(F_A * 3 + k) * N + i], st[(F_J * 3 + k) * N + i],
                          st[(F_S * 3 + k) * N + i], st[(F_C * 3 + k) * N + i], d);
        const double mi = m[i];
        if (jb64) {
            jb64[i] = make_double2(p[0].x, p[1].x);
            jb64[N + i] = make_double2(p[2].x, mi);
            jb64[2 * N + i] = make_double2(p[0].v, p[1].v);
            jb64[3 * N + i] = make_double2(p[2].v, p[0].a);
            jb64[4 * N + i] = make_double2(p[1].a, p[2].a);
        }
        if (jf32) {
            float h[3], l[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                h[k] = __double2float_rn(p[k].x);
                l[k] = __double2float_rn(p[k].x - static_cast<double>(h[k]));
            }
            jf32[0 * npad + i] = h[0];
            jf32[1 * npad + i] = h[1];
            jf32[2 * npad + i] = h[2];
            jf32[3 * npad + i] = __double2float_rn(mi);
            jf32[4 * npad + i] = l[0];
            jf32[5 * npad + i] = l[1];
            jf32[6 * npad + i] = l[2];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                jf32[(7 + k) * npad + i] = __double2float_rn(p[k].v);
                jf32[(10 + k) * npad + i] = __double2float_rn(p[k].a);
            }
        }
    }
}

}  // namespace

cudaError_t nb_launch_predict(nb_ctx *c, double t)
{
    const int n = static_cast<int>(c->n);
    const int block = 256;
    int grid = (n + block - 1) / block;
    grid = grid < c->sm_count * 16 ? grid : c->sm_count * 16;
    const bool mixed = c->cfg.precision == NB_MIXED;
    predict_kernel<<<grid, block, 0, c->stream>>>(c->st, c->t, c->m, n, t, mixed ? nullptr : c->jb64,
                                                  mixed ? c->jf32 : nullptr,
                                                  static_cast<size_t>(c->npad));
    c->launches += 1;
    return cudaGetLastError();
}
