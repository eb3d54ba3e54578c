// Predictor stage of the 6th-order Hermite scheme (paper, section 3): every
// particle's x, v and a are Taylor-expanded from its own time t_i to the
// common time t through crackle, in FP64, and written into the layout the
// evaluation kernel streams (one coalesced pass): FP64 records, for the
// mixed path 13 FP32 rows with positions split into hi + lo, or for the
// extended-precision path 20 FP32 rows of double words.
#include "nb_device.cuh"
#include "nb_internal.cuh"

namespace {

// Layouts of the FP32 j-buffer: 13 rows (positions hi + lo, the rest FP32),
// the same with the lo rows zero (single precision), or 20 rows of double
// words (extended precision).
constexpr int kModeMixed = 0, kModeSp = 1, kModeEx = 2;

using nbk::Taylor;
using nbk::taylor;

__global__ void __launch_bounds__(256) predict_kernel(const double *__restrict__ st,
                                                      const double *__restrict__ ti,
                                                      const double *__restrict__ m, int n, double t,
                                                      double2 *__restrict__ jb64,
                                                      float *__restrict__ jf32, size_t npad,
                                                      int mode)
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
        if (jf32 && mode == kModeEx) {
            // 20 rows: x, v, a (hi then lo per component group), m hi, m lo
            const double q[9] = {p[0].x, p[1].x, p[2].x, p[0].v, p[1].v, p[2].v, p[0].a, p[1].a, p[2].a};
#pragma unroll
            for (int g = 0; g < 3; ++g)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double d = q[3 * g + k];
                    const float h = __double2float_rn(d);
                    jf32[(6 * g + k) * npad + i] = h;
                    jf32[(6 * g + 3 + k) * npad + i] = __double2float_rn(d - static_cast<double>(h));
                }
            const float mh = __double2float_rn(mi);
            jf32[18 * npad + i] = mh;
            jf32[19 * npad + i] = __double2float_rn(mi - static_cast<double>(mh));
        } else if (jf32) {
            const bool drop_lo = mode == kModeSp;
            float h[3], l[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                h[k] = __double2float_rn(p[k].x);
                l[k] = drop_lo ? 0.0f : __double2float_rn(p[k].x - static_cast<double>(h[k]));
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
    const bool rows = nb_jrows(c->cfg.precision) > 0;
    const int mode = c->cfg.precision == NB_EX ? kModeEx : (c->cfg.precision == NB_SP ? kModeSp : kModeMixed);
    predict_kernel<<<grid, block, 0, c->stream>>>(c->st, c->t, c->m, n, t, rows ? nullptr : c->jb64,
                                                  rows ? c->jf32 : nullptr,
                                                  static_cast<size_t>(c->npad), mode);
    c->launches += 1;
    return cudaGetLastError();
}
