// Internal declarations of libnb: the context, device helpers shared by the
// kernels (TMA bulk copies, bounded mbarrier waits, FP64 reciprocal square
// root, TwoSum), and the launch functions of each kernel file.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "nb.h"

// ------------------------------------------------------------------ layout
//
// State (FP64, structure of arrays, component-major, stride n):
//   st[(F * 3 + k) * n + i] for field F in {X, V, A, J, S, C}, component k.
// Evaluation buffers written by the predictor (stride n):
//   FP64:  jb64[c * n + i], c = 0..4: (x, y) (z, m) (vx, vy) (vz, ax) (ay, az)
//   mixed: jf32[c * npad + i], 13 float rows c = 0..12:
//          xh yh zh m xl yl zl vx vy vz ax ay az, with xh = fp32(x) and
//          xl = fp32(x - xh); npad = n rounded up to a multiple of 4, the
//          padding rows hold zero-mass particles (contribute exactly 0).
// Evaluation output (stride ostride): out[q * ostride + k], q = 0..8 for
//   acc x,y,z, jerk x,y,z, snap x,y,z of the k-th listed particle.
enum { F_X = 0, F_V = 1, F_A = 2, F_J = 3, F_S = 4, F_C = 5, NFIELD = 6 };

// Evaluations that use the FP32 row buffer and the packed FP32 kernel.
inline bool nb_fp32_eval(int precision) { return precision == NB_MIXED || precision == NB_SP; }
// FP32 rows per particle of the predicted j-buffer (0: FP64 records).
inline int nb_jrows(int precision)
{
    return precision == NB_EX ? 20 : (nb_fp32_eval(precision) ? 13 : 0);
}

struct nb_ctl {                      // small device control block
    unsigned long long tnext_bits;   // min over i of (t_i + dt_i), as bits
    int32_t n_act;                   // active count from the scheduler
    int32_t err;                     // bit flags, see NB_ERR_*
    int64_t floor_hits;              // steps clamped at dt_min
};
#define NB_ERR_NONFINITE 1
#define NB_ERR_TIMEOUT 2

struct nb_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    nb_config cfg{};
    int64_t n = 0;
    double eps = 0;
    int sm_count = 0;

    double *m = nullptr;       // [n]
    double *st = nullptr;      // [18][n]
    double *t = nullptr;       // [n]
    double *dt = nullptr;      // [n]
    double2 *jb64 = nullptr;   // [5][n]
    float *jf32 = nullptr;     // [13][npad]
    int64_t npad = 0;
    int32_t *act = nullptr;    // [n] active set of the last step evaluated
    int32_t *act_next = nullptr;  // [n] active set found by the scheduler, swapped in by the step
    double *anew = nullptr;    // [9][n]
    double *stage = nullptr;   // [3][n][3] output staging
    double *part = nullptr;    // split-j partials
    size_t part_cap = 0;       // doubles
    unsigned *tile_cnt = nullptr;
    size_t tile_cnt_cap = 0;
    int32_t *blk = nullptr;    // scheduler block counts
    double *red = nullptr;     // reduction scratch
    size_t red_cap = 0;        // doubles
    nb_ctl *ctl = nullptr;     // device
    nb_ctl *ctl_h = nullptr;   // pinned host mirror
    double *diag = nullptr;    // [8] device results of energy / angmom
    double *diag_h = nullptr;  // [8] pinned host mirror
    double *ring = nullptr;    // [ring_cap][8] diagnostics samples of nb_run_diag
    int64_t ring_cap = 0;
    // device-resident stepper (k_stepper.cu): per-block scratch, results, log
    double *stp_bmin = nullptr;
    int *stp_bcnt = nullptr, *stp_cand = nullptr;
    double *stp_part = nullptr;
    void *stp_out = nullptr, *stp_out_h = nullptr;
    double *stp_log_t = nullptr;
    int64_t *stp_log_n = nullptr;

    int64_t n_act = 0;         // size of the last evaluated set
    bool have_pred = false;
    double t_pred = 0;
    bool have_eval = false;
    double t_eval = 0;
    double t_sys = 0;          // min t_i after the last block step (host copy)
    int64_t launches = 0;
    double interactions = 0;
    int32_t inject = 0;        // one-shot fault injection for tests (nb_inject_fault)
    bool dead = false;
    std::string err;
};

// --------------------------------------------------------- device helpers

namespace nbk {

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D TMA bulk copy global -> shared, completion signalled on bar.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, "
        "p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of bar to complete, giving up after limit_ns of
// wall-clock time (globaltimer).  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns)
{
    if (mbar_test(bar, parity))
        return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_test(bar, parity)) {
        if (globaltimer_ns() - t0 > limit_ns)
            return false;
    }
    return true;
}

constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s

// Reciprocal square root of a positive normal double: an FP32 hardware
// estimate (inputs and result converted by exponent re-biasing on the
// integer pipe) refined by one third-order Householder step,
//   y = y0 (1 + h/2 + 3 h^2 / 8),  h = 1 - x y0^2,
// the series of (1 - h)^(-1/2) truncated after h^2.  From a 2^-22 estimate
// the truncation error is below 2^-63, so the result is within about one
// rounding of 1/sqrt(x).  Valid for 2^-126 < x < 2^127 (FP32 normal range).
__device__ __forceinline__ double rsqrt_fp64(double x)
{
    const int hi = __double2hiint(x);
    const unsigned lo = static_cast<unsigned>(__double2loint(x));
    // double (11-bit exponent, bias 1023) -> float (8-bit, bias 127), mantissa truncated
    const unsigned fb = (static_cast<unsigned>(hi - (896 << 20)) << 3) | (lo >> 29);
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__uint_as_float(fb)));
    const unsigned yb = __float_as_uint(yf);
    const double y0 = __hiloint2double(static_cast<int>((yb >> 3) + (896u << 20)),
                                       static_cast<int>(yb << 29));
    const double h = fma(-x, y0 * y0, 1.0);
    const double p = fma(h, 0.375, 0.5);
    return fma(h * y0, p, y0);
}

// TwoSum (Knuth): s + e == a + b exactly.  Accumulates the rounding error
// of hi + p into lo.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float p)
{
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

}  // namespace nbk

// ------------------------------------------------------- launch functions

struct EvalLaunch {
    const int32_t *act;  // device list of n_act indices
    int n_act;
    double *out;         // [9][ostride]
    int ostride;
    nb_tiles tiles;      // resolved
    int64_t j0 = 0, j1 = -1;  // j-range [j0, j1) of the evaluation buffer; j1 < 0: all of it
};

// k_eval.cu
cudaError_t nb_launch_eval(nb_ctx *c, const EvalLaunch &L);
// j_count: length of the j-range evaluated (0: the whole buffer)
nb_tiles nb_auto_tiles(const nb_ctx *c, int64_t n_act, const nb_tiles &req, int64_t j_count = 0);
cudaError_t nb_eval_smem_setup();
// k_predict.cu
cudaError_t nb_launch_predict(nb_ctx *c, double t);
// k_correct.cu
cudaError_t nb_launch_correct(nb_ctx *c, double t1, int n_act);
cudaError_t nb_launch_init_state(nb_ctx *c, int pass);
cudaError_t nb_launch_transpose_out(nb_ctx *c, int n_act, int q0, double *dst);
cudaError_t nb_launch_rows_to_soa(nb_ctx *c, const double *rows, int field);
cudaError_t nb_launch_soa_to_rows(nb_ctx *c, int field, double *rows);
// k_sched.cu
cudaError_t nb_launch_schedule(nb_ctx *c);
cudaError_t nb_launch_iota(nb_ctx *c, int n, int32_t *dst);
// nb_api.cu: message returned by nb_last_error(NULL) on this thread
void nb_set_thread_error(const char *msg);
// k_stepper.cu
int nb_stepper_small();
cudaError_t nb_run_stepper(nb_ctx *c, double t_end, int64_t log_cap, int64_t log_base, int64_t *steps,
                           int64_t *act_sum, int *reason, int *n_act, double *t_last);

// k_energy.cu
cudaError_t nb_launch_energy(nb_ctx *c, double *ek_pe_dev);
cudaError_t nb_launch_angmom(nb_ctx *c, double *l4_dev);
// k_kappa.cu: condition numbers sum_j |A_ij|, |J_ij|, |S_ij| of the listed
// particles against the predicted j-buffer, out_dev [3][n_act].
cudaError_t nb_launch_kappa(nb_ctx *c, const int32_t *act_dev, int n_act, double *out_dev);
