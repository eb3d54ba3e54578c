// Device-resident block stepping for one system (paper, section 3: block
// time steps, predictor / evaluation / corrector).
//
// Most block steps of a cluster integration have only a few active
// particles; driven from the host, each costs several launches and a host
// round trip for the size of the active set, more than its arithmetic.  This
// kernel runs such steps back to back in ONE cooperative launch whose blocks
// stay resident on every SM, separated by grid barriers:
//   schedule  every block scans its contiguous slice of the particles for
//             the earliest t_i + dt_i and lists the particles that reach it;
//             after a grid barrier all blocks read the same minima and counts
//             and take the same decision;
//   evaluate  every block predicts its slice into shared memory (chunk by
//             chunk, the layout of the evaluation buffer of the precision),
//             predicts the active particles itself, and sums the active set
//             against its slice; partial sums go to global memory;
//   correct   after a second grid barrier the block that owns an active
//             particle adds the partial sums of all blocks in block order and
//             applies the FP64 corrector and step selection (the same device
//             function as the corrector kernel).
// It returns to the host when the next active set holds more than
// kStepSmall particles (the host then runs that step with the tuned
// evaluation kernels), when the next block time passes t_end, or after an
// error flag.  Every block takes the same branch at every barrier (decisions
// come from the same global values), and no block waits on a flag.
#include <cooperative_groups.h>

#include <algorithm>

#include "nb_correct.cuh"
#include "nb_device.cuh"
#include "nb_ff.cuh"
#include "nb_internal.cuh"

namespace cg = cooperative_groups;

namespace {

using namespace nbk;

constexpr int kStepThreads = 128;
constexpr int kStepSmall = 128;  // active sets up to this size are stepped on the device
constexpr int kChunkCap = 1024;  // j-records per shared-memory chunk

struct StepOut {
    int64_t steps;     // block steps taken by the launch
    int64_t act_sum;   // active particles summed over those steps
    int32_t reason;    // 0: next block time beyond t_end, 1: next active set too large, 2: error
    int32_t n_act;     // active count of the last step taken
    double t_last;     // time of the last step taken
};

struct StepArgs {
    int n;
    double *st, *t, *dt;
    const double *m;
    double eps2, eta, dt_min, dt_max, dt_shared, t_end, noise;
    int drop_lo;        // single-precision control: positions without their low part
    double *bmin;       // [B] per-block earliest t_i + dt_i
    int *bcnt;          // [B] particles reaching it
    int *cand;          // [B][kStepSmall] their indices, ascending
    double *part;       // [B][kStepSmall][9] partial sums
    int32_t *act;       // active set of the last step taken
    nb_ctl *ctl;
    StepOut *out;
    double *log_t;      // per-step log (device), entries [log_base, log_cap)
    int64_t *log_n;
    int64_t log_cap, log_base;
};

// Bytes per j-record in shared memory: FP64 5 x 16, mixed 13 x 4, EX 20 x 4.
__host__ __device__ constexpr int rec_bytes(int pr) { return pr == 0 ? 80 : (pr == 1 ? NCF * 4 : NCX * 4); }

__device__ __forceinline__ double block_min_d(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1)
        v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = red[0];
    for (int q = 1; q < static_cast<int>(blockDim.x >> 5); ++q)
        r = fmin(r, red[q]);
    return r;
}

__device__ __forceinline__ int block_scan_excl(int v, int *red, int *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += u;
    }
    __syncthreads();
    if (lane == 31)
        red[w] = incl;
    __syncthreads();
    int base = 0, tot = 0;
    for (int q = 0; q < nw; ++q) {
        if (q < w)
            base += red[q];
        tot += red[q];
    }
    *total = tot;
    return base + incl - v;
}

// The predicted record of particle i at time tp in the precision's layout:
// FP64 5 double2 rows; mixed 13 FP32 rows (x_hi, m, x_lo, v, a; x_lo = 0 for
// the single-precision control); EX 20 FP32 rows (hi then lo of x, v, a; m
// hi, lo).  Rows go to rf[row * stride] (FP32 layouts) or rd[row * stride]
// (FP64 layout).
template <int PR>
__device__ __forceinline__ void predict_record(const StepArgs &a, int i, double tp, float *rf,
                                               double2 *rd, int stride)
{
    const size_t N = static_cast<size_t>(a.n);
    const double d = tp - a.t[i];
    Taylor p[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        p[k] = taylor(a.st[(F_X * 3 + k) * N + i], a.st[(F_V * 3 + k) * N + i], a.st[(F_A * 3 + k) * N + i],
                      a.st[(F_J * 3 + k) * N + i], a.st[(F_S * 3 + k) * N + i], a.st[(F_C * 3 + k) * N + i], d);
    const double mi = a.m[i];
    if constexpr (PR == 0) {
        rd[0] = make_double2(p[0].x, p[1].x);
        rd[stride] = make_double2(p[2].x, mi);
        rd[2 * stride] = make_double2(p[0].v, p[1].v);
        rd[3 * stride] = make_double2(p[2].v, p[0].a);
        rd[4 * stride] = make_double2(p[1].a, p[2].a);
    } else if constexpr (PR == 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float h = __double2float_rn(p[k].x);
            rf[k * stride] = h;
            rf[(4 + k) * stride] = a.drop_lo ? 0.0f : __double2float_rn(p[k].x - static_cast<double>(h));
            rf[(7 + k) * stride] = __double2float_rn(p[k].v);
            rf[(10 + k) * stride] = __double2float_rn(p[k].a);
        }
        rf[3 * stride] = __double2float_rn(mi);
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double q[3] = {p[k].x, p[k].v, p[k].a};
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const float h = __double2float_rn(q[g]);
                rf[(6 * g + k) * stride] = h;
                rf[(6 * g + 3 + k) * stride] = __double2float_rn(q[g] - static_cast<double>(h));
            }
        }
        const float mh = __double2float_rn(mi);
        rf[18 * stride] = mh;
        rf[19 * stride] = __double2float_rn(mi - static_cast<double>(mh));
    }
}

// i-values of active particle i (the same arithmetic as its j-record):
// FP64 x, v, a; mixed 12 negated FP32 (x_hi, x_lo, v, a); EX 18 negated FP32
// (hi then lo of x, v, a).  iv holds 9 doubles = 18 floats.
template <int PR>
__device__ __forceinline__ void ivalues(const StepArgs &a, int i, double tp, double *iv)
{
    if constexpr (PR == 0) {
        double2 r[5];
        predict_record<0>(a, i, tp, nullptr, r, 1);
        iv[0] = r[0].x; iv[1] = r[0].y; iv[2] = r[1].x;
        iv[3] = r[2].x; iv[4] = r[2].y; iv[5] = r[3].x;
        iv[6] = r[3].y; iv[7] = r[4].x; iv[8] = r[4].y;
    } else if constexpr (PR == 1) {
        float r[NCF];
        predict_record<1>(a, i, tp, r, nullptr, 1);
        float *f = reinterpret_cast<float *>(iv);
        constexpr int kRow[12] = {0, 1, 2, 4, 5, 6, 7, 8, 9, 10, 11, 12};
#pragma unroll
        for (int q = 0; q < 12; ++q)
            f[q] = -r[kRow[q]];
    } else {
        float r[NCX];
        predict_record<2>(a, i, tp, r, nullptr, 1);
        float *f = reinterpret_cast<float *>(iv);
#pragma unroll
        for (int q = 0; q < 18; ++q)
            f[q] = -r[q];
    }
}

// Partial sums of the K active particles (i-values iv) over the j of
// [lo, hi), predicted to tp chunk by chunk into shared memory, written to
// part[K][9].  L = T / K2 lanes per active particle (K2 the power of two
// >= K) take every L-th j (pair of j in the FP32 precisions); lanes are
// combined in a fixed order.
template <int PR>
__device__ void eval_slice(const StepArgs &a, int lo, int hi, double tp, int K, const double (*iv)[9],
                           double *part, double (*wred)[9], unsigned char *smem)
{
    const int T = blockDim.x, tid = threadIdx.x;
    int K2 = 1;
    while (K2 < K)
        K2 <<= 1;
    const int L = T / K2;
    const int g = tid / L, lane = tid - g * L;
    const bool valid = g < K;
    const int gi = valid ? g : 0;
    constexpr int cap = kChunkCap;
    float *sf = reinterpret_cast<float *>(smem);
    double2 *sd = reinterpret_cast<double2 *>(smem);
    double acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q)
        acc[q] = 0.0;
    // FP32 precisions: packed pair sums, folded every 32 iterations
    float2 ni[12], pm[9];
    float ah[9], al[9];
    ExI<float2> nie;
    ff::FF<float2> px[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        pm[q] = f2(0.0f);
        ah[q] = al[q] = 0.0f;
        px[q] = {f2(0.0f), f2(0.0f)};
    }
    if (PR == 1) {
        const float *f = reinterpret_cast<const float *>(iv[gi]);
#pragma unroll
        for (int q = 0; q < 12; ++q)
            ni[q] = f2(f[q]);
    } else if (PR == 2) {
        const float *f = reinterpret_cast<const float *>(iv[gi]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            nie.x[k] = {f2(f[k]), f2(f[3 + k])};
            nie.v[k] = {f2(f[6 + k]), f2(f[9 + k])};
            nie.a[k] = {f2(f[12 + k]), f2(f[15 + k])};
        }
    }
    const float2 eps2f = f2(__double2float_rn(a.eps2));
    const float e2h = __double2float_rn(a.eps2);
    const ff::FF<float2> eps2x = {f2(e2h), f2(__double2float_rn(a.eps2 - static_cast<double>(e2h)))};
    int cnt = 0;
    for (int b = lo; b < hi; b += cap) {
        const int len = min(cap, hi - b);
        for (int u = tid; u < len; u += T)
            predict_record<PR>(a, b + u, tp, sf + u, sd + u, cap);
        __syncthreads();
        if constexpr (PR == 0) {
            const double *v = iv[gi];
            for (int jj = lane; jj < len; jj += L)
                pair_fp64(sd[jj], sd[cap + jj], sd[2 * cap + jj], sd[3 * cap + jj], sd[4 * cap + jj], v[0], v[1],
                          v[2], v[3], v[4], v[5], v[6], v[7], v[8], a.eps2, acc);
        } else {
            constexpr int NR = PR == 1 ? NCF : NCX;
            constexpr int mrow = PR == 1 ? 3 : 18;  // first mass row
            for (int jj = 2 * lane; jj < len; jj += 2 * L) {
                float2 c[NR];
                if (jj + 1 < len) {
#pragma unroll
                    for (int r = 0; r < NR; ++r)
                        c[r] = *reinterpret_cast<const float2 *>(sf + r * cap + jj);
                } else {
                    // odd tail: the second half repeats the first j with no mass
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const float x0 = sf[r * cap + jj];
                        c[r] = make_float2(x0, r >= mrow ? 0.0f : x0);
                    }
                }
                if constexpr (PR == 1)
                    pair_mixed2(c, ni, eps2f, pm);
                else
                    pair_ex(c, nie, eps2x, px);
                if (++cnt == 32) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        if (PR == 1) {
                            two_sum_acc(ah[q], al[q], __fadd_rn(pm[q].x, pm[q].y));
                            pm[q] = f2(0.0f);
                        } else {
                            acc[q] += (static_cast<double>(px[q].h.x) + static_cast<double>(px[q].l.x)) +
                                      (static_cast<double>(px[q].h.y) + static_cast<double>(px[q].l.y));
                            px[q] = {f2(0.0f), f2(0.0f)};
                        }
                    }
                    cnt = 0;
                }
            }
        }
        __syncthreads();
    }
    const int w = tid >> 5;
    const int span = L < 32 ? L : 32;
    if (PR == 1) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            two_sum_acc(ah[q], al[q], __fadd_rn(pm[q].x, pm[q].y));
            for (int o = span >> 1; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, ah[q], o);
                const float ol = __shfl_xor_sync(0xffffffffu, al[q], o);
                two_sum_acc(ah[q], al[q], oh);
                al[q] = __fadd_rn(al[q], ol);
            }
            acc[q] = static_cast<double>(ah[q]) + static_cast<double>(al[q]);
        }
    } else {
        if (PR == 2)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                acc[q] += (static_cast<double>(px[q].h.x) + static_cast<double>(px[q].l.x)) +
                          (static_cast<double>(px[q].h.y) + static_cast<double>(px[q].l.y));
        for (int o = span >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    }
    if (L <= 32) {
        if (valid && lane == 0)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                part[g * 9 + q] = acc[q];
    } else {
        if ((tid & 31) == 0)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                wred[w][q] = acc[q];
        __syncthreads();
        const int wpg = L >> 5;
        if (tid < K)
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                double s = 0.0;
                for (int u = 0; u < wpg; ++u)
                    s += wred[tid * wpg + u][q];
                part[tid * 9 + q] = s;
            }
    }
    __syncthreads();
}

template <int PR>
__global__ void __launch_bounds__(kStepThreads) step_kernel(StepArgs a)
{
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red_d[32];
    __shared__ int red_i[32];
    __shared__ int s_act[kStepSmall];
    __shared__ double s_iv[kStepSmall][9];
    __shared__ double s_wred[kStepThreads / 32][9];
    __shared__ double s_f[kStepSmall][9];
    __shared__ int s_nb, s_qb[kStepSmall], s_blk[kStepSmall], s_cnt[kStepSmall];
    const int B = gridDim.x, bk = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
    const int per = (a.n + B - 1) / B;
    const int lo = min(a.n, bk * per), hi = min(a.n, lo + per);
    const int per_t = (hi - lo + T - 1) / T;
    const int c0 = min(hi, lo + tid * per_t), c1 = min(hi, c0 + per_t);
    int64_t steps = 0, act_sum = 0;
    int reason = 0, last_n = 0;
    double last_t = 0.0;
    for (;;) {
        // schedule: this block's earliest t_i + dt_i, the particles reaching it
        double mt = INFINITY;
        int ct = 0;
        for (int i = c0; i < c1; ++i) {
            const double tt = a.t[i] + a.dt[i];
            if (tt < mt) {
                mt = tt;
                ct = 1;
            } else if (tt == mt) {
                ++ct;
            }
        }
        const double mb = block_min_d(mt, red_d);
        const int mine = (mt == mb) ? ct : 0;
        int tot_b = 0;
        const int ex = block_scan_excl(mine, red_i, &tot_b);
        if (mine > 0 && tot_b <= kStepSmall) {
            int pos = ex;
            for (int i = c0; i < c1; ++i)
                if (a.t[i] + a.dt[i] == mb)
                    a.cand[bk * kStepSmall + pos++] = i;
        }
        if (tid == 0) {
            a.bmin[bk] = mb;
            a.bcnt[bk] = tot_b;
        }
        grid.sync();
        // the same decision in every block
        double mn = INFINITY;
        for (int q = tid; q < B; q += T)
            mn = fmin(mn, __ldcg(&a.bmin[q]));
        mn = block_min_d(mn, red_d);
        int c = 0;
        for (int q = tid; q < B; q += T)
            c += (__ldcg(&a.bmin[q]) == mn) ? __ldcg(&a.bcnt[q]) : 0;
        int total = 0;
        block_scan_excl(c, red_i, &total);
        const int err = *reinterpret_cast<volatile int *>(&a.ctl->err);
        if (err) {
            reason = 2;
            break;
        }
        if (mn > a.t_end) {
            reason = 0;
            break;
        }
        if (total > kStepSmall) {
            reason = 1;
            break;
        }
        // the blocks holding the active set, in block order (at most total)
        if (tid == 0)
            s_nb = 0;
        __syncthreads();
        for (int q = tid; q < B; q += T)
            if (__ldcg(&a.bmin[q]) == mn && __ldcg(&a.bcnt[q]) > 0)
                s_qb[atomicAdd(&s_nb, 1)] = q;
        __syncthreads();
        const int nb = s_nb;
        if (tid < nb) {
            const int q = s_qb[tid];
            int r = 0;
            for (int u = 0; u < nb; ++u)
                r += s_qb[u] < q ? 1 : 0;
            s_blk[r] = q;
            s_cnt[r] = __ldcg(&a.bcnt[q]);
        }
        __syncthreads();
        // active list (ascending) and the predicted i-values
        for (int k = tid; k < total; k += T) {
            int base = 0, r = 0;
            while (k >= base + s_cnt[r])
                base += s_cnt[r++];
            const int i = __ldcg(&a.cand[s_blk[r] * kStepSmall + (k - base)]);
            s_act[k] = i;
            ivalues<PR>(a, i, mn, s_iv[k]);
        }
        __syncthreads();
        eval_slice<PR>(a, lo, hi, mn, total, s_iv, a.part + static_cast<size_t>(bk) * kStepSmall * 9, s_wred,
                       smem);
        grid.sync();
        // owners: the partial sums of all blocks in block order, then correct
        bool owns_any = false;
        for (int k = 0; k < total; ++k) {
            const int i = s_act[k];
            if (i < lo || i >= hi)
                continue;
            owns_any = true;
            double s9[9];
#pragma unroll
            for (int q = 0; q < 9; ++q)
                s9[q] = 0.0;
            for (int q2 = tid; q2 < B; q2 += T) {
                const double *pp = a.part + (static_cast<size_t>(q2) * kStepSmall + k) * 9;
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    s9[q] += __ldcg(&pp[q]);
            }
            // fixed-order combination of the threads' sums
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    s9[q] += __shfl_xor_sync(0xffffffffu, s9[q], o);
            if ((tid & 31) == 0)
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    s_wred[tid >> 5][q] = s9[q];
            __syncthreads();
            if (tid < 9) {
                double s = 0.0;
                for (int u = 0; u < (T >> 5); ++u)
                    s += s_wred[u][tid];
                s_f[k][tid] = s;
            }
            __syncthreads();
        }
        if (owns_any)
            for (int k = tid; k < total; k += T) {
                const int i = s_act[k];
                if (i < lo || i >= hi)
                    continue;
                double f[9];
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    f[q] = s_f[k][q];
                correct_particle_fp64(a.st, a.t, a.dt, static_cast<size_t>(a.n), i, mn, f, a.eta, a.dt_min,
                                      a.dt_max, a.dt_shared, a.ctl, a.noise);
            }
        if (bk == 0) {
            for (int k = tid; k < total; k += T)
                a.act[k] = s_act[k];
            if (tid == 0) {
                const int64_t li = a.log_base + steps;
                if (li < a.log_cap) {
                    a.log_t[li] = mn;
                    a.log_n[li] = total;
                }
            }
        }
        ++steps;
        act_sum += total;
        last_t = mn;
        last_n = total;
        __syncthreads();
    }
    if (bk == 0 && tid == 0) {
        a.out->steps = steps;
        a.out->act_sum = act_sum;
        a.out->reason = reason;
        a.out->n_act = last_n;
        a.out->t_last = last_t;
    }
}

template <int PR>
cudaError_t launch_stepper(nb_ctx *c, StepArgs &a, int grid_max)
{
    const size_t smem = static_cast<size_t>(kChunkCap) * rec_bytes(PR);
    cudaError_t e = cudaFuncSetAttribute(step_kernel<PR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess)
        return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<PR>, kStepThreads, smem);
    if (e != cudaSuccess)
        return e;
    if (per_sm < 1)
        return cudaErrorInvalidConfiguration;
    int grid = std::min(c->sm_count * per_sm, grid_max);                  // all blocks resident
    grid = std::min(grid, std::max(1, static_cast<int>((c->n + 31) / 32)));  // >= 32 particles per block
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(step_kernel<PR>), dim3(grid),
                                       dim3(kStepThreads), args, smem, c->stream);
}

}  // namespace

int nb_stepper_small() { return kStepSmall; }

// One launch of the device-resident stepper; reports what it did in
// *steps, *act_sum, *reason, *n_act, *t_last (synchronises the stream).
cudaError_t nb_run_stepper(nb_ctx *c, double t_end, int64_t log_cap, int64_t log_base, int64_t *steps,
                           int64_t *act_sum, int *reason, int *n_act, double *t_last)
{
    // scratch sized for the largest grid this device can hold
    const int grid_max = c->sm_count * 16;
    if (!c->stp_bmin) {
        cudaError_t e;
        if ((e = cudaMalloc(&c->stp_bmin, grid_max * sizeof(double))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&c->stp_bcnt, grid_max * sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&c->stp_cand, static_cast<size_t>(grid_max) * kStepSmall * sizeof(int))) != cudaSuccess)
            return e;
        if ((e = cudaMalloc(&c->stp_part, static_cast<size_t>(grid_max) * kStepSmall * 9 * sizeof(double))) !=
            cudaSuccess)
            return e;
        if ((e = cudaMalloc(&c->stp_out, sizeof(StepOut))) != cudaSuccess) return e;
        if ((e = cudaMallocHost(&c->stp_out_h, sizeof(StepOut))) != cudaSuccess) return e;
    }
    StepArgs a;
    a.n = static_cast<int>(c->n);
    a.st = c->st;
    a.t = c->t;
    a.dt = c->dt;
    a.m = c->m;
    a.eps2 = c->eps * c->eps;
    a.eta = c->cfg.eta;
    a.noise = c->cfg.step_noise;
    a.dt_min = c->cfg.dt_min;
    a.dt_max = c->cfg.dt_max;
    a.dt_shared = c->cfg.dt_shared;
    a.t_end = t_end;
    a.drop_lo = c->cfg.precision == NB_SP ? 1 : 0;
    a.bmin = c->stp_bmin;
    a.bcnt = c->stp_bcnt;
    a.cand = c->stp_cand;
    a.part = c->stp_part;
    a.act = c->act;
    a.ctl = c->ctl;
    a.out = static_cast<StepOut *>(c->stp_out);
    a.log_t = c->stp_log_t;
    a.log_n = c->stp_log_n;
    a.log_cap = c->stp_log_t ? log_cap : 0;
    a.log_base = log_base;
    const int pr = c->cfg.precision == NB_EX ? 2 : (nb_fp32_eval(c->cfg.precision) ? 1 : 0);
    cudaError_t e = pr == 2 ? launch_stepper<2>(c, a, grid_max)
                            : (pr == 1 ? launch_stepper<1>(c, a, grid_max) : launch_stepper<0>(c, a, grid_max));
    if (e != cudaSuccess)
        return e;
    c->launches += 1;
    e = cudaMemcpyAsync(c->stp_out_h, c->stp_out, sizeof(StepOut), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess)
        return e;
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return e;
    const StepOut *o = static_cast<const StepOut *>(c->stp_out_h);
    *steps = o->steps;
    *act_sum = o->act_sum;
    *reason = o->reason;
    *n_act = o->n_act;
    *t_last = o->t_last;
    return cudaSuccess;
}
