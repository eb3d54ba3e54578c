// Ensemble of independent N-body systems, each on its own block time steps
// (paper, sections 2-3: block steps, predictor / evaluation / corrector),
// advanced together in ONE persistent launch.
//
// Work division on GB300: the grid is made of thread-block clusters of G
// CTAs (G <= 16, co-scheduled by the hardware; above 8 with the non-portable
// cluster-size opt-in).  Each hardware cluster takes
// the next system from an atomic queue (largest systems first) and runs its
// whole block-step loop to t_end:
//   schedule  t_next = min(t_i + dt_i) over the system; active set in
//             ascending order (each CTA scans its slice once, the minima and
//             counts meet through distributed shared memory);
//   predict   each CTA its slice: for small active sets straight into
//             shared memory, otherwise into the system's evaluation buffer;
//   evaluate  small active sets (<= small_set(PR), at most one per thread):
//             every CTA evaluates the whole
//             set against its own slice and the owner of each active
//             particle adds the CTAs' partial sums in rank order (two cluster
//             barriers per block step); larger sets: each CTA a share of the
//             active particles against all of the system's particles, j-tiles
//             by TMA bulk copy into shared memory;
//   correct   the owner (small sets) or the evaluating CTA (larger sets).
// Precisions (kernel template PR): FP64 (0); mixed (1): FP32 pair arithmetic
// with the FP64 predictor and corrector; EX double words (2) with the FP64
// predictor and corrector; mixed with an FP32 state copy (3): the mixed pair
// arithmetic, with the predictor, the corrector's increments and the step
// criterion in FP32 from an FP32 copy of the state.
// Phases are separated by the cluster barrier (a hardware barrier with
// release/acquire semantics at cluster scope, no flag spinning).  Systems are
// independent, so no grid-wide synchronisation exists.  The only waits that
// poll (TMA completion) give up after a time limit; a failure is made
// uniform across the cluster and ends the launch with an error flag.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "nb_correct.cuh"
#include "nb_device.cuh"
#include "nb_ff.cuh"
#include "nb_internal.cuh"

namespace cg = cooperative_groups;

struct nb_ensemble {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    nb_config cfg{};
    double eps = 0;
    int nc = 0;
    int64_t P = 0;  // padded particle total
    std::vector<int32_t> off, cnt;
    int32_t *d_off = nullptr, *d_cnt = nullptr, *d_order = nullptr;
    double *m = nullptr, *st = nullptr, *t = nullptr, *dt = nullptr, *anew = nullptr;
    double2 *jb64 = nullptr;
    float *jf32 = nullptr;
    float *st32 = nullptr;  // NB_MIXED32: FP32 copy of the state [24][P] (rows: see predict_one_mixed)
    double *gpart = nullptr;  // j-split partial sums, [clusters in the grid][G][9][nmax4]
    size_t gpart_cap = 0;     // doubles
    int64_t nmax4 = 4;        // largest system, padded to a multiple of 4
    // optional step log (nb_ensemble_set_log): counters [2] = steps, indices
    unsigned long long *log_cnt = nullptr;
    int32_t *log_sys = nullptr, *log_n = nullptr, *log_idx = nullptr;
    double *log_t = nullptr;
    int64_t *log_off = nullptr;
    int64_t log_cap = 0, idx_cap = 0;
    int32_t *act = nullptr;
    int *queue = nullptr;
    int64_t *steps = nullptr;
    unsigned long long *inter = nullptr;
    nb_ctl *ctl = nullptr, *ctl_h = nullptr;
    int G = 4, threads = 128, jtile = 256;   // set per precision by nb_ensemble_init
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double graph_t_end = -1.0;
    int64_t launches = 0;
    bool dead = false;
    std::string err;
};

namespace {

using namespace nbk;

struct EnsArgs {
    int nc;
    const int32_t *off, *cnt, *order;
    int P;
    double *st, *t, *dt;
    const double *m;
    double2 *jb64;
    float *jf32;
    float *st32;
    int32_t *act;
    double *anew;
    int *queue;
    int64_t *steps;
    unsigned long long *inter;
    nb_ctl *ctl;
    double *gpart;                 // j-split partial sums: [clusters][G][9][gstride]
    long long gstride;             // largest system, padded to a multiple of 4
    unsigned long long *log_cnt;   // NULL: no step log
    int32_t *log_sys, *log_n, *log_idx;
    double *log_t;
    int64_t *log_off;
    long long log_cap, idx_cap;
    double t_end, eps2, eta, eta_s, dt_min, dt_max, dt_shared;
    double noise;                  // step-criterion rounding floor (nb_config.step_noise)
    int mode;  // 0: block steps to t_end, 1: start-up (a, jerk, snap, starting steps)
    int jtile;
};

constexpr int kEnsThreads = 256;
constexpr int kMaxCluster = 16;  // blocks per system: 8 portable, 16 with the opt-in attribute

__device__ __forceinline__ double block_min(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1)
        v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
        red[w] = v;
    __syncthreads();
    double r = red[0];
    for (int q = 1; q < static_cast<int>(blockDim.x >> 5); ++q)
        r = fmin(r, red[q]);
    return r;
}

__device__ int block_exclusive_scan(int v, int *red, int *total)
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

// Taylor prediction of particle i to tp (FP64, through crackle).
__device__ __forceinline__ void predict_one(const EnsArgs &a, int i, double tp, Taylor (&p)[3])
{
    const size_t P = static_cast<size_t>(a.P);
    const double d = tp - a.t[i];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        p[k] = taylor(a.st[(F_X * 3 + k) * P + i], a.st[(F_V * 3 + k) * P + i], a.st[(F_A * 3 + k) * P + i],
                      a.st[(F_J * 3 + k) * P + i], a.st[(F_S * 3 + k) * P + i], a.st[(F_C * 3 + k) * P + i], d);
}

// The record the mixed evaluation reads (x_hi, x_lo, v, a in FP32) predicted
// to tp from an FP32 copy of the state: rows 0-2 v_hi, 3-5 a, 6-8 jerk,
// 9-11 snap, 12-14 crackle, 15-17 x_hi, 18-20 x_lo, 21-23 v_lo (x and v as
// double words, hi + lo of the FP64 values).  The predicted v and a are
// Horner sums in FP32; x = x0 + d (v0 + d/2 I) with
// I = a0 + d/3 (j0 + d/4 (s0 + d/5 c0)) is formed in double-word
// arithmetic: d v_hi exactly by TwoProd (d = tp - t_i is a dyadic step of at
// most 18 significant bits, exact in FP32), the smaller terms in FP32, then
// TwoSum with x and one renormalisation.  x then carries about 2^-47 |x|
// plus the FP32 rounding of its acceleration term, about 1e-7 of d^2 |a| / 2,
// below the FP32 rounding the pair arithmetic applies to the differences.
struct MixedRec {
    float xh[3], xl[3], v[3], a[3];
};

constexpr int kSt32Rows = 24;

__device__ __forceinline__ void predict_one_mixed(const EnsArgs &a, int i, double tp, MixedRec &r)
{
    const size_t P = static_cast<size_t>(a.P);
    const float df = __double2float_rn(tp - a.t[i]);
    const float d2 = df * 0.5f, d3 = df * (1.0f / 3.0f), d4 = df * 0.25f, d5 = df * 0.2f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float vh = a.st32[k * P + i], ac = a.st32[(3 + k) * P + i], j = a.st32[(6 + k) * P + i];
        const float sn = a.st32[(9 + k) * P + i], c = a.st32[(12 + k) * P + i];
        const float xh = a.st32[(15 + k) * P + i], xl = a.st32[(18 + k) * P + i];
        const float vl = a.st32[(21 + k) * P + i];
        r.a[k] = fmaf(df, fmaf(d2, fmaf(d3, c, sn), j), ac);
        r.v[k] = __fadd_rn(fmaf(df, fmaf(d2, fmaf(d3, fmaf(d4, c, sn), j), ac), vh), vl);
        const float I = fmaf(d3, fmaf(d4, fmaf(d5, c, sn), j), ac);
        const float p = __fmul_rn(df, vh);
        const float e = fmaf(df, fmaf(d2, I, vl), fmaf(df, vh, -p));
        // TwoSum(xh, p), low parts gathered, renormalised
        const float s = __fadd_rn(xh, p);
        const float bp = __fsub_rn(s, xh);
        const float t = __fadd_rn(__fadd_rn(__fsub_rn(xh, __fsub_rn(s, bp)), __fsub_rn(p, bp)),
                                  __fadd_rn(xl, e));
        const float h = __fadd_rn(s, t);
        r.xh[k] = h;
        r.xl[k] = __fsub_rn(t, __fsub_rn(h, s));
    }
}

// Write the FP32 copy of a particle's x and v (double words) from FP64.
__device__ __forceinline__ void store_xv32(const EnsArgs &a, int i, int k, double x, double v)
{
    const size_t P = static_cast<size_t>(a.P);
    const float xh = __double2float_rn(x), vh = __double2float_rn(v);
    a.st32[(15 + k) * P + i] = xh;
    a.st32[(18 + k) * P + i] = __double2float_rn(x - static_cast<double>(xh));
    a.st32[k * P + i] = vh;
    a.st32[(21 + k) * P + i] = __double2float_rn(v - static_cast<double>(vh));
}

// The mixed j-record of particle i predicted to tp.  NB_MIXED (PR 1): the
// FP64 Taylor predictor, as in a single-system context, then x rounded to a
// hi + lo pair of FP32 numbers and v, a to FP32.  NB_MIXED32 (PR 3): the
// FP32 predictor from the FP32 state copy.
template <int PR>
__device__ __forceinline__ void mixed_record(const EnsArgs &a, int i, double tp, MixedRec &r)
{
    if (PR == 3) {
        predict_one_mixed(a, i, tp, r);
        return;
    }
    Taylor p[3];
    predict_one(a, i, tp, p);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float h = __double2float_rn(p[k].x);
        r.xh[k] = h;
        r.xl[k] = __double2float_rn(p[k].x - static_cast<double>(h));
        r.v[k] = __double2float_rn(p[k].v);
        r.a[k] = __double2float_rn(p[k].a);
    }
}

template <int PR>
__device__ void predict_slice(const EnsArgs &a, int lo, int hi, double tp)
{
    [[maybe_unused]] constexpr bool MIXED = PR == 1 || PR == 3, EXP = PR == 2;
    const size_t P = static_cast<size_t>(a.P);
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        if (MIXED) {
            MixedRec r;
            mixed_record<PR>(a, i, tp, r);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                a.jf32[k * P + i] = r.xh[k];
                a.jf32[(4 + k) * P + i] = r.xl[k];
                a.jf32[(7 + k) * P + i] = r.v[k];
                a.jf32[(10 + k) * P + i] = r.a[k];
            }
            a.jf32[3 * P + i] = __double2float_rn(a.m[i]);
        } else if (EXP) {
            // 20 FP32 rows: hi then lo of x, v, a (three rows each), m hi, m lo
            Taylor p[3];
            predict_one(a, i, tp, p);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double q[3] = {p[k].x, p[k].v, p[k].a};
#pragma unroll
                for (int g = 0; g < 3; ++g) {
                    const float h = __double2float_rn(q[g]);
                    a.jf32[(6 * g + k) * P + i] = h;
                    a.jf32[(6 * g + 3 + k) * P + i] = __double2float_rn(q[g] - static_cast<double>(h));
                }
            }
            const float mh = __double2float_rn(a.m[i]);
            a.jf32[18 * P + i] = mh;
            a.jf32[19 * P + i] = __double2float_rn(a.m[i] - static_cast<double>(mh));
        } else {
            Taylor p[3];
            predict_one(a, i, tp, p);
            a.jb64[i] = make_double2(p[0].x, p[1].x);
            a.jb64[P + i] = make_double2(p[2].x, a.m[i]);
            a.jb64[2 * P + i] = make_double2(p[0].v, p[1].v);
            a.jb64[3 * P + i] = make_double2(p[2].v, p[0].a);
            a.jb64[4 * P + i] = make_double2(p[1].a, p[2].a);
        }
    }
    // the evaluation reads this buffer through TMA (async proxy)
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

template <int PR>
__device__ __forceinline__ void issue_ens_tile(const EnsArgs &a, unsigned char *smem, uint64_t *bar,
                                               int stage, int j0, int len)
{
    [[maybe_unused]] constexpr bool MIXED = PR == 1 || PR == 3, EXP = PR == 2;
    const int jt = a.jtile;
    const size_t P = static_cast<size_t>(a.P);
    if (MIXED || EXP) {
        constexpr int NR = EXP ? NCX : NCF;
        float *dst = reinterpret_cast<float *>(smem) + static_cast<size_t>(stage) * NR * jt;
        mbar_expect_tx(&bar[stage], static_cast<uint32_t>(NR * len * 4));
#pragma unroll
        for (int r = 0; r < NR; ++r)
            bulk_g2s(dst + r * jt, a.jf32 + r * P + j0, static_cast<uint32_t>(len * 4), &bar[stage]);
    } else {
        double2 *dst = reinterpret_cast<double2 *>(smem) + static_cast<size_t>(stage) * 5 * jt;
        mbar_expect_tx(&bar[stage], static_cast<uint32_t>(5 * len * 16));
#pragma unroll
        for (int r = 0; r < 5; ++r)
            bulk_g2s(dst + r * jt, a.jb64 + r * P + j0, static_cast<uint32_t>(len * 16), &bar[stage]);
    }
}

// Evaluate active slots [s0, s1) of the system starting at `off` against its
// j-records [j0, j1) (local indices; j0 a multiple of 4), writing the sums of
// slot p to out[q * ostride + p].  The slots go in rounds of at most one per
// thread; a round with fewer slots than threads gives each slot `lanes`
// threads that split its j-tiles, so the last round of a large set and a
// small set keep the block busy (an idle slot would repeat a particle on
// the slow FP64 pipe).  Returns false if a TMA wait timed out (uniform in
// the CTA).
template <int PR>
__device__ bool eval_share(const EnsArgs &a, int off, int j0, int j1, int s0, int s1, double *out,
                           size_t ostride, unsigned char *smem, uint64_t *bar, unsigned &seq)
{
    [[maybe_unused]] constexpr bool MIXED = PR == 1 || PR == 3, EXP = PR == 2;
    const int T = blockDim.x, tid = threadIdx.x, jt = a.jtile;
    if (s1 <= s0)
        return true;
    const size_t P = static_cast<size_t>(a.P);
    const int nj = j1 - j0;
    const int ntiles = (nj + jt - 1) / jt;
    constexpr int kRow[12] = {0, 1, 2, 4, 5, 6, 7, 8, 9, 10, 11, 12};
    // the j-records were written by other blocks of the cluster (generic
    // stores, then the cluster barrier); order them before the bulk copies
    if (tid == 0)
        asm volatile("fence.proxy.async.global;" ::: "memory");

    for (int ib = s0; ib < s1;) {
        int lanes = 1;
        while (lanes < 32 && (T / (2 * lanes)) >= s1 - ib)
            lanes *= 2;
        const int slots = T / lanes, slot = tid / lanes, lj = tid - slot * lanes;
        const int p = ib + slot;
        const bool valid = p < s1;
        const int i = a.act[off + (valid ? p : s1 - 1)];
        double acc[9];
        for (int q = 0; q < 9; ++q)
            acc[q] = 0.0;
        // i-particle data (the same predicted records the j-loop reads)
        float2 ni[12];
        float hi[9], lo[9];
        ExI<float2> nie;
        double xi = 0, yi = 0, zi = 0, vxi = 0, vyi = 0, vzi = 0, axi = 0, ayi = 0, azi = 0;
        if (EXP) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                nie.x[k] = {f2(-a.jf32[k * P + i]), f2(-a.jf32[(3 + k) * P + i])};
                nie.v[k] = {f2(-a.jf32[(6 + k) * P + i]), f2(-a.jf32[(9 + k) * P + i])};
                nie.a[k] = {f2(-a.jf32[(12 + k) * P + i]), f2(-a.jf32[(15 + k) * P + i])};
            }
        } else if (MIXED) {
#pragma unroll
            for (int q = 0; q < 12; ++q)
                ni[q] = f2(-a.jf32[kRow[q] * P + i]);
#pragma unroll
            for (int q = 0; q < 9; ++q)
                hi[q] = lo[q] = 0.0f;
        } else {
            const double2 r0 = a.jb64[i], r1 = a.jb64[P + i], r2 = a.jb64[2 * P + i];
            const double2 r3 = a.jb64[3 * P + i], r4 = a.jb64[4 * P + i];
            xi = r0.x; yi = r0.y; zi = r1.x;
            vxi = r2.x; vyi = r2.y; vzi = r3.x;
            axi = r3.y; ayi = r4.x; azi = r4.y;
        }
        if (tid == 0)
            for (int q = 0; q < min(2, ntiles); ++q)
                issue_ens_tile<PR>(a, smem, bar, (seq + q) & 1, off + j0 + q * jt, min(jt, nj - q * jt));
        for (int tl = 0; tl < ntiles; ++tl) {
            const unsigned sq = seq + tl;
            const int stg = sq & 1;
            const bool ok = mbar_wait_bounded(&bar[stg], (sq >> 1) & 1, kWaitLimitNs);
            if (!__syncthreads_and(ok)) {
                if (tid == 0) {
                    for (int u = tl; u < min(tl + 2, ntiles); ++u)
                        mbar_wait_bounded(&bar[(seq + u) & 1], ((seq + u) >> 1) & 1, kWaitLimitNs);
                    atomicOr(&a.ctl->err, NB_ERR_TIMEOUT);
                }
                return false;
            }
            const int len = min(jt, nj - tl * jt);
            if (EXP) {
                const float *s = reinterpret_cast<const float *>(smem) + static_cast<size_t>(stg) * NCX * jt;
                const float e2h = __double2float_rn(a.eps2);
                const ff::FF<float2> eps2x = {f2(e2h), f2(__double2float_rn(a.eps2 - static_cast<double>(e2h)))};
                ff::FF<float2> part[9];
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    part[q] = {f2(0.0f), f2(0.0f)};
                for (int jj = 2 * lj; jj < len; jj += 2 * lanes) {
                    float2 c[NCX];
#pragma unroll
                    for (int r = 0; r < NCX; ++r)
                        c[r] = *reinterpret_cast<const float2 *>(s + r * jt + jj);
                    pair_ex(c, nie, eps2x, part);
                }
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    acc[q] += (static_cast<double>(part[q].h.x) + static_cast<double>(part[q].l.x)) +
                              (static_cast<double>(part[q].h.y) + static_cast<double>(part[q].l.y));
            } else if (MIXED) {
                const float *s = reinterpret_cast<const float *>(smem) + static_cast<size_t>(stg) * NCF * jt;
                // FP32 running sums over at most kMixedFoldJ j per lane
                for (int f0 = 0; f0 < len; f0 += kMixedFoldJ * lanes) {
                    const int f1 = min(len, f0 + kMixedFoldJ * lanes);
                    float2 part[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q)
                        part[q] = f2(0.0f);
                    for (int jj = f0 + 4 * lj; jj < f1; jj += 4 * lanes) {
                        float2 c0[NCF], c1[NCF];
#pragma unroll
                        for (int r = 0; r < NCF; ++r) {
                            const float4 w = *reinterpret_cast<const float4 *>(s + r * jt + jj);
                            c0[r] = make_float2(w.x, w.y);
                            c1[r] = make_float2(w.z, w.w);
                        }
                        pair_mixed2(c0, ni, f2(static_cast<float>(a.eps2)), part);
                        pair_mixed2(c1, ni, f2(static_cast<float>(a.eps2)), part);
                    }
#pragma unroll
                    for (int q = 0; q < 9; ++q)
                        two_sum_acc(hi[q], lo[q], __fadd_rn(part[q].x, part[q].y));
                }
            } else {
                const double2 *s = reinterpret_cast<const double2 *>(smem) + static_cast<size_t>(stg) * 5 * jt;
                double part[9];
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    part[q] = 0.0;
                for (int jj = lj; jj < len; jj += lanes)
                    pair_fp64(s[jj], s[jt + jj], s[2 * jt + jj], s[3 * jt + jj], s[4 * jt + jj], xi, yi,
                              zi, vxi, vyi, vzi, axi, ayi, azi, a.eps2, part);
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    acc[q] += part[q];
            }
            __syncthreads();
            if (tid == 0 && tl + 2 < ntiles)
                issue_ens_tile<PR>(a, smem, bar, stg, off + j0 + (tl + 2) * jt, min(jt, nj - (tl + 2) * jt));
        }
        seq += ntiles;
        if (MIXED)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                acc[q] = static_cast<double>(hi[q]) + static_cast<double>(lo[q]);
        for (int o = lanes >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        if (valid && lj == 0)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                out[static_cast<size_t>(q) * ostride + p] = acc[q];
        ib += slots;
    }
    return true;
}

// Corrector, interpolation and new step of particle i at time tn, with its
// new acceleration, jerk and snap f[0..8]: the FP64 corrector a context uses
// (so an ensemble takes a context's decisions), with the ensemble's
// step-criterion noise floor (nb_config.step_noise).
__device__ __forceinline__ void correct_one(const EnsArgs &a, int i, double tn, const double (&f)[9])
{
    correct_particle_fp64(a.st, a.t, a.dt, static_cast<size_t>(a.P), i, tn, f, a.eta, a.dt_min, a.dt_max,
                          a.dt_shared, a.ctl, a.noise);
}

// |v| of a 3-vector in FP32 without overflow of the squares.
__device__ __forceinline__ float norm3f(float x, float y, float z)
{
    const float m = fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z)));
    if (m == 0.0f)
        return 0.0f;
    const float r = 1.0f / m;
    const float u = x * r, v = y * r, w = z * r;
    return m * sqrtf(fmaf(u, u, fmaf(v, v, w * w)));
}

// NB_MIXED32 ensembles: the same corrector, interpolation and step with the
// arithmetic in FP32 (the forces carry FP32 pair rounding already, about
// 1e-7 of each sum's condition number): the velocity and position
// increments are formed in FP32 and added to the FP64 state, the crackle,
// pop and a^(5) of the quintic and the Aarseth criterion use FP32 copies of
// the old derivatives.  h = tn - t_i is a power of two, so 1/h is exact.
__device__ void correct_one_mixed(const EnsArgs &a, int i, double tn, const double (&f)[9])
{
    const size_t P = static_cast<size_t>(a.P);
    const float h = __double2float_rn(tn - a.t[i]);
    const float ih = 1.0f / h;
    const float ih3 = ih * ih * ih;
    float an[3], jn[3], sn[3], cn[3], dn[3], en[3], ao[3], jo[3], so[3];
    bool finite = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float a0 = a.st32[(3 + d) * P + i], j0 = a.st32[(6 + d) * P + i], s0 = a.st32[(9 + d) * P + i];
        ao[d] = a0;
        jo[d] = j0;
        so[d] = s0;
        const float a1 = __double2float_rn(f[d]), j1 = __double2float_rn(f[3 + d]);
        const float s1 = __double2float_rn(f[6 + d]);
        const float v0f = a.st32[d * P + i];
        const float dv = h * fmaf(h, fmaf(h, (s0 + s1) * (1.0f / 120.0f), -(j1 - j0) * 0.1f), 0.5f * (a0 + a1));
        const float v1f = v0f + dv;
        const float dx = h * fmaf(h, fmaf(h, (j0 + j1) * (1.0f / 120.0f), -(a1 - a0) * 0.1f), 0.5f * (v0f + v1f));
        double *px = a.st + (F_X * 3 + d) * P + i, *pv = a.st + (F_V * 3 + d) * P + i;
        const double v1 = *pv + static_cast<double>(dv);
        const double x1 = *px + static_cast<double>(dx);
        const float R1 = a1 - fmaf(h, fmaf(0.5f * h, s0, j0), a0);
        const float R2 = h * (j1 - fmaf(h, s0, j0));
        const float R3 = h * h * (s1 - s0);
        const float c1 = (60.0f * R1 - 36.0f * R2 + 9.0f * R3) * ih3;
        const float d1 = (360.0f * R1 - 192.0f * R2 + 36.0f * R3) * ih3 * ih;
        const float e1 = (720.0f * R1 - 360.0f * R2 + 60.0f * R3) * ih3 * ih * ih;
        finite = finite && isfinite(x1) && isfinite(v1) && isfinite(c1);
        *px = x1;
        *pv = v1;
        a.st[(F_A * 3 + d) * P + i] = f[d];
        a.st[(F_J * 3 + d) * P + i] = f[3 + d];
        a.st[(F_S * 3 + d) * P + i] = f[6 + d];
        a.st[(F_C * 3 + d) * P + i] = static_cast<double>(c1);
        store_xv32(a, i, d, x1, v1);
        a.st32[(3 + d) * P + i] = a1;
        a.st32[(6 + d) * P + i] = j1;
        a.st32[(9 + d) * P + i] = s1;
        a.st32[(12 + d) * P + i] = c1;
        an[d] = a1;
        jn[d] = j1;
        sn[d] = s1;
        cn[d] = c1;
        dn[d] = d1;
        en[d] = e1;
    }
    a.t[i] = tn;
    bool hit = false;
    if (a.dt_shared > 0.0) {
        a.dt[i] = a.dt_shared;
    } else {
        // generalised Aarseth criterion eta (A1 / A4)^(1/3); with a noise
        // level, crackle, pop and a^(5) less their rounding floors (as in
        // correct_particle_fp64)
        const float na1 = norm3f(an[0], an[1], an[2]), nj1 = norm3f(jn[0], jn[1], jn[2]);
        const float ns1 = norm3f(sn[0], sn[1], sn[2]);
        float nc = norm3f(cn[0], cn[1], cn[2]), nd = norm3f(dn[0], dn[1], dn[2]);
        float ne = norm3f(en[0], en[1], en[2]);
        if (a.noise > 0.0) {
            const float z = static_cast<float>(a.noise);
            const float o_a = norm3f(ao[0], ao[1], ao[2]), o_j = norm3f(jo[0], jo[1], jo[2]);
            const float o_s = norm3f(so[0], so[1], so[2]);
            const float s1f = z * (na1 + o_a + h * (o_j + 0.5f * h * o_s));
            const float s2f = z * h * (nj1 + o_j + h * o_s);
            const float s3f = z * h * h * (ns1 + o_s);
            nc = fmaxf(nc - (60.0f * s1f + 36.0f * s2f + 9.0f * s3f) * ih3, 0.0f);
            nd = fmaxf(nd - (360.0f * s1f + 192.0f * s2f + 36.0f * s3f) * ih3 * ih, 0.0f);
            ne = fmaxf(ne - (720.0f * s1f + 360.0f * s2f + 60.0f * s3f) * ih3 * ih * ih, 0.0f);
        }
        const float A1 = sqrtf(na1) * sqrtf(ns1) + nj1;
        const float A4 = sqrtf(nc) * sqrtf(ne) + nd;
        // A1 = A4 = 0: no force, no bound (dt_max), as in aarseth_dt()
        const float crit = (A1 == 0.0f && A4 == 0.0f) ? INFINITY : static_cast<float>(a.eta) * cbrtf(A1 / A4);
        a.dt[i] = quantise(static_cast<double>(crit), a.dt[i], tn, a.dt_min, a.dt_max, &hit);
    }
    if (hit)
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctl->floor_hits), 1ull);
    if (!finite)
        atomicOr(&a.ctl->err, NB_ERR_NONFINITE);
}

template <int PR>
__device__ __forceinline__ void correct_particle(const EnsArgs &a, int i, double tn, const double (&f)[9])
{
    [[maybe_unused]] constexpr bool MIXED = PR == 1 || PR == 3, EXP = PR == 2;
    if (PR == 3)
        correct_one_mixed(a, i, tn, f);
    else
        correct_one(a, i, tn, f);
}

// Small active sets (at most small_set(PR) particles, the usual case once close
// pairs sit at small steps): every block evaluates the whole active set
// against its own slice of the system, just predicted by itself, and leaves
// 9 partial sums per active particle in shared memory; the block that owns
// a particle adds the cluster's partials in rank order and corrects it.
// FP64 and EX: up to 128 (and at most the block's thread count), so that
// moderate sets also take this path, where every CTA works on its own
// j-slice and the i-values sit in shared memory.  Mixed: 16, which keeps
// the static shared memory small beside the mixed path's long j-tiles (two
// blocks per SM); its steps with more active particles take the j-split
// large-set path, which is as well balanced.
constexpr int kSmallMax = 128;
__host__ __device__ constexpr int small_set(int pr) { return pr == 1 || pr == 3 ? 16 : kSmallMax; }

// i-values of the small active set: FP64 x, v, a; in mixed precision the
// same slots hold 12 negated FP32 values (x_hi, x_lo, v, a) of the record the
// predictor writes for particle i.
template <int PR>
__device__ __forceinline__ void store_ivalues(const EnsArgs &a, int i, double tn, double *iv)
{
    [[maybe_unused]] constexpr bool MIXED = PR == 1 || PR == 3, EXP = PR == 2;
    if (MIXED) {
        MixedRec r;
        mixed_record<PR>(a, i, tn, r);
        float *f = reinterpret_cast<float *>(iv);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            f[k] = -r.xh[k];
            f[3 + k] = -r.xl[k];
            f[6 + k] = -r.v[k];
            f[9 + k] = -r.a[k];
        }
    } else if (EXP) {
        // 18 negated FP32 values: hi then lo of x, v, a (the j-record's split)
        Taylor p[3];
        predict_one(a, i, tn, p);
        float *f = reinterpret_cast<float *>(iv);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double q[3] = {p[k].x, p[k].v, p[k].a};
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const float h = __double2float_rn(q[g]);
                f[6 * g + k] = -h;
                f[6 * g + 3 + k] = -__double2float_rn(q[g] - static_cast<double>(h));
            }
        }
    } else {
        Taylor p[3];
        predict_one(a, i, tn, p);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            iv[k] = p[k].x;
            iv[3 + k] = p[k].v;
            iv[6 + k] = p[k].a;
        }
    }
}

// Partial sums of the K active particles (i-values in iv) over the j of
// [lo, hi), written to part[K][9].  The j are predicted to tn chunk by chunk
// straight into shared memory (cap records per chunk, the layout of the
// evaluation buffer: 13 or 20 FP32 rows, or 5 rows of double2), so the sums read
// on-chip data only.  L = T / K2 lanes per active particle (K2 the power of
// two >= K); lanes take every L-th j (pair of j in mixed precision) and are
// combined in a fixed order.
template <int PR>
__device__ void eval_small(const EnsArgs &a, int lo, int hi, double tn, int K, const double (*iv)[9],
                           double (*part)[9], double (*wred)[9], unsigned char *smem, int cap)
{
    [[maybe_unused]] constexpr bool MIXED = PR == 1 || PR == 3, EXP = PR == 2;
    const int T = blockDim.x, tid = threadIdx.x;
    int K2 = 1;
    while (K2 < K)
        K2 <<= 1;
    const int L = T / K2;
    const int g = tid / L, lane = tid - g * L;
    const bool valid = g < K;
    const int gi = valid ? g : 0;
    double acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q)
        acc[q] = 0.0;
    float2 ni[12];
    float2 pt[9];
    float ah[9], al[9];  // mixed: compensated (hi, lo) running sums
#pragma unroll
    for (int q = 0; q < 9; ++q)
        ah[q] = al[q] = 0.0f;
    int cnt = 0;
    ExI<float2> nie;
    ff::FF<float2> px[9];
    if (EXP) {
        const float *ivf = reinterpret_cast<const float *>(iv[gi]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            nie.x[k] = {f2(ivf[k]), f2(ivf[3 + k])};
            nie.v[k] = {f2(ivf[6 + k]), f2(ivf[9 + k])};
            nie.a[k] = {f2(ivf[12 + k]), f2(ivf[15 + k])};
        }
#pragma unroll
        for (int q = 0; q < 9; ++q)
            px[q] = {f2(0.0f), f2(0.0f)};
    }
    if (MIXED) {
        const float *ivf = reinterpret_cast<const float *>(iv[gi]);
#pragma unroll
        for (int q = 0; q < 12; ++q)
            ni[q] = f2(ivf[q]);
#pragma unroll
        for (int q = 0; q < 9; ++q)
            pt[q] = f2(0.0f);
    }
    const float2 eps2f = f2(static_cast<float>(a.eps2));
    float *sf = reinterpret_cast<float *>(smem);
    double2 *sd = reinterpret_cast<double2 *>(smem);
    for (int b = lo; b < hi; b += cap) {
        const int len = min(cap, hi - b);
        for (int u = tid; u < len; u += T) {
            const double mj = a.m[b + u];
            if (MIXED) {
                MixedRec r;
                mixed_record<PR>(a, b + u, tn, r);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    sf[k * cap + u] = r.xh[k];
                    sf[(4 + k) * cap + u] = r.xl[k];
                    sf[(7 + k) * cap + u] = r.v[k];
                    sf[(10 + k) * cap + u] = r.a[k];
                }
                sf[3 * cap + u] = __double2float_rn(mj);
            } else if (EXP) {
                Taylor p[3];
                predict_one(a, b + u, tn, p);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double q[3] = {p[k].x, p[k].v, p[k].a};
#pragma unroll
                    for (int gg = 0; gg < 3; ++gg) {
                        const float h = __double2float_rn(q[gg]);
                        sf[(6 * gg + k) * cap + u] = h;
                        sf[(6 * gg + 3 + k) * cap + u] = __double2float_rn(q[gg] - static_cast<double>(h));
                    }
                }
                const float mh = __double2float_rn(mj);
                sf[18 * cap + u] = mh;
                sf[19 * cap + u] = __double2float_rn(mj - static_cast<double>(mh));
            } else {
                Taylor p[3];
                predict_one(a, b + u, tn, p);
                sd[u] = make_double2(p[0].x, p[1].x);
                sd[cap + u] = make_double2(p[2].x, mj);
                sd[2 * cap + u] = make_double2(p[0].v, p[1].v);
                sd[3 * cap + u] = make_double2(p[2].v, p[0].a);
                sd[4 * cap + u] = make_double2(p[1].a, p[2].a);
            }
        }
        __syncthreads();
        if (EXP) {
            const float e2h = __double2float_rn(a.eps2);
            const ff::FF<float2> eps2x = {f2(e2h), f2(__double2float_rn(a.eps2 - static_cast<double>(e2h)))};
            for (int jj = 2 * lane; jj < len; jj += 2 * L) {
                float2 c[NCX];
                if (jj + 1 < len) {
#pragma unroll
                    for (int r = 0; r < NCX; ++r)
                        c[r] = *reinterpret_cast<const float2 *>(sf + r * cap + jj);
                } else {
                    // odd tail: the second half repeats the first j with no mass
#pragma unroll
                    for (int r = 0; r < NCX; ++r) {
                        const float x0 = sf[r * cap + jj];
                        c[r] = make_float2(x0, r >= 18 ? 0.0f : x0);
                    }
                }
                pair_ex(c, nie, eps2x, px);
                if (++cnt == 32) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        acc[q] += (static_cast<double>(px[q].h.x) + static_cast<double>(px[q].l.x)) +
                                  (static_cast<double>(px[q].h.y) + static_cast<double>(px[q].l.y));
                        px[q] = {f2(0.0f), f2(0.0f)};
                    }
                    cnt = 0;
                }
            }
        } else if (MIXED) {
            for (int jj = 2 * lane; jj < len; jj += 2 * L) {
                float2 c[NCF];
                if (jj + 1 < len) {
#pragma unroll
                    for (int r = 0; r < NCF; ++r)
                        c[r] = *reinterpret_cast<const float2 *>(sf + r * cap + jj);
                } else {
                    // odd tail: the second half repeats the first j with no mass
#pragma unroll
                    for (int r = 0; r < NCF; ++r) {
                        const float x0 = sf[r * cap + jj];
                        c[r] = make_float2(x0, r == 3 ? 0.0f : x0);
                    }
                }
                pair_mixed2(c, ni, eps2f, pt);
                if (++cnt == 32) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        two_sum_acc(ah[q], al[q], __fadd_rn(pt[q].x, pt[q].y));
                        pt[q] = f2(0.0f);
                    }
                    cnt = 0;
                }
            }
        } else {
            const double *v = iv[gi];
            for (int jj = lane; jj < len; jj += L)
                pair_fp64(sd[jj], sd[cap + jj], sd[2 * cap + jj], sd[3 * cap + jj], sd[4 * cap + jj], v[0],
                          v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8], a.eps2, acc);
        }
        __syncthreads();
    }
    const int w = tid >> 5;
    const int span = L < 32 ? L : 32;  // lanes combined by shuffles
    if (EXP)
#pragma unroll
        for (int q = 0; q < 9; ++q)
            acc[q] += (static_cast<double>(px[q].h.x) + static_cast<double>(px[q].l.x)) +
                      (static_cast<double>(px[q].h.y) + static_cast<double>(px[q].l.y));
    if (MIXED) {
        // fixed-order double-word sums across the lanes; one FP64 conversion
        // per group (or warp) leader
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            two_sum_acc(ah[q], al[q], __fadd_rn(pt[q].x, pt[q].y));
            for (int o = span >> 1; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, ah[q], o);
                const float ol = __shfl_xor_sync(0xffffffffu, al[q], o);
                two_sum_acc(ah[q], al[q], oh);
                al[q] = __fadd_rn(al[q], ol);
            }
        }
        if ((tid & (span - 1)) == 0)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                acc[q] = static_cast<double>(ah[q]) + static_cast<double>(al[q]);
    } else {
        for (int o = span >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    }
    if (L <= 32) {
        if (valid && lane == 0)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                part[g][q] = acc[q];
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
                double sum = 0.0;
                for (int u = 0; u < wpg; ++u)
                    sum += wred[tid * wpg + u][q];
                part[tid][q] = sum;
            }
    }
    // the chunk area is also a TMA destination in later steps
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
}

// Start-up stores for slots [s0, s1) (all particles, in order).
__device__ void init_share(const EnsArgs &a, int off, int s0, int s1, int pass)
{
    const size_t P = static_cast<size_t>(a.P);
    for (int k = s0 + threadIdx.x; k < s1; k += blockDim.x) {
        const int i = off + k;
        if (pass == 0) {
            for (int d = 0; d < 3; ++d) {
                a.st[(F_A * 3 + d) * P + i] = a.anew[(0 + d) * P + i];
                a.st[(F_J * 3 + d) * P + i] = a.anew[(3 + d) * P + i];
                if (a.st32) {
                    a.st32[(3 + d) * P + i] = __double2float_rn(a.anew[(0 + d) * P + i]);
                    a.st32[(6 + d) * P + i] = __double2float_rn(a.anew[(3 + d) * P + i]);
                }
            }
            continue;
        }
        double na = 0, nj = 0, ns = 0;
        for (int d = 0; d < 3; ++d) {
            const double av = a.st[(F_A * 3 + d) * P + i], jv = a.st[(F_J * 3 + d) * P + i];
            const double sv = a.anew[(6 + d) * P + i];
            a.st[(F_S * 3 + d) * P + i] = sv;
            a.st[(F_C * 3 + d) * P + i] = 0.0;
            if (a.st32) {
                a.st32[(9 + d) * P + i] = __double2float_rn(sv);
                a.st32[(12 + d) * P + i] = 0.0f;
            }
            na = fma(av, av, na);
            nj = fma(jv, jv, nj);
            ns = fma(sv, sv, ns);
        }
        bool hit = false;
        if (a.dt_shared > 0.0) {
            a.dt[i] = a.dt_shared;
        } else {
            a.dt[i] = quantise(initial_dt(sqrt(na), nj, ns, a.eta_s), -1.0, 0.0, a.dt_min, a.dt_max, &hit);
        }
        if (hit)
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctl->floor_hits), 1ull);
    }
}

// Step log (nb_ensemble_set_log), written by rank 0 of the system's
// cluster: the step's system, time and active count, and the active
// particles' indices within the system (list[] holds ensemble indices).
// Entries beyond the capacities are counted, not kept.
__device__ void log_step(const EnsArgs &a, int c, double tn, int total, const int32_t *list, int off,
                         long long *s_ip)
{
    if (threadIdx.x == 0) {
        const unsigned long long e = atomicAdd(&a.log_cnt[0], 1ull);
        const unsigned long long ip = atomicAdd(&a.log_cnt[1], static_cast<unsigned long long>(total));
        const bool keep = ip + static_cast<unsigned long long>(total) <=
                          static_cast<unsigned long long>(a.idx_cap);
        if (e < static_cast<unsigned long long>(a.log_cap)) {
            a.log_sys[e] = c;
            a.log_t[e] = tn;
            a.log_n[e] = total;
            a.log_off[e] = keep ? static_cast<long long>(ip) : -1;
        }
        *s_ip = keep ? static_cast<long long>(ip) : -1;
    }
    __syncthreads();
    const long long ip = *s_ip;
    if (ip >= 0)
        for (int k = threadIdx.x; k < total; k += blockDim.x)
            a.log_idx[ip + k] = list[k] - off;
    __syncthreads();
}

template <int PR>
__global__ void __launch_bounds__(kEnsThreads, 1) ensemble_kernel(EnsArgs a)
{
    [[maybe_unused]] constexpr bool MIXED = PR == 1 || PR == 3, EXP = PR == 2;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double red_d[32];
    __shared__ int red_i[32];
    __shared__ int s_job;
    __shared__ int s_fail;
    __shared__ double s_min2[2];
    __shared__ int s_cnt2[2];
    constexpr int KS = small_set(PR);
    __shared__ int s_cand[2][KS];
    __shared__ int s_act[KS];
    __shared__ int s_rcnt[kMaxCluster];
    __shared__ double s_iv[KS][9];
    __shared__ double s_part[KS][9];
    __shared__ double s_wred[kEnsThreads / 32][9];
    __shared__ long long s_log_ip;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = static_cast<int>(cl.block_rank());
    const int G = static_cast<int>(cl.num_blocks());
    const int tid = threadIdx.x;
    unsigned seq = 0;  // TMA stage sequence (continues across chunks and systems)
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        s_fail = 0;
    }
    __syncthreads();

    for (;;) {
        if (rank == 0 && tid == 0)
            s_job = atomicAdd(a.queue, 1);
        cl.sync();
        const int job = *cl.map_shared_rank(&s_job, 0);
        int fail_any = 0;
        for (int r = 0; r < G; ++r)
            fail_any |= *cl.map_shared_rank(&s_fail, r);
        cl.sync();
        if (job >= a.nc || fail_any)
            break;
        const int c = a.order[job];
        const int off = a.off[c], n = a.cnt[c];
        const int nj = (MIXED || EXP) ? (n + 3) / 4 * 4 : n;
        const int per = (n + G - 1) / G;
        const int lo = off + min(n, rank * per), hi = off + min(n, (rank + 1) * per);

        if (a.mode == 1) {
            for (int k = lo - off + tid; k < hi - off; k += blockDim.x)
                a.act[off + k] = off + k;
            for (int pass = 0; pass < 2; ++pass) {
                predict_slice<PR>(a, lo, hi, 0.0);
                cl.sync();
                const bool ok = eval_share<PR>(a, off, 0, nj, lo - off, hi - off, a.anew + off,
                                               static_cast<size_t>(a.P), smem, bar, seq);
                if (!ok && tid == 0)
                    s_fail = 1;
                __syncthreads();
                init_share(a, off, lo - off, hi - off, pass);
                cl.sync();
            }
            continue;
        }

        int64_t steps = 0;
        const int T = blockDim.x;
        const int per_t = (hi - lo + T - 1) / T;  // contiguous chunk per thread (ordered scans)
        const int c0 = min(hi, lo + tid * per_t), c1 = min(hi, c0 + per_t);
        for (;;) {
            const int par = static_cast<int>(steps & 1);
            // schedule, one pass: the slice's earliest t_i + dt_i and how many
            // particles reach it; a small set is listed in shared memory
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
            const double mb = block_min(mt, red_d);
            const int mine = (mt == mb) ? ct : 0;
            int tot_b = 0;
            const int ex = block_exclusive_scan(mine, red_i, &tot_b);
            const int small_max = min(KS, T);
            if (mine > 0 && tot_b <= small_max) {
                int pos = ex;
                for (int i = c0; i < c1; ++i)
                    if (a.t[i] + a.dt[i] == mb)
                        s_cand[par][pos++] = i;
            }
            if (tid == 0) {
                s_min2[par] = mb;
                s_cnt2[par] = tot_b;
            }
            cl.sync();
            double tn = INFINITY;
            int fail = 0;
            for (int r = 0; r < G; ++r) {
                tn = fmin(tn, *cl.map_shared_rank(&s_min2[par], r));
                fail |= *cl.map_shared_rank(&s_fail, r);
            }
            if (tn > a.t_end || fail)
                break;
            int total = 0, prefix = 0;
            for (int r = 0; r < G; ++r) {
                const int v = (*cl.map_shared_rank(&s_min2[par], r) == tn) ? *cl.map_shared_rank(&s_cnt2[par], r) : 0;
                prefix += r < rank ? v : 0;
                total += v;
            }
            if (total <= small_max) {
                // active list in ascending order from the blocks' lists, and
                // its predicted values (the arithmetic of the j-records)
                if (tid < G) {
                    const int v = (*cl.map_shared_rank(&s_min2[par], tid) == tn) ? *cl.map_shared_rank(&s_cnt2[par], tid) : 0;
                    s_rcnt[tid] = v;
                }
                __syncthreads();
                for (int k = tid; k < total; k += T) {
                    int base = 0, r = 0;
                    while (k >= base + s_rcnt[r])
                        base += s_rcnt[r++];
                    const int i = *cl.map_shared_rank(&s_cand[par][k - base], r);
                    s_act[k] = i;
                    store_ivalues<PR>(a, i, tn, s_iv[k]);
                }
                __syncthreads();
                if (a.log_cnt && rank == 0)
                    log_step(a, c, tn, total, s_act, off, &s_log_ip);
                eval_small<PR>(a, lo, hi, tn, total, s_iv, s_part, s_wred, smem, 2 * a.jtile);
                cl.sync();
                for (int k = tid; k < total; k += T) {
                    const int i = s_act[k];
                    if (i < lo || i >= hi)
                        continue;
                    double f[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q)
                        f[q] = 0.0;
                    for (int r = 0; r < G; ++r) {
                        const double *pr = cl.map_shared_rank(&s_part[k][0], r);
#pragma unroll
                        for (int q = 0; q < 9; ++q)
                            f[q] += pr[q];
                    }
                    correct_particle<PR>(a, i, tn, f);
                }
                __syncthreads();
            } else {
                if (mine > 0 && mb == tn) {
                    int pos = prefix + ex;
                    for (int i = c0; i < c1; ++i)
                        if (a.t[i] + a.dt[i] == tn)
                            a.act[off + pos++] = i;
                }
                predict_slice<PR>(a, lo, hi, tn);
                cl.sync();
                if (a.log_cnt && rank == 0)
                    log_step(a, c, tn, total, a.act + off, off, &s_log_ip);
                // j-split: this block's share of the j-records (4-aligned)
                // against every active particle, partial sums to the
                // cluster's scratch; then each block adds, in rank order,
                // the partials of its share of the active particles and
                // corrects them
                const int per4 = ((nj + G - 1) / G + 3) / 4 * 4;
                const int jl = min(nj, rank * per4), jh = min(nj, jl + per4);
                const size_t gs = static_cast<size_t>(a.gstride);
                double *gcl = a.gpart + static_cast<size_t>(blockIdx.x / G) * G * 9 * gs;
                const bool ok = eval_share<PR>(a, off, jl, jh, 0, total, gcl + rank * 9 * gs, gs, smem, bar, seq);
                if (!ok && tid == 0)
                    s_fail = 1;
                cl.sync();
                int bad = 0;
                for (int r = 0; r < G; ++r)
                    bad |= *cl.map_shared_rank(&s_fail, r);
                const int q = (total + G - 1) / G;
                const int s0 = min(total, rank * q), s1 = min(total, s0 + q);
                for (int k = s0 + tid; k < s1 && !bad; k += T) {
                    double f[9];
#pragma unroll
                    for (int u = 0; u < 9; ++u)
                        f[u] = 0.0;
                    for (int r = 0; r < G; ++r)
#pragma unroll
                        for (int u = 0; u < 9; ++u)
                            f[u] += gcl[(static_cast<size_t>(r) * 9 + u) * gs + k];
                    correct_particle<PR>(a, a.act[off + k], tn, f);
                }
                cl.sync();
            }
            ++steps;
            if (rank == 0 && tid == 0)
                atomicAdd(a.inter, static_cast<unsigned long long>(total) * static_cast<unsigned long long>(n));
        }
        if (rank == 0 && tid == 0)
            a.steps[c] = steps;
        cl.sync();
    }
}

nb_status efail(nb_ensemble *e, nb_status s, const std::string &msg)
{
    e->err = msg;
    return s;
}

nb_status ecuda(nb_ensemble *e, cudaError_t c, const char *where)
{
    e->dead = true;
    e->err = std::string(where) + ": " + cudaGetErrorString(c);
    return NB_ECUDA;
}

#define ECU(e, call)                                \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess)                      \
            return ecuda((e), e_, #call);           \
    } while (0)

// Kernel instantiation of a precision: 0 FP64, 1 mixed, 2 EX, 3 mixed with
// an FP32 state copy.
int ens_kind(const nb_ensemble *e)
{
    switch (e->cfg.precision) {
    case NB_MIXED: return 1;
    case NB_EX: return 2;
    case NB_MIXED32: return 3;
    default: return 0;
    }
}

bool ens_mixed(const nb_ensemble *e)
{
    return e->cfg.precision == NB_MIXED || e->cfg.precision == NB_MIXED32;
}

size_t ens_smem(const nb_ensemble *e)
{
    const int k = ens_kind(e);
    return static_cast<size_t>(2) * (k == 1 || k == 3 ? NCF * 4 : (k == 2 ? NCX * 4 : 5 * 16)) * e->jtile;
}

template <int PR>
cudaError_t launch_ens(nb_ensemble *e, const EnsArgs &a, int grid_clusters)
{
    [[maybe_unused]] constexpr bool MIXED = PR == 1 || PR == 3, EXP = PR == 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid_clusters * e->G);
    cfg.blockDim = dim3(e->threads);
    cfg.dynamicSmemBytes = ens_smem(e);
    cfg.stream = e->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = e->G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ensemble_kernel<PR>, a);
}

template <int PR>
cudaError_t max_clusters(nb_ensemble *e, int *out)
{
    [[maybe_unused]] constexpr bool MIXED = PR == 1 || PR == 3, EXP = PR == 2;
    cudaError_t err = cudaFuncSetAttribute(ensemble_kernel<PR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(ens_smem(e)));
    if (err != cudaSuccess)
        return err;
    // clusters of more than 8 blocks need the non-portable size opt-in
    err = cudaFuncSetAttribute(ensemble_kernel<PR>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                               e->G > 8 ? 1 : 0);
    if (err != cudaSuccess)
        return err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(e->G);
    cfg.blockDim = dim3(e->threads);
    cfg.dynamicSmemBytes = ens_smem(e);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = e->G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(out, ensemble_kernel<PR>, &cfg);
}

// Default blocks per system: mixed ensembles 4 (their steps are latency-
// bound); FP64 8; EX, whose steps carry most of the arithmetic at the FP32
// rate, 16 where the device co-schedules clusters of 16 blocks, else 8.
int default_ctas(nb_ensemble *e)
{
    if (ens_mixed(e))
        return 4;
    // FP64: 8 (with the j-split large-set path, smaller clusters run more
    // systems at once and finish the largest ones no later: 256-system
    // config 60.9 s against 66.7 s with 16)
    if (e->cfg.precision == NB_FP64)
        return 8;
    const int keep = e->G;
    e->G = 16;
    int maxc = 0;
    const cudaError_t err = ens_kind(e) == 2 ? max_clusters<2>(e, &maxc) : max_clusters<0>(e, &maxc);
    e->G = keep;
    if (err != cudaSuccess) {
        (void)cudaGetLastError();
        return 8;
    }
    return maxc >= 1 ? 16 : 8;
}

int default_jtile(const nb_ensemble *e) { return ens_mixed(e) ? 1024 : 256; }

template <int PR>
cudaError_t max_clusters(nb_ensemble *e, int *out);

cudaError_t max_clusters_kind(nb_ensemble *e, int *out)
{
    switch (ens_kind(e)) {
    case 1: return max_clusters<1>(e, out);
    case 2: return max_clusters<2>(e, out);
    case 3: return max_clusters<3>(e, out);
    default: return max_clusters<0>(e, out);
    }
}

EnsArgs make_args(nb_ensemble *e, int mode, double t_end)
{
    EnsArgs a;
    a.nc = e->nc;
    a.off = e->d_off;
    a.cnt = e->d_cnt;
    a.order = e->d_order;
    a.P = static_cast<int>(e->P);
    a.st = e->st;
    a.t = e->t;
    a.dt = e->dt;
    a.m = e->m;
    a.jb64 = e->jb64;
    a.jf32 = e->jf32;
    a.st32 = e->st32;
    a.act = e->act;
    a.anew = e->anew;
    a.queue = e->queue;
    a.steps = e->steps;
    a.inter = e->inter;
    a.ctl = e->ctl;
    a.gpart = e->gpart;
    a.gstride = e->nmax4;
    a.log_cnt = e->log_cnt;
    a.log_sys = e->log_sys;
    a.log_n = e->log_n;
    a.log_idx = e->log_idx;
    a.log_t = e->log_t;
    a.log_off = e->log_off;
    a.log_cap = e->log_cap;
    a.idx_cap = e->idx_cap;
    a.t_end = t_end;
    a.eps2 = e->eps * e->eps;
    a.eta = e->cfg.eta;
    a.noise = e->cfg.step_noise;
    a.eta_s = e->cfg.eta_s;
    a.dt_min = e->cfg.dt_min;
    a.dt_max = e->cfg.dt_max;
    a.dt_shared = e->cfg.dt_shared;
    a.mode = mode;
    a.jtile = e->jtile;
    return a;
}

// Clusters in the grid (at most the number the device co-schedules, at most
// one per system) and the j-split scratch for them; call outside stream
// capture (it may allocate).
nb_status prepare_grid(nb_ensemble *e, int *grid)
{
    int maxc = 0;
    ECU(e, max_clusters_kind(e, &maxc));
    if (maxc < 1)
        return efail(e, NB_EINVAL, "ensemble launch shape does not fit on an SM");
    *grid = std::min(maxc, e->nc);
    const size_t need = static_cast<size_t>(*grid) * e->G * 9 * static_cast<size_t>(e->nmax4);
    if (need > e->gpart_cap) {
        cudaFree(e->gpart);
        e->gpart = nullptr;
        e->gpart_cap = 0;
        const cudaError_t c = cudaMalloc(&e->gpart, need * sizeof(double));
        if (c == cudaErrorMemoryAllocation) {
            (void)cudaGetLastError();
            return efail(e, NB_ENOMEM, "no device memory for the ensemble's partial sums");
        }
        ECU(e, c);
        e->gpart_cap = need;
    }
    return NB_OK;
}

// Enqueue one persistent launch (queue reset + kernel) on e->stream; the
// grid was prepared by prepare_grid.
nb_status enqueue_run(nb_ensemble *e, int mode, double t_end, int grid)
{
    const int kind = ens_kind(e);
    ECU(e, cudaMemsetAsync(e->queue, 0, sizeof(int), e->stream));
    const EnsArgs a = make_args(e, mode, t_end);
    cudaError_t le;
    switch (kind) {
    case 1: le = launch_ens<1>(e, a, grid); break;
    case 2: le = launch_ens<2>(e, a, grid); break;
    case 3: le = launch_ens<3>(e, a, grid); break;
    default: le = launch_ens<0>(e, a, grid); break;
    }
    ECU(e, le);
    return NB_OK;
}

nb_status ens_sync(nb_ensemble *e)
{
    ECU(e, cudaMemcpyAsync(e->ctl_h, e->ctl, sizeof(nb_ctl), cudaMemcpyDeviceToHost, e->stream));
    ECU(e, cudaStreamSynchronize(e->stream));
    if (e->ctl_h->err) {
        const int err = e->ctl_h->err;
        ECU(e, cudaMemsetAsync(&e->ctl->err, 0, sizeof(int32_t), e->stream));
        ECU(e, cudaStreamSynchronize(e->stream));
        if (err & NB_ERR_TIMEOUT)
            return efail(e, NB_ETIMEOUT, "a device-side wait timed out in the ensemble launch");
        return efail(e, NB_ENONFINITE, "non-finite value produced on the device");
    }
    return NB_OK;
}

void ens_free_all(nb_ensemble *e)
{
    if (e->exec)
        cudaGraphExecDestroy(e->exec);
    if (e->graph)
        cudaGraphDestroy(e->graph);
    cudaFree(e->d_off);
    cudaFree(e->d_cnt);
    cudaFree(e->d_order);
    cudaFree(e->m);
    cudaFree(e->st);
    cudaFree(e->t);
    cudaFree(e->dt);
    cudaFree(e->anew);
    cudaFree(e->jb64);
    cudaFree(e->jf32);
    cudaFree(e->st32);
    cudaFree(e->gpart);
    cudaFree(e->log_cnt);
    cudaFree(e->log_sys);
    cudaFree(e->log_n);
    cudaFree(e->log_idx);
    cudaFree(e->log_t);
    cudaFree(e->log_off);
    cudaFree(e->act);
    cudaFree(e->queue);
    cudaFree(e->steps);
    cudaFree(e->inter);
    cudaFree(e->ctl);
    if (e->ctl_h)
        cudaFreeHost(e->ctl_h);
    if (e->own_stream && e->stream)
        cudaStreamDestroy(e->stream);
}

bool pow2(double x)
{
    int ex;
    return x > 0 && std::isfinite(x) && std::frexp(x, &ex) == 0.5;
}

}  // namespace

extern "C" {

nb_status nb_ensemble_init(nb_ensemble **out, int32_t n_systems, const int64_t *sizes, const double *m,
                           const double *x, const double *v, double eps, const nb_config *cfg)
{
    if (!out) {
        nb_set_thread_error("out must not be NULL");
        return NB_EINVAL;
    }
    *out = nullptr;
    nb_config cf;
    if (cfg)
        cf = *cfg;
    else
        nb_config_default(&cf);
    if (n_systems < 1 || !sizes || !m || !x || !v) {
        nb_set_thread_error("n_systems >= 1 and non-NULL sizes, m, x, v are required");
        return NB_EINVAL;
    }
    if ((cf.precision != NB_FP64 && cf.precision != NB_MIXED && cf.precision != NB_EX &&
         cf.precision != NB_MIXED32) || !(cf.eta > 0) ||
        !(cf.eta_s > 0) ||
        !pow2(cf.dt_min) || !pow2(cf.dt_max) || cf.dt_min > cf.dt_max ||
        (cf.dt_shared != 0.0 && !pow2(cf.dt_shared)) || !(cf.step_noise >= 0.0) || !(cf.step_noise <= 1e-3)) {
        nb_set_thread_error("invalid configuration");
        return NB_EINVAL;
    }
    const double eps_min = cf.precision != NB_FP64 ? std::ldexp(1.0, -40) : std::ldexp(1.0, -60);
    if (!(eps >= eps_min) || !(eps <= 1e18)) {
        nb_set_thread_error("eps out of range");
        return NB_EINVAL;
    }
    int64_t total = 0, padded = 0;
    for (int c = 0; c < n_systems; ++c) {
        if (sizes[c] < 1) {
            nb_set_thread_error("every system needs at least one particle");
            return NB_EINVAL;
        }
        total += sizes[c];
        padded += (sizes[c] + 3) / 4 * 4;
    }
    if (padded > 0x7fffffffLL / 16) {
        nb_set_thread_error("ensemble too large");
        return NB_EINVAL;
    }
    for (int64_t i = 0; i < total; ++i)
        if (!std::isfinite(m[i]) || m[i] < 0.0) {
            nb_set_thread_error("masses must be finite and >= 0");
            return NB_ENONFINITE;
        }
    for (int64_t i = 0; i < 3 * total; ++i)
        if (!std::isfinite(x[i]) || !std::isfinite(v[i])) {
            nb_set_thread_error("positions and velocities must be finite");
            return NB_ENONFINITE;
        }

    nb_ensemble *e = new nb_ensemble();
    e->cfg = cf;
    e->eps = eps;
    e->nc = n_systems;
    e->P = padded;
    // defaults from shape sweeps on GB300: mixed 4 x 128 threads, j-tile
    // 1024; FP64 and EX 16 (or 8) x 128, j-tile 256 (set below, once the
    // device is known)
    e->jtile = default_jtile(e);
    e->G = ens_mixed(e) ? 4 : 8;
    auto bail = [&](nb_status s) {
        nb_set_thread_error(e->err.c_str());
        ens_free_all(e);
        delete e;
        return s;
    };
#define EI(call)                                              \
    do {                                                      \
        cudaError_t c_ = (call);                              \
        if (c_ != cudaSuccess) {                              \
            ecuda(e, c_, #call);                              \
            return bail(c_ == cudaErrorMemoryAllocation ? NB_ENOMEM : NB_ECUDA); \
        }                                                     \
    } while (0)
    EI(cudaGetDevice(&e->dev));
    if (cf.stream) {
        e->stream = static_cast<cudaStream_t>(cf.stream);
    } else {
        EI(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking));
        e->own_stream = true;
    }
    e->G = default_ctas(e);
    e->off.resize(n_systems);
    e->cnt.resize(n_systems);
    {
        int64_t o = 0;
        for (int c = 0; c < n_systems; ++c) {
            e->off[c] = static_cast<int32_t>(o);
            e->cnt[c] = static_cast<int32_t>(sizes[c]);
            o += (sizes[c] + 3) / 4 * 4;
        }
    }
    for (int c = 0; c < n_systems; ++c)
        e->nmax4 = std::max<int64_t>(e->nmax4, (e->cnt[c] + 3) / 4 * 4);
    std::vector<int32_t> order(n_systems);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return e->cnt[a] > e->cnt[b]; });
    const size_t P = static_cast<size_t>(e->P);
    EI(cudaMalloc(&e->d_off, n_systems * sizeof(int32_t)));
    EI(cudaMalloc(&e->d_cnt, n_systems * sizeof(int32_t)));
    EI(cudaMalloc(&e->d_order, n_systems * sizeof(int32_t)));
    EI(cudaMalloc(&e->m, P * sizeof(double)));
    EI(cudaMalloc(&e->st, 18 * P * sizeof(double)));
    EI(cudaMalloc(&e->t, P * sizeof(double)));
    EI(cudaMalloc(&e->dt, P * sizeof(double)));
    EI(cudaMalloc(&e->anew, 9 * P * sizeof(double)));
    EI(cudaMalloc(&e->act, P * sizeof(int32_t)));
    if (ens_mixed(e)) {
        EI(cudaMalloc(&e->jf32, 13 * P * sizeof(float)));
        EI(cudaMemsetAsync(e->jf32, 0, 13 * P * sizeof(float), e->stream));
        if (cf.precision == NB_MIXED32) {
            EI(cudaMalloc(&e->st32, kSt32Rows * P * sizeof(float)));
            EI(cudaMemsetAsync(e->st32, 0, kSt32Rows * P * sizeof(float), e->stream));
        }
    } else if (cf.precision == NB_EX) {
        EI(cudaMalloc(&e->jf32, NCX * P * sizeof(float)));
        EI(cudaMemsetAsync(e->jf32, 0, NCX * P * sizeof(float), e->stream));
    } else {
        EI(cudaMalloc(&e->jb64, 5 * P * sizeof(double2)));
        EI(cudaMemsetAsync(e->jb64, 0, 5 * P * sizeof(double2), e->stream));
    }
    EI(cudaMalloc(&e->queue, sizeof(int)));
    EI(cudaMalloc(&e->steps, n_systems * sizeof(int64_t)));
    EI(cudaMalloc(&e->inter, sizeof(unsigned long long)));
    EI(cudaMalloc(&e->ctl, sizeof(nb_ctl)));
    EI(cudaMallocHost(&e->ctl_h, sizeof(nb_ctl)));
    std::vector<double> hst(18 * P, 0.0), hm(P, 0.0), ht(P, 0.0);
    {
        int64_t src = 0;
        for (int c = 0; c < n_systems; ++c)
            for (int k = 0; k < e->cnt[c]; ++k, ++src) {
                const size_t i = static_cast<size_t>(e->off[c]) + k;
                hm[i] = m[src];
                for (int d = 0; d < 3; ++d) {
                    hst[(F_X * 3 + d) * P + i] = x[3 * src + d];
                    hst[(F_V * 3 + d) * P + i] = v[3 * src + d];
                }
            }
    }
    EI(cudaMemcpyAsync(e->d_off, e->off.data(), n_systems * sizeof(int32_t), cudaMemcpyHostToDevice, e->stream));
    EI(cudaMemcpyAsync(e->d_cnt, e->cnt.data(), n_systems * sizeof(int32_t), cudaMemcpyHostToDevice, e->stream));
    EI(cudaMemcpyAsync(e->d_order, order.data(), n_systems * sizeof(int32_t), cudaMemcpyHostToDevice, e->stream));
    EI(cudaMemcpyAsync(e->st, hst.data(), 18 * P * sizeof(double), cudaMemcpyHostToDevice, e->stream));
    std::vector<float> h32;
    if (e->st32) {  // FP32 copy of the starting x and v (a, jerk, snap, crackle start at 0)
        h32.assign(kSt32Rows * P, 0.0f);
        for (size_t q = 0; q < 3 * P; ++q) {
            const double xv = hst[F_X * 3 * P + q], vv = hst[F_V * 3 * P + q];
            const float xh = static_cast<float>(xv), vh = static_cast<float>(vv);
            h32[15 * P + q] = xh;
            h32[18 * P + q] = static_cast<float>(xv - static_cast<double>(xh));
            h32[q] = vh;
            h32[21 * P + q] = static_cast<float>(vv - static_cast<double>(vh));
        }
        EI(cudaMemcpyAsync(e->st32, h32.data(), kSt32Rows * P * sizeof(float), cudaMemcpyHostToDevice, e->stream));
    }
    EI(cudaMemcpyAsync(e->m, hm.data(), P * sizeof(double), cudaMemcpyHostToDevice, e->stream));
    EI(cudaMemcpyAsync(e->t, ht.data(), P * sizeof(double), cudaMemcpyHostToDevice, e->stream));
    // padding particles: dt = +inf keeps them out of every schedule
    std::vector<double> hdt(P, INFINITY);
    EI(cudaMemcpyAsync(e->dt, hdt.data(), P * sizeof(double), cudaMemcpyHostToDevice, e->stream));
    EI(cudaMemsetAsync(e->steps, 0, n_systems * sizeof(int64_t), e->stream));
    EI(cudaMemsetAsync(e->inter, 0, sizeof(unsigned long long), e->stream));
    EI(cudaMemsetAsync(e->ctl, 0, sizeof(nb_ctl), e->stream));
    int grid = 0;
    nb_status s = prepare_grid(e, &grid);
    if (s == NB_OK)
        s = enqueue_run(e, 1, 0.0, grid);
    if (s != NB_OK)
        return bail(s);
    e->launches += 1;
    s = ens_sync(e);
    if (s != NB_OK)
        return bail(s);
    *out = e;
    return NB_OK;
#undef EI
}

nb_status nb_ensemble_set_shape(nb_ensemble *e, int32_t ctas_per_system, int32_t threads, int32_t jtile)
{
    if (!e)
        return NB_EINVAL;
    if (e->dead)
        return NB_ECUDA;
    if (threads == 0)
        threads = 128;
    if (jtile == 0)
        jtile = default_jtile(e);
    if (ctas_per_system < 0 || ctas_per_system > kMaxCluster || threads < 64 || threads > kEnsThreads ||
        threads % 32 || jtile < 4 || jtile > 1024 || jtile % 4)
        return efail(e, NB_EINVAL, "ctas_per_system in [0, 16], threads 0 or a multiple of 32 in [64, 256], "
                                   "jtile 0 or a multiple of 4 in [4, 1024]");
    e->threads = threads;
    e->jtile = jtile;
    e->G = ctas_per_system == 0 ? default_ctas(e) : ctas_per_system;
    if (e->exec) {
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
    }
    if (e->graph) {
        cudaGraphDestroy(e->graph);
        e->graph = nullptr;
    }
    e->graph_t_end = -1.0;
    return NB_OK;
}

nb_status nb_ensemble_run(nb_ensemble *e, double t_end, int use_graph)
{
    if (!e)
        return NB_EINVAL;
    if (e->dead)
        return NB_ECUDA;
    const double unit = e->cfg.dt_shared > 0.0 ? e->cfg.dt_shared : e->cfg.dt_max;
    if (!std::isfinite(t_end) || t_end < 0.0 || std::fmod(t_end, unit) != 0.0)
        return efail(e, NB_EINVAL, "t_end must be a non-negative multiple of dt_max (dt_shared)");
    if (!use_graph) {
        int grid = 0;
        nb_status s = prepare_grid(e, &grid);
        if (s == NB_OK)
            s = enqueue_run(e, 0, t_end, grid);
        if (s != NB_OK)
            return s;
        e->launches += 1;
        return ens_sync(e);
    }
    if (!e->exec || e->graph_t_end != t_end) {
        if (e->exec) {
            cudaGraphExecDestroy(e->exec);
            e->exec = nullptr;
        }
        if (e->graph) {
            cudaGraphDestroy(e->graph);
            e->graph = nullptr;
        }
        // occupancy query, attributes and scratch before capture
        int grid = 0;
        nb_status s = prepare_grid(e, &grid);
        if (s != NB_OK)
            return s;
        ECU(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
        s = enqueue_run(e, 0, t_end, grid);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
        if (s != NB_OK) {
            if (g)
                cudaGraphDestroy(g);
            return s;
        }
        ECU(e, ce);
        e->graph = g;
        ECU(e, cudaGraphInstantiate(&e->exec, e->graph, 0));
        e->graph_t_end = t_end;
    }
    ECU(e, cudaGraphLaunch(e->exec, e->stream));
    e->launches += 1;
    return ens_sync(e);
}

nb_status nb_ensemble_get_state(nb_ensemble *e, double *x, double *v, double *a, double *j, double *s,
                                double *c, double *t, double *dt)
{
    if (!e)
        return NB_EINVAL;
    if (e->dead)
        return NB_ECUDA;
    const size_t P = static_cast<size_t>(e->P);
    std::vector<double> hst(18 * P), ht(P), hdt(P);
    ECU(e, cudaMemcpyAsync(hst.data(), e->st, 18 * P * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
    ECU(e, cudaMemcpyAsync(ht.data(), e->t, P * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
    ECU(e, cudaMemcpyAsync(hdt.data(), e->dt, P * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
    nb_status st = ens_sync(e);
    if (st != NB_OK)
        return st;
    double *outs[6] = {x, v, a, j, s, c};
    int64_t dst = 0;
    for (int q = 0; q < e->nc; ++q)
        for (int k = 0; k < e->cnt[q]; ++k, ++dst) {
            const size_t i = static_cast<size_t>(e->off[q]) + k;
            for (int f = 0; f < 6; ++f)
                if (outs[f])
                    for (int d = 0; d < 3; ++d)
                        outs[f][3 * dst + d] = hst[(f * 3 + d) * P + i];
            if (t)
                t[dst] = ht[i];
            if (dt)
                dt[dst] = hdt[i];
        }
    return NB_OK;
}

nb_status nb_ensemble_get_shape(nb_ensemble *e, int32_t *ctas_per_system, int32_t *threads, int32_t *jtile)
{
    if (!e)
        return NB_EINVAL;
    if (ctas_per_system)
        *ctas_per_system = e->G;
    if (threads)
        *threads = e->threads;
    if (jtile)
        *jtile = e->jtile;
    return NB_OK;
}

nb_status nb_ensemble_stats(nb_ensemble *e, int64_t *steps, double *interactions, int64_t *launches)
{
    if (!e)
        return NB_EINVAL;
    if (e->dead)
        return NB_ECUDA;
    unsigned long long it = 0;
    if (steps)
        ECU(e, cudaMemcpyAsync(steps, e->steps, e->nc * sizeof(int64_t), cudaMemcpyDeviceToHost, e->stream));
    ECU(e, cudaMemcpyAsync(&it, e->inter, sizeof(it), cudaMemcpyDeviceToHost, e->stream));
    ECU(e, cudaStreamSynchronize(e->stream));
    if (interactions)
        *interactions = static_cast<double>(it);
    if (launches)
        *launches = e->launches;
    return NB_OK;
}

nb_status nb_ensemble_set_log(nb_ensemble *e, int64_t step_cap, int64_t idx_cap)
{
    if (!e)
        return NB_EINVAL;
    if (e->dead)
        return NB_ECUDA;
    if (step_cap < 0 || idx_cap < 0 || step_cap > (int64_t(1) << 32) || idx_cap > (int64_t(1) << 34))
        return efail(e, NB_EINVAL, "step_cap in [0, 2^32] and idx_cap in [0, 2^34] required");
    ECU(e, cudaStreamSynchronize(e->stream));
    cudaFree(e->log_cnt);
    cudaFree(e->log_sys);
    cudaFree(e->log_n);
    cudaFree(e->log_idx);
    cudaFree(e->log_t);
    cudaFree(e->log_off);
    e->log_cnt = nullptr;
    e->log_sys = e->log_n = e->log_idx = nullptr;
    e->log_t = nullptr;
    e->log_off = nullptr;
    e->log_cap = e->idx_cap = 0;
    // the launch arguments (captured in the graph) change
    if (e->exec) {
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
    }
    if (e->graph) {
        cudaGraphDestroy(e->graph);
        e->graph = nullptr;
    }
    e->graph_t_end = -1.0;
    if (step_cap == 0 && idx_cap == 0)
        return NB_OK;
    const size_t sc = static_cast<size_t>(std::max<int64_t>(1, step_cap));
    const size_t ic = static_cast<size_t>(std::max<int64_t>(1, idx_cap));
    cudaError_t c = cudaMalloc(&e->log_cnt, 2 * sizeof(unsigned long long));
    if (c == cudaSuccess) c = cudaMalloc(&e->log_sys, sc * sizeof(int32_t));
    if (c == cudaSuccess) c = cudaMalloc(&e->log_n, sc * sizeof(int32_t));
    if (c == cudaSuccess) c = cudaMalloc(&e->log_t, sc * sizeof(double));
    if (c == cudaSuccess) c = cudaMalloc(&e->log_off, sc * sizeof(int64_t));
    if (c == cudaSuccess) c = cudaMalloc(&e->log_idx, ic * sizeof(int32_t));
    if (c == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        nb_ensemble_set_log(e, 0, 0);
        return efail(e, NB_ENOMEM, "no device memory for the step log");
    }
    ECU(e, c);
    ECU(e, cudaMemsetAsync(e->log_cnt, 0, 2 * sizeof(unsigned long long), e->stream));
    e->log_cap = step_cap;
    e->idx_cap = idx_cap;
    return NB_OK;
}

nb_status nb_ensemble_get_log(nb_ensemble *e, int32_t *sys, double *t, int32_t *n_act, int64_t *idx_off,
                              int32_t *idx, int64_t *n_steps, int64_t *n_idx)
{
    if (!e)
        return NB_EINVAL;
    if (e->dead)
        return NB_ECUDA;
    unsigned long long cnt[2] = {0, 0};
    if (e->log_cnt)
        ECU(e, cudaMemcpyAsync(cnt, e->log_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, e->stream));
    ECU(e, cudaStreamSynchronize(e->stream));
    const size_t ks = static_cast<size_t>(std::min<unsigned long long>(cnt[0], e->log_cap));
    const size_t ki = static_cast<size_t>(std::min<unsigned long long>(cnt[1], e->idx_cap));
    if (ks > 0) {
        if (sys) ECU(e, cudaMemcpyAsync(sys, e->log_sys, ks * sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
        if (t) ECU(e, cudaMemcpyAsync(t, e->log_t, ks * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
        if (n_act) ECU(e, cudaMemcpyAsync(n_act, e->log_n, ks * sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
        if (idx_off)
            ECU(e, cudaMemcpyAsync(idx_off, e->log_off, ks * sizeof(int64_t), cudaMemcpyDeviceToHost, e->stream));
    }
    if (ki > 0 && idx)
        ECU(e, cudaMemcpyAsync(idx, e->log_idx, ki * sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
    ECU(e, cudaStreamSynchronize(e->stream));
    if (n_steps)
        *n_steps = static_cast<int64_t>(cnt[0]);
    if (n_idx)
        *n_idx = static_cast<int64_t>(cnt[1]);
    return NB_OK;
}

const char *nb_ensemble_last_error(const nb_ensemble *e)
{
    return e ? e->err.c_str() : nb_last_error(nullptr);
}

void nb_ensemble_free(nb_ensemble *e)
{
    if (!e)
        return;
    cudaStreamSynchronize(e->stream);
    ens_free_all(e);
    delete e;
}

}  // extern "C"
