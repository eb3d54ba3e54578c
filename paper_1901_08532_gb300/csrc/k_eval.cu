// Evaluation step of the 6th-order Hermite scheme (paper, section 3 item 4):
// acceleration, jerk and snap of every listed i-particle from all
// j-particles, Plummer-softened, G = 1.
//
// Layout of one launch (GB300, sm_103a):
//   * grid.x tiles the active list: a block holds (threads / lanes) * KI
//     i-particles in registers (section 3 item 4 step ii);
//   * grid.y splits the j-range into `split` contiguous chunks (split-j);
//   * j-particles stream through shared memory in tiles of `jtile` records,
//     loaded by 1-D TMA bulk copies into a two-stage mbarrier pipeline
//     (section 3 item 4 steps i and iii);
//   * `lanes` consecutive threads share one i and take every lanes-th j of a
//     tile; their sums are combined with warp shuffles in a fixed order;
//   * with split > 1 each block writes FP64 partials, and the last block of
//     an i-tile to finish adds the `split` partials in index order, so the
//     result does not depend on block scheduling.
// The self term needs no test: eps > 0 makes r = v = a = 0 contribute 0.
#include <algorithm>
#include <mutex>
#include <vector>

#include "nb_device.cuh"
#include "nb_ff.cuh"
#include "nb_internal.cuh"

namespace {

using namespace nbk;

// Largest block for KI i-particles per thread (register budget: 255 per
// thread at 256 threads, 128 at 512).
__host__ __device__ constexpr int max_threads_for(int ki) { return ki == 1 ? 512 : (ki == 2 ? 256 : 128); }

struct EvalArgs {
    const void *jb;      // [NC][n] 16-byte records
    int n;               // record stride (j count of the buffer)
    int j0, j1;          // j-range evaluated, [j0, j1) (the whole buffer: 0, n)
    const int32_t *act;  // [n_act]
    int n_act;
    double *out;         // [9][ostride]
    int ostride;
    double *part;        // [split][9][n_act] when split > 1
    unsigned *cnt;       // [gridDim.x] arrival counters, zero between launches
    int jtile, lanes, split, jchunk;
    double eps2;
    nb_ctl *ctl;
    uint32_t tx_extra;   // bytes added to the first tile's expected count (fault injection)
};

template <int NC>
__device__ __forceinline__ void issue_tile(unsigned char *smem, uint64_t *bar, const EvalArgs &a,
                                           int stage, int j0, int len, uint32_t extra = 0)
{
    const uint4 *src = static_cast<const uint4 *>(a.jb);
    uint4 *dst = reinterpret_cast<uint4 *>(smem) + static_cast<size_t>(stage) * NC * a.jtile;
    nbk::mbar_expect_tx(&bar[stage], static_cast<uint32_t>(NC * len * 16) + extra);
#pragma unroll
    for (int c = 0; c < NC; ++c)
        nbk::bulk_g2s(dst + c * a.jtile, src + static_cast<size_t>(c) * a.n + j0,
                      static_cast<uint32_t>(len * 16), &bar[stage]);
}

// After a timed-out wait: let the copies still in flight land (bounded)
// before the block's shared memory is released, then flag the error.
__device__ void drain_after_timeout(uint64_t *bar, int consumed, int issued, nb_ctl *ctl)
{
    for (int t = consumed; t < issued; ++t)
        nbk::mbar_wait_bounded(&bar[t & 1], (t >> 1) & 1, nbk::kWaitLimitNs);
    atomicOr(&ctl->err, NB_ERR_TIMEOUT);
}

// Split-j epilogue shared by both precisions: write this block's sums (or
// partials) and, when split > 1, fold the partials in the last block.
template <int KI>
__device__ __forceinline__ void store_or_fold(const EvalArgs &a, double (&acc)[9][KI],
                                              const int (&kidx)[KI], int lj, int slots, int ibase)
{
    __shared__ int s_last;
    if (lj == 0) {
#pragma unroll
        for (int k = 0; k < KI; ++k) {
            if (kidx[k] < 0)
                continue;
            if (a.split == 1) {
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    a.out[static_cast<size_t>(q) * a.ostride + kidx[k]] = acc[q][k];
            } else {
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    a.part[(static_cast<size_t>(blockIdx.y) * 9 + q) * a.n_act + kidx[k]] = acc[q][k];
            }
        }
    }
    if (a.split == 1)
        return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = (atomicAdd(&a.cnt[blockIdx.x], 1u) == static_cast<unsigned>(a.split - 1));
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    const int itile = slots * KI;
    for (int e = threadIdx.x; e < itile * 9; e += blockDim.x) {
        const int q = e / itile;
        const int p = ibase + (e - q * itile);
        if (p >= a.n_act)
            continue;
        double s = 0.0;
        for (int sp = 0; sp < a.split; ++sp)
            s += __ldcg(&a.part[(static_cast<size_t>(sp) * 9 + q) * a.n_act + p]);
        a.out[static_cast<size_t>(q) * a.ostride + p] = s;
    }
    if (threadIdx.x == 0)
        a.cnt[blockIdx.x] = 0u;
}

// ------------------------------------------------------------------ FP64

// With four i-particles per thread the running totals (9 x KI doubles,
// touched once per tile) live in shared memory after the tiles, rows
// [9 * KI][threads]: in registers they would not fit beside the tile partial
// sums and the i-values (255 registers per thread at most).
__host__ __device__ constexpr bool fp64_shared_totals(int ki) { return ki >= 4; }

template <int KI>
__global__ void __launch_bounds__(max_threads_for(KI)) eval_fp64_kernel(EvalArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    constexpr int NC = 5;
    const int tid = threadIdx.x, lanes = a.lanes, jt = a.jtile;
    const int slot = tid / lanes, lj = tid - slot * lanes;
    const int slots = blockDim.x / lanes;
    const int ibase = blockIdx.x * slots * KI;
    const double2 *jb = static_cast<const double2 *>(a.jb);

    constexpr bool SH = fp64_shared_totals(KI);
    int kidx[KI];
    double xi[KI], yi[KI], zi[KI], vxi[KI], vyi[KI], vzi[KI], axi[KI], ayi[KI], azi[KI];
    double acc[9][SH ? 1 : KI], part[9][KI];
    double *acc_s = reinterpret_cast<double *>(smem) + static_cast<size_t>(2) * NC * 2 * jt;
    const int nthr = blockDim.x;
#pragma unroll
    for (int k = 0; k < KI; ++k) {
        const int p = ibase + slot + k * slots;
        kidx[k] = p < a.n_act ? p : -1;
        const int i = a.act[p < a.n_act ? p : a.n_act - 1];
        const double2 r0 = jb[i], r1 = jb[(size_t)a.n + i], r2 = jb[2 * (size_t)a.n + i];
        const double2 r3 = jb[3 * (size_t)a.n + i], r4 = jb[4 * (size_t)a.n + i];
        xi[k] = r0.x; yi[k] = r0.y; zi[k] = r1.x;
        vxi[k] = r2.x; vyi[k] = r2.y; vzi[k] = r3.x;
        axi[k] = r3.y; ayi[k] = r4.x; azi[k] = r4.y;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            if (SH)
                acc_s[(q * KI + k) * nthr + tid] = 0.0;
            else
                acc[q][SH ? 0 : k] = 0.0;
        }
    }

    const int jbeg = a.j0 + blockIdx.y * a.jchunk;
    const int jend = min(a.j1, jbeg + a.jchunk);
    const int ntiles = jend > jbeg ? (jend - jbeg + jt - 1) / jt : 0;
    int issued = 0;
    if (tid == 0) {
        nbk::mbar_init(&bar[0], 1);
        nbk::mbar_init(&bar[1], 1);
        nbk::fence_mbar_init();
        for (; issued < min(2, ntiles); ++issued)
            issue_tile<NC>(smem, bar, a, issued, jbeg + issued * jt, min(jt, jend - (jbeg + issued * jt)),
                           issued == 0 ? a.tx_extra : 0u);
    }
    __syncthreads();

    for (int tl = 0; tl < ntiles; ++tl) {
        const int st = tl & 1;
        const bool ok = nbk::mbar_wait_bounded(&bar[st], (tl >> 1) & 1, nbk::kWaitLimitNs);
        if (!__syncthreads_and(ok)) {
            if (tid == 0)
                drain_after_timeout(bar, tl, issued, a.ctl);
            return;
        }
        const int len = min(jt, jend - (jbeg + tl * jt));
        const double2 *s = reinterpret_cast<const double2 *>(smem) + static_cast<size_t>(st) * NC * jt;
#pragma unroll
        for (int k = 0; k < KI; ++k)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                part[q][k] = 0.0;
        for (int jj = lj; jj < len; jj += lanes) {
            const double2 p0 = s[jj], p1 = s[jt + jj], p2 = s[2 * jt + jj], p3 = s[3 * jt + jj],
                          p4 = s[4 * jt + jj];
#pragma unroll
            for (int k = 0; k < KI; ++k) {
                double pk[9];
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    pk[q] = part[q][k];
                pair_fp64(p0, p1, p2, p3, p4, xi[k], yi[k], zi[k], vxi[k], vyi[k], vzi[k], axi[k],
                          ayi[k], azi[k], a.eps2, pk);
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    part[q][k] = pk[q];
            }
        }
        // two-level summation: tile partial, then running total
#pragma unroll
        for (int k = 0; k < KI; ++k)
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                if (SH)
                    acc_s[(q * KI + k) * nthr + tid] += part[q][k];
                else
                    acc[q][SH ? 0 : k] += part[q][k];
            }
        __syncthreads();
        if (tid == 0 && tl + 2 < ntiles) {
            issue_tile<NC>(smem, bar, a, st, jbeg + (tl + 2) * jt, min(jt, jend - (jbeg + (tl + 2) * jt)));
            ++issued;
        }
    }

    // the totals (from shared memory for SH; the tile partials are dead here)
#pragma unroll
    for (int k = 0; k < KI; ++k)
#pragma unroll
        for (int q = 0; q < 9; ++q)
            part[q][k] = SH ? acc_s[(q * KI + k) * nthr + tid] : acc[q][SH ? 0 : k];
    for (int off = lanes >> 1; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < KI; ++k)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                part[q][k] += __shfl_xor_sync(0xffffffffu, part[q][k], off);
    store_or_fold<KI>(a, part, kidx, lj, slots, ibase);
}

// ----------------------------------------------------------------- mixed
//
// FP32 pair arithmetic in packed form: every f32x2 instruction works on two
// j-particles at once (fma.rn.f32x2 and friends, sm_100+), which halves the
// issue slots the pair formula needs, so the FP32 pipe rather than
// instruction issue sets the pace.  The j-tile sits in shared memory as 13
// FP32 rows, so two (or four) consecutive j of one component load as one
// 64- (128-) bit word; the i-particle's values are held negated and
// duplicated into both halves of a pair.
//
// Position differences are formed from hi/lo FP32 pairs,
// (xj_hi - xi_hi) + (xj_lo - xi_lo), which keeps them accurate to FP32
// rounding of the difference itself even for close pairs far from the
// origin; velocity and acceleration differences use FP32 copies.  q and q^2
// are separate special-function-unit estimates of R^(-1/2) and 1/R (which
// moves their cost off the FMA pipe).  Each thread sums a tile in
// FP32 (two halves), then folds the tile sum into a TwoSum-compensated
// (hi, lo) accumulator.

// NR bulk copies per tile, one per FP32 row; len and j0 are multiples of 4.
template <int NR = NCF>
__device__ __forceinline__ void issue_tile_rows(unsigned char *smem, uint64_t *bar, const EvalArgs &a,
                                                int stage, int j0, int len, uint32_t extra = 0)
{
    const float *src = static_cast<const float *>(a.jb);
    float *dst = reinterpret_cast<float *>(smem) + static_cast<size_t>(stage) * NR * a.jtile;
    nbk::mbar_expect_tx(&bar[stage], static_cast<uint32_t>(NR * len * 4) + extra);
#pragma unroll
    for (int c = 0; c < NR; ++c)
        nbk::bulk_g2s(dst + c * a.jtile, src + static_cast<size_t>(c) * a.n + j0,
                      static_cast<uint32_t>(len * 4), &bar[stage]);
}

// Block-size limit and minimum resident blocks of the mixed kernel: KI = 2
// runs 3 blocks of 128 threads per SM (12 warps, <= 170 registers), KI = 3
// 2 blocks of 128 (<= 255 registers), KI = 1 2 blocks of 256.  The
// compensated (hi, lo) accumulators, touched once per tile, live in shared
// memory after the tiles: rows [18 * KI][threads].
__host__ __device__ constexpr int mixed_max_threads(int ki) { return ki == 1 ? 256 : 128; }
__host__ __device__ constexpr int mixed_min_blocks(int ki) { return ki == 2 ? 3 : 2; }

// JU j-particles per inner iteration (2: one pair, 4: two pairs from one
// 128-bit load per row).  JT > 0 fixes the j-tile length at compile time
// (the launch's jtile must equal it), so that every shared-memory row of the
// inner loop is addressed by a constant offset from one base; JT = 0 takes
// it from the launch.  More i-particles per thread (KI) give each warp more
// independent pair terms, which the packed FMAs need: each reads three
// 64-bit register operands, and the register file sustains that for only
// about two thirds of the pipe's rate (k_peaks.cu, kind 8).
template <int KI, int JU, int JT>
__global__ void __launch_bounds__(mixed_max_threads(KI), mixed_min_blocks(KI))
    eval_mixed_kernel(EvalArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = threadIdx.x, lanes = a.lanes;
    const int jt = JT > 0 ? JT : a.jtile;
    const int slot = tid / lanes, lj = tid - slot * lanes;
    const int slots = blockDim.x / lanes;
    const int ibase = blockIdx.x * slots * KI;
    const float *jf = static_cast<const float *>(a.jb);
    const size_t np = static_cast<size_t>(a.n);
    const float2 eps2 = f2(static_cast<float>(a.eps2));
    constexpr int kRow[12] = {0, 1, 2, 4, 5, 6, 7, 8, 9, 10, 11, 12};

    int kidx[KI];
    float2 ni[KI][12];
    float2 part[9][KI];
    float *acc_s = reinterpret_cast<float *>(smem) + static_cast<size_t>(2) * NCF * jt;
    const int nthr = blockDim.x;
#pragma unroll
    for (int k = 0; k < KI; ++k) {
        const int p = ibase + slot + k * slots;
        kidx[k] = p < a.n_act ? p : -1;
        const int i = a.act[p < a.n_act ? p : a.n_act - 1];
#pragma unroll
        for (int q = 0; q < 12; ++q)
            ni[k][q] = f2(-jf[kRow[q] * np + i]);
#pragma unroll
        for (int q = 0; q < 18; ++q)
            acc_s[(q * KI + k) * nthr + tid] = 0.0f;
    }

    const int jbeg = a.j0 + blockIdx.y * a.jchunk;
    const int jend = min(a.j1, jbeg + a.jchunk);
    const int ntiles = jend > jbeg ? (jend - jbeg + jt - 1) / jt : 0;
    int issued = 0;
    if (tid == 0) {
        nbk::mbar_init(&bar[0], 1);
        nbk::mbar_init(&bar[1], 1);
        nbk::fence_mbar_init();
        for (; issued < min(2, ntiles); ++issued)
            issue_tile_rows(smem, bar, a, issued, jbeg + issued * jt, min(jt, jend - (jbeg + issued * jt)),
                            issued == 0 ? a.tx_extra : 0u);
    }
    __syncthreads();

    for (int tl = 0; tl < ntiles; ++tl) {
        const int st = tl & 1;
        const bool ok = nbk::mbar_wait_bounded(&bar[st], (tl >> 1) & 1, nbk::kWaitLimitNs);
        if (!__syncthreads_and(ok)) {
            if (tid == 0)
                drain_after_timeout(bar, tl, issued, a.ctl);
            return;
        }
        const int len = min(jt, jend - (jbeg + tl * jt));
        const float *s = reinterpret_cast<const float *>(smem) + static_cast<size_t>(st) * NCF * jt;
        // FP32 running sums over at most kMixedFoldJ j per lane, then folded
        // into the compensated sums
        for (int f0 = 0; f0 < len; f0 += nbk::kMixedFoldJ * lanes) {
            const int f1 = min(len, f0 + nbk::kMixedFoldJ * lanes);
#pragma unroll
            for (int k = 0; k < KI; ++k)
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    part[q][k] = f2(0.0f);
            for (int jj = f0 + JU * lj; jj < f1; jj += JU * lanes) {
                if (JU == 4) {
                    float2 c0[NCF], c1[NCF];
#pragma unroll
                    for (int r = 0; r < NCF; ++r) {
                        const float4 w = *reinterpret_cast<const float4 *>(s + r * jt + jj);
                        c0[r] = make_float2(w.x, w.y);
                        c1[r] = make_float2(w.z, w.w);
                    }
#pragma unroll
                    for (int k = 0; k < KI; ++k) {
                        float2 pk[9];
#pragma unroll
                        for (int q = 0; q < 9; ++q)
                            pk[q] = part[q][k];
                        pair_mixed2(c0, ni[k], eps2, pk);
                        pair_mixed2(c1, ni[k], eps2, pk);
#pragma unroll
                        for (int q = 0; q < 9; ++q)
                            part[q][k] = pk[q];
                    }
                } else {
                    float2 c0[NCF];
#pragma unroll
                    for (int r = 0; r < NCF; ++r)
                        c0[r] = *reinterpret_cast<const float2 *>(s + r * jt + jj);
#pragma unroll
                    for (int k = 0; k < KI; ++k) {
                        float2 pk[9];
#pragma unroll
                        for (int q = 0; q < 9; ++q)
                            pk[q] = part[q][k];
                        pair_mixed2(c0, ni[k], eps2, pk);
#pragma unroll
                        for (int q = 0; q < 9; ++q)
                            part[q][k] = pk[q];
                    }
                }
            }
            // fold the FP32 sums (both halves) into the compensated accumulators
#pragma unroll
            for (int k = 0; k < KI; ++k)
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    float h = acc_s[(q * KI + k) * nthr + tid];
                    float l = acc_s[((9 + q) * KI + k) * nthr + tid];
                    nbk::two_sum_acc(h, l, __fadd_rn(part[q][k].x, part[q][k].y));
                    acc_s[(q * KI + k) * nthr + tid] = h;
                    acc_s[((9 + q) * KI + k) * nthr + tid] = l;
                }
        }
        __syncthreads();
        if (tid == 0 && tl + 2 < ntiles) {
            issue_tile_rows(smem, bar, a, st, jbeg + (tl + 2) * jt, min(jt, jend - (jbeg + (tl + 2) * jt)));
            ++issued;
        }
    }

    double acc[9][KI];
#pragma unroll
    for (int k = 0; k < KI; ++k)
#pragma unroll
        for (int q = 0; q < 9; ++q)
            acc[q][k] = static_cast<double>(acc_s[(q * KI + k) * nthr + tid]) +
                        static_cast<double>(acc_s[((9 + q) * KI + k) * nthr + tid]);
    for (int off = lanes >> 1; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < KI; ++k)
#pragma unroll
            for (int q = 0; q < 9; ++q)
                acc[q][k] += __shfl_xor_sync(0xffffffffu, acc[q][k], off);
    store_or_fold<KI>(a, acc, kidx, lj, slots, ibase);
}

// -------------------------------------------------------------------- EX
//
// Double-word ("float-float") pair arithmetic from FP32 operations only
// (section 3 item 6): the j-tile holds 20 FP32 rows (every position,
// velocity, acceleration and mass as a high and a low part), each pair term
// is formed with the error-free transformations of nb_ff.cuh, a thread sums
// the terms of one tile in unnormalised double words (Sum2), and each
// tile's sum is added to an FP64 total.  T = float2 evaluates two j per
// instruction in the lanes of the packed f32x2 operations, T = float one.
// One i-particle per thread slot.

constexpr int kExThreads = 128;
// j per lane in one double-word running sum of the EX kernel before it is
// added into the tile's sums: the Sum2 low part gathers every rounding error
// in FP32, so its own rounding grows with the number of terms; over all
// 2^20 particles, whole 512-j tiles left 4 snaps above 1e-12 of their
// condition number (at most 1.24e-12); 128 j leaves none (at most 8.1e-13),
// for about 1 % more time.
constexpr int kExFoldJ = 128;

template <class T>
__global__ void __launch_bounds__(kExThreads, 2) eval_ex_kernel(EvalArgs a)
{
    using ff::FF;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    constexpr int JU = sizeof(T) / sizeof(float);
    const int tid = threadIdx.x, lanes = a.lanes, jt = a.jtile;
    const int slot = tid / lanes, lj = tid - slot * lanes;
    const int slots = blockDim.x / lanes;
    const int ibase = blockIdx.x * slots;
    const float *jf = static_cast<const float *>(a.jb);
    const size_t np = static_cast<size_t>(a.n);
    const T z = ff::splat(T{}, 0.0f);
    const float e2h = __double2float_rn(a.eps2);
    const FF<T> eps2 = {ff::splat(z, e2h), ff::splat(z, __double2float_rn(a.eps2 - static_cast<double>(e2h)))};

    int kidx[1];
    const int p = ibase + slot;
    kidx[0] = p < a.n_act ? p : -1;
    const int i = a.act[p < a.n_act ? p : a.n_act - 1];
    ExI<T> ni;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ni.x[k] = {ff::splat(z, -jf[k * np + i]), ff::splat(z, -jf[(3 + k) * np + i])};
        ni.v[k] = {ff::splat(z, -jf[(6 + k) * np + i]), ff::splat(z, -jf[(9 + k) * np + i])};
        ni.a[k] = {ff::splat(z, -jf[(12 + k) * np + i]), ff::splat(z, -jf[(15 + k) * np + i])};
    }
    double acc[9][1];
#pragma unroll
    for (int q = 0; q < 9; ++q)
        acc[q][0] = 0.0;

    const int jbeg = a.j0 + blockIdx.y * a.jchunk;
    const int jend = min(a.j1, jbeg + a.jchunk);
    const int ntiles = jend > jbeg ? (jend - jbeg + jt - 1) / jt : 0;
    int issued = 0;
    if (tid == 0) {
        nbk::mbar_init(&bar[0], 1);
        nbk::mbar_init(&bar[1], 1);
        nbk::fence_mbar_init();
        for (; issued < min(2, ntiles); ++issued)
            issue_tile_rows<NCX>(smem, bar, a, issued, jbeg + issued * jt,
                                 min(jt, jend - (jbeg + issued * jt)), issued == 0 ? a.tx_extra : 0u);
    }
    __syncthreads();

    for (int tl = 0; tl < ntiles; ++tl) {
        const int st = tl & 1;
        const bool ok = nbk::mbar_wait_bounded(&bar[st], (tl >> 1) & 1, nbk::kWaitLimitNs);
        if (!__syncthreads_and(ok)) {
            if (tid == 0)
                drain_after_timeout(bar, tl, issued, a.ctl);
            return;
        }
        const int len = min(jt, jend - (jbeg + tl * jt));
        const float *s = reinterpret_cast<const float *>(smem) + static_cast<size_t>(st) * NCX * jt;
        // double-word running sums over at most kExFoldJ j per lane, added
        // (Sum2) into the tile's double-word sums, which go to FP64 per tile
        FF<T> tile[9];
#pragma unroll
        for (int q = 0; q < 9; ++q)
            tile[q] = {z, z};
        for (int f0 = 0; f0 < len; f0 += kExFoldJ * lanes) {
            const int f1 = min(len, f0 + kExFoldJ * lanes);
            FF<T> part[9];
#pragma unroll
            for (int q = 0; q < 9; ++q)
                part[q] = {z, z};
            for (int jj = f0 + JU * lj; jj < f1; jj += JU * lanes) {
                T c[NCX];
#pragma unroll
                for (int r = 0; r < NCX; ++r)
                    c[r] = *reinterpret_cast<const T *>(s + r * jt + jj);
                pair_ex(c, ni, eps2, part);
            }
#pragma unroll
            for (int q = 0; q < 9; ++q)
                ff::accumulate(tile[q], part[q]);
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float *h = reinterpret_cast<const float *>(&tile[q].h);
            const float *l = reinterpret_cast<const float *>(&tile[q].l);
#pragma unroll
            for (int u = 0; u < JU; ++u)
                acc[q][0] += static_cast<double>(h[u]) + static_cast<double>(l[u]);
        }
        __syncthreads();
        if (tid == 0 && tl + 2 < ntiles) {
            issue_tile_rows<NCX>(smem, bar, a, st, jbeg + (tl + 2) * jt, min(jt, jend - (jbeg + (tl + 2) * jt)));
            ++issued;
        }
    }

    for (int off = lanes >> 1; off > 0; off >>= 1)
#pragma unroll
        for (int q = 0; q < 9; ++q)
            acc[q][0] += __shfl_xor_sync(0xffffffffu, acc[q][0], off);
    store_or_fold<1>(a, acc, kidx, lj, slots, ibase);
}

constexpr int kRecBytes64 = 5 * 16;
constexpr int kRecBytes32 = NCF * 4;
constexpr int kRecBytesEx = NCX * 4;

using EvalKernel = void (*)(EvalArgs);

// The mixed kernel for KI i-particles per thread, JU j per inner iteration
// and j-tile jt (compile-time where an instantiation exists); nullptr for a
// combination that is not built (KI = 3 runs with JU = 4 only).
EvalKernel mixed_kernel(int ki, int ju, int jt)
{
    if (ki == 1)
        return ju == 2 ? eval_mixed_kernel<1, 2, 0> : eval_mixed_kernel<1, 4, 0>;
    if (ki == 2 && ju == 2)
        return eval_mixed_kernel<2, 2, 0>;
    if (ki == 2)
        return jt == 512 ? eval_mixed_kernel<2, 4, 512> : jt == 256 ? eval_mixed_kernel<2, 4, 256>
                                                                    : eval_mixed_kernel<2, 4, 0>;
    if (ki == 3 && ju == 4)
        return jt == 512 ? eval_mixed_kernel<3, 4, 512> : jt == 256 ? eval_mixed_kernel<3, 4, 256>
                                                                    : eval_mixed_kernel<3, 4, 0>;
    return nullptr;
}

template <typename K>
cudaError_t set_smem_attr(K kernel)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

cudaError_t nb_eval_smem_setup()
{
    cudaError_t e;
    if ((e = set_smem_attr(eval_fp64_kernel<1>)) != cudaSuccess) return e;
    if ((e = set_smem_attr(eval_fp64_kernel<2>)) != cudaSuccess) return e;
    if ((e = set_smem_attr(eval_fp64_kernel<4>)) != cudaSuccess) return e;
    for (int ki = 1; ki <= 3; ++ki)
        for (int ju = 2; ju <= 4; ju += 2)
            for (int jt = 0; jt <= 512; jt += 256)
                if (const EvalKernel k = mixed_kernel(ki, ju, jt))
                    if ((e = set_smem_attr(k)) != cudaSuccess) return e;
    if ((e = set_smem_attr(eval_ex_kernel<float>)) != cudaSuccess) return e;
    if ((e = set_smem_attr(eval_ex_kernel<float2>)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Blocks of the chosen evaluation kernel that fit on one SM.
int resident_blocks(const nb_ctx *c, const nb_tiles &t)
{
    const bool mixed = nb_fp32_eval(c->cfg.precision);
    const bool ex = c->cfg.precision == NB_EX;
    const size_t smem = static_cast<size_t>(2) * (ex ? kRecBytesEx : mixed ? kRecBytes32 : kRecBytes64) * t.jtile +
                        (mixed ? static_cast<size_t>(18) * t.ki * t.threads * sizeof(float) : 0) +
                        (!mixed && !ex && fp64_shared_totals(t.ki)
                             ? static_cast<size_t>(9) * t.ki * t.threads * sizeof(double) : 0);
    int nb = 0;
    cudaError_t e;
    if (ex) {
        if (t.junroll == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_ex_kernel<float>, t.threads, smem);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_ex_kernel<float2>, t.threads, smem);
    } else if (mixed) {
        const EvalKernel k = mixed_kernel(t.ki, t.junroll, t.jtile);
        e = k ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, t.threads, smem) : cudaErrorInvalidValue;
    } else {
        if (t.ki == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_fp64_kernel<1>, t.threads, smem);
        else if (t.ki == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_fp64_kernel<2>, t.threads, smem);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eval_fp64_kernel<4>, t.threads, smem);
    }
    if (e != cudaSuccess || nb < 1) {
        (void)cudaGetLastError();
        return 1;
    }
    return nb;
}

// Automatic launch shape.  Large active sets: one i per thread slot, no
// split.  Small ones: lanes share an i so that a block's i-slots are not
// mostly empty, and the j-range is split across blocks until the grid
// covers every SM several times.
nb_tiles nb_auto_tiles(const nb_ctx *c, int64_t n_act, const nb_tiles &req, int64_t j_count)
{
    nb_tiles t = req;
    const bool ex = c->cfg.precision == NB_EX;
    const bool mixed = nb_fp32_eval(c->cfg.precision);
    // defaults from the launch-shape sweeps on GB300 (autotune.py): mixed
    // KI = 2 with four j per iteration for small active sets, three
    // i-particles per thread and 512-j tiles from 8192 active on
    const bool big = n_act >= 8192;
    if (t.ki <= 0)
        t.ki = mixed ? (big ? 3 : 2) : 1;
    if (t.threads <= 0)
        t.threads = ex ? kExThreads : mixed ? mixed_max_threads(t.ki) : 128;
    if (t.junroll <= 0)
        t.junroll = ex ? 2 : 4;
    if (t.lanes <= 0) {
        // two lanes per i-particle below 4096 active in the mixed kernel
        // (fewer, deeper j-chunks to fold); more while the block would hold
        // more i-slots than there are active particles
        int l = mixed && t.ki == 2 && n_act < 4096 ? 2 : 1;
        while (l < 32 && static_cast<int64_t>(t.threads / (2 * l)) * t.ki >= n_act)
            l *= 2;
        t.lanes = l;
    }
    if (t.jtile <= 0)
        t.jtile = mixed ? (n_act >= 512 ? 512 : 256) : (ex ? 512 : 256);
    if ((mixed || ex) && t.jtile % 4)
        t.jtile = (t.jtile / 4 + 1) * 4;   // whole 16-byte rows per bulk copy
    if (t.split <= 0) {
        // Split the j-range so that the grid fills whole waves of resident
        // blocks: all blocks of a launch do equal work, so a partial last
        // wave idles the rest of the GPU for a whole block's duration.
        const int64_t jn = j_count > 0 ? j_count : ((mixed || ex) ? c->npad : c->n);
        const int64_t itile = static_cast<int64_t>(t.threads / t.lanes) * t.ki;
        const int64_t nblk = (n_act + itile - 1) / itile;
        const int64_t cap = static_cast<int64_t>(c->sm_count) * resident_blocks(c, t);
        const int64_t max_s = std::max<int64_t>(1, std::min<int64_t>(1024, jn / (2 * t.jtile)));
        // Each block does 1/s of an i-tile's work, so the launch takes about
        // ceil(nblk s / cap) / s block-times; take the smallest s within 2 %
        // of the best (fewer partial sums to fold).
        int64_t best = 1;
        if (nblk < 4 * cap) {
            double tmin = 1e300;
            std::vector<double> ts(static_cast<size_t>(max_s) + 1, 0.0);
            for (int64_t s = 1; s <= max_s; ++s) {
                ts[s] = static_cast<double>((nblk * s + cap - 1) / cap) / static_cast<double>(s);
                tmin = std::min(tmin, ts[s]);
            }
            for (int64_t s = 1; s <= max_s; ++s)
                if (ts[s] <= 1.02 * tmin) {
                    best = s;
                    break;
                }
        }
        t.split = static_cast<int32_t>(best);
    }
    return t;
}

cudaError_t nb_launch_eval(nb_ctx *c, const EvalLaunch &L)
{
    const nb_tiles &t = L.tiles;
    if (L.n_act <= 0)
        return cudaSuccess;
    const bool mixed = nb_fp32_eval(c->cfg.precision);
    const bool ex = c->cfg.precision == NB_EX;
    if (!(t.ki == 1 || (t.ki == 2 && !ex) || (t.ki == 3 && mixed && t.junroll == 4) ||
          (t.ki == 4 && !mixed && !ex)) || t.threads < 32 ||
        t.threads > (ex ? kExThreads : mixed ? mixed_max_threads(t.ki) : max_threads_for(t.ki)) ||
        t.threads % 32 || !is_pow2(t.lanes) || t.lanes > 32 || t.jtile < 1 || t.split < 1)
        return cudaErrorInvalidValue;
    if (mixed && (!(t.junroll == 2 || t.junroll == 4) || t.jtile % 4))
        return cudaErrorInvalidValue;
    if (ex && (!(t.junroll == 1 || t.junroll == 2) || t.jtile % 4))
        return cudaErrorInvalidValue;
    const int rec = ex ? kRecBytesEx : mixed ? kRecBytes32 : kRecBytes64;
    const size_t smem = static_cast<size_t>(2) * rec * t.jtile +
                        (mixed ? static_cast<size_t>(18) * t.ki * t.threads * sizeof(float) : 0) +
                        (!mixed && !ex && fp64_shared_totals(t.ki)
                             ? static_cast<size_t>(9) * t.ki * t.threads * sizeof(double) : 0);
    if (smem > 200 * 1024)
        return cudaErrorInvalidValue;
    const int itile = (t.threads / t.lanes) * t.ki;
    const int gx = (L.n_act + itile - 1) / itile;
    // j-range (the whole buffer unless L.j1 >= 0) and chunk per split, a
    // whole number of tiles
    const int64_t nbuf = (mixed || ex) ? c->npad : c->n;
    const int64_t j0 = L.j1 >= 0 ? L.j0 : 0, j1 = L.j1 >= 0 ? L.j1 : nbuf;
    if (j0 < 0 || j1 > nbuf || j0 > j1 || ((mixed || ex) && (j0 % 4 || j1 % 4)))
        return cudaErrorInvalidValue;
    const int64_t jn = j1 - j0;
    int64_t chunk = std::max<int64_t>(1, (jn + t.split - 1) / t.split);
    chunk = (chunk + t.jtile - 1) / t.jtile * t.jtile;
    const int split = std::max(1, static_cast<int>((jn + chunk - 1) / chunk));

    EvalArgs a;
    a.jb = (mixed || ex) ? static_cast<const void *>(c->jf32) : static_cast<const void *>(c->jb64);
    a.n = static_cast<int>(nbuf);
    a.j0 = static_cast<int>(j0);
    a.j1 = static_cast<int>(j1);
    a.act = L.act;
    a.n_act = L.n_act;
    a.out = L.out;
    a.ostride = L.ostride;
    a.jtile = t.jtile;
    a.lanes = t.lanes;
    a.split = split;
    a.jchunk = static_cast<int>(chunk);
    a.eps2 = c->eps * c->eps;
    a.ctl = c->ctl;
    a.part = nullptr;
    a.cnt = nullptr;
    a.tx_extra = c->inject == 1 ? 16u : 0u;
    c->inject = 0;
    if (split > 1) {
        const size_t need = static_cast<size_t>(split) * 9 * L.n_act;
        if (need > c->part_cap) {
            cudaFree(c->part);
            c->part = nullptr;
            c->part_cap = 0;
            cudaError_t e = cudaMalloc(&c->part, need * sizeof(double));
            if (e != cudaSuccess)
                return e;
            c->part_cap = need;
        }
        if (static_cast<size_t>(gx) > c->tile_cnt_cap) {
            cudaFree(c->tile_cnt);
            c->tile_cnt = nullptr;
            c->tile_cnt_cap = 0;
            cudaError_t e = cudaMalloc(&c->tile_cnt, static_cast<size_t>(gx) * sizeof(unsigned));
            if (e != cudaSuccess)
                return e;
            e = cudaMemsetAsync(c->tile_cnt, 0, static_cast<size_t>(gx) * sizeof(unsigned), c->stream);
            if (e != cudaSuccess)
                return e;
            c->tile_cnt_cap = gx;
        }
        a.part = c->part;
        a.cnt = c->tile_cnt;
    }
    const dim3 grid(gx, split), block(t.threads);
    if (ex) {
        if (t.junroll == 1) eval_ex_kernel<float><<<grid, block, smem, c->stream>>>(a);
        else eval_ex_kernel<float2><<<grid, block, smem, c->stream>>>(a);
    } else if (mixed) {
        mixed_kernel(t.ki, t.junroll, t.jtile)<<<grid, block, smem, c->stream>>>(a);
    } else {
        if (t.ki == 1) eval_fp64_kernel<1><<<grid, block, smem, c->stream>>>(a);
        else if (t.ki == 2) eval_fp64_kernel<2><<<grid, block, smem, c->stream>>>(a);
        else eval_fp64_kernel<4><<<grid, block, smem, c->stream>>>(a);
    }
    c->launches += 1;
    c->interactions += static_cast<double>(L.n_act) *
                       static_cast<double>(L.j1 >= 0 ? std::min<int64_t>(j1, c->n) - j0 : c->n);
    return cudaGetLastError();
}

// Stateless all-active FP64 evaluation on caller-packed records (used by the
// differentiable trajectory path): no split, lanes chosen so the grid holds
// at least two blocks per SM.
cudaError_t nb_launch_eval_fp64_rows(const double2 *rec, int n, const int32_t *act, double *out,
                                     double eps2, nb_ctl *ctl, cudaStream_t stream, int sm_count)
{
    cudaError_t e = set_smem_attr(eval_fp64_kernel<1>);
    if (e != cudaSuccess)
        return e;
    const int threads = 128, jt = 128;
    int lanes = 1;
    while (lanes < 32 && (static_cast<int64_t>(n) * lanes + threads - 1) / threads < 2 * sm_count)
        lanes *= 2;
    const int itile = threads / lanes;
    EvalArgs a;
    a.jb = rec;
    a.n = n;
    a.j0 = 0;
    a.j1 = n;
    a.act = act;
    a.n_act = n;
    a.out = out;
    a.ostride = n;
    a.part = nullptr;
    a.cnt = nullptr;
    a.jtile = jt;
    a.lanes = lanes;
    a.split = 1;
    a.jchunk = n;
    a.eps2 = eps2;
    a.ctl = ctl;
    a.tx_extra = 0;
    const size_t smem = static_cast<size_t>(2) * kRecBytes64 * jt;
    eval_fp64_kernel<1><<<(n + itile - 1) / itile, threads, smem, stream>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------ allocation-free variant
//
// For callers that must not allocate device memory, the FP64 evaluation can
// run with its split-j scratch (partial sums and arrival counters) in a
// fixed array that lives in the library image.  The array is reserved on
// every GPU that loads the library, for as long as the library stays loaded.

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr size_t kStaticCtlBytes = 256;                    // nb_ctl (error flags)
constexpr int kStaticMaxTiles = 4096;                      // arrival counters
constexpr size_t kStaticPartOffset = kStaticCtlBytes + sizeof(unsigned) * kStaticMaxTiles;
constexpr size_t kStaticPartDoubles = (kStaticScratchBytes - kStaticPartOffset) / sizeof(double);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
void *g_static_addr[kMaxDevices] = {};  // device address of g_static_scratch, per device

// Per-device set-up (with that device current): the array's device address
// and the kernel's shared-memory limit.  Host code may not use the array's
// name as an address; it is a host-side stand-in.
nb_status static_setup(int dev, void **addr)
{
    if (dev < 0 || dev >= kMaxDevices) {
        nb_set_thread_error("nb_evaluate_fp64_static: device ordinal out of range");
        return NB_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) {
            nb_set_thread_error(cudaGetErrorString(e));
            return NB_ECUDA;
        }
        e = set_smem_attr(eval_fp64_kernel<1>);
        if (e != cudaSuccess) {
            nb_set_thread_error(cudaGetErrorString(e));
            return NB_ECUDA;
        }
        g_static_addr[dev] = p;
    }
    *addr = g_static_addr[dev];
    return NB_OK;
}

}  // namespace

extern "C" nb_status nb_evaluate_fp64_static(const void *jrec, int64_t n, const int32_t *active,
                                             int64_t n_act, double eps, int32_t split, double *out,
                                             void *stream)
{
    // every argument check comes before the first CUDA call, so a rejected
    // call never launches or queues anything
    if (!jrec || !active || !out || n < 1 || n > 0x7fffffffLL || n_act < 0 || n_act > n ||
        split < 0 || !(eps >= 0x1p-60) || !(eps <= 1e18)) {
        nb_set_thread_error("nb_evaluate_fp64_static: invalid argument");
        return NB_EINVAL;
    }
    if ((reinterpret_cast<uintptr_t>(jrec) & 15) || (reinterpret_cast<uintptr_t>(active) & 3) ||
        (reinterpret_cast<uintptr_t>(out) & 7)) {
        nb_set_thread_error("nb_evaluate_fp64_static: jrec must be 16-byte, active 4-byte and out "
                            "8-byte aligned");
        return NB_EINVAL;
    }
    if (n_act == 0)
        return NB_OK;

    // launch shape: one i per thread slot, lanes share an i for small sets
    const int threads = 128, jt = 128;
    int lanes = 1;
    while (lanes < 32 && static_cast<int64_t>(threads / (2 * lanes)) >= n_act)
        lanes *= 2;
    const int itile = threads / lanes;
    const int64_t gx = (n_act + itile - 1) / itile;
    const size_t part_per_split = static_cast<size_t>(9) * n_act;
    if (split > 1) {
        int64_t chunk = (n + split - 1) / split;
        chunk = (chunk + jt - 1) / jt * jt;
        const int64_t splits = (n + chunk - 1) / chunk;
        if (splits > 65535) {
            nb_set_thread_error("nb_evaluate_fp64_static: split gives more than 65535 j-chunks");
            return NB_EINVAL;
        }
        if (static_cast<size_t>(splits) * part_per_split > kStaticPartDoubles || gx > kStaticMaxTiles) {
            nb_set_thread_error("nb_evaluate_fp64_static: split * 9 * n_act doubles exceed the "
                                "16 MiB static scratch");
            return NB_EINVAL;
        }
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        nb_set_thread_error(cudaGetErrorString(e));
        return NB_ECUDA;
    }
    void *base = nullptr;
    nb_status st = static_setup(dev, &base);
    if (st != NB_OK)
        return st;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        nb_set_thread_error(cudaGetErrorString(e));
        return NB_ECUDA;
    }

    int64_t s = split;
    if (s == 0) {
        // enough blocks to cover every SM four times, within the scratch
        const int64_t target = static_cast<int64_t>(sms) * 4;
        s = gx >= target ? 1 : (target + gx - 1) / gx;
        s = std::min<int64_t>(s, std::max<int64_t>(1, n / (2 * jt)));
        s = std::min<int64_t>(s, static_cast<int64_t>(kStaticPartDoubles / part_per_split));
        if (gx > kStaticMaxTiles)
            s = 1;
        s = std::max<int64_t>(1, std::min<int64_t>(s, 65535));
    }
    int64_t chunk = (n + s - 1) / s;
    chunk = (chunk + jt - 1) / jt * jt;
    const int splits = static_cast<int>((n + chunk - 1) / chunk);

    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    unsigned char *b = static_cast<unsigned char *>(base);
    // every call clears the error word and the counters it may use
    e = cudaMemsetAsync(b, 0, kStaticPartOffset, strm);
    if (e != cudaSuccess) {
        nb_set_thread_error(cudaGetErrorString(e));
        return NB_ECUDA;
    }
    EvalArgs a;
    a.jb = jrec;
    a.n = static_cast<int>(n);
    a.j0 = 0;
    a.j1 = static_cast<int>(n);
    a.act = active;
    a.n_act = static_cast<int>(n_act);
    a.out = out;
    a.ostride = static_cast<int>(n_act);
    a.part = splits > 1 ? reinterpret_cast<double *>(b + kStaticPartOffset) : nullptr;
    a.cnt = splits > 1 ? reinterpret_cast<unsigned *>(b + kStaticCtlBytes) : nullptr;
    a.jtile = jt;
    a.lanes = lanes;
    a.split = splits;
    a.jchunk = static_cast<int>(chunk);
    a.eps2 = eps * eps;
    a.ctl = reinterpret_cast<nb_ctl *>(b);
    a.tx_extra = 0;
    const size_t smem = static_cast<size_t>(2) * kRecBytes64 * jt;
    eval_fp64_kernel<1><<<dim3(static_cast<unsigned>(gx), splits), threads, smem, strm>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        nb_set_thread_error(cudaGetErrorString(e));
        return NB_ECUDA;
    }
    return NB_OK;
}
