// Block-time-step scheduler (paper, section 2: block time steps): the next
// time is t_next = min_i(t_i + dt_i) and the active set is every i with
// t_i + dt_i == t_next, listed in ascending index order.  All times are
// dyadic rationals, so the sums and the equality test are exact.
//
// Three small launches over the 16 bytes/particle of (t, dt):
//   1. min-reduction (positive doubles order like their bit patterns, so an
//      integer atomicMin on the bits is exact),
//   2. per-block counts of due particles,
//   3. ordered compaction: each block adds the counts of the blocks before
//      it, scans its own flags and writes indices; the last block stores
//      n_act.
#include "nb_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 4;
constexpr int kPerBlock = kThreads * kPerThread;

__global__ void __launch_bounds__(kThreads) tmin_kernel(const double *t, const double *dt, int n,
                                                        nb_ctl *ctl)
{
    unsigned long long best = ~0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(t[i] + dt[i]));
        best = b < best ? b : best;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
        best = o < best ? o : best;
    }
    if ((threadIdx.x & 31) == 0)
        atomicMin(&ctl->tnext_bits, best);
}

__device__ __forceinline__ bool due(const double *t, const double *dt, int i, double tn)
{
    return t[i] + dt[i] == tn;
}

__global__ void __launch_bounds__(kThreads) count_kernel(const double *t, const double *dt, int n,
                                                         const nb_ctl *ctl, int32_t *blk)
{
    __shared__ int s_cnt[kThreads / 32];
    const double tn = __longlong_as_double(static_cast<long long>(ctl->tnext_bits));
    const int base = blockIdx.x * kPerBlock + threadIdx.x * kPerThread;
    int c = 0;
#pragma unroll
    for (int q = 0; q < kPerThread; ++q)
        c += (base + q < n && due(t, dt, base + q, tn)) ? 1 : 0;
    for (int off = 16; off > 0; off >>= 1)
        c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0)
        s_cnt[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kThreads / 32; ++w)
            s += s_cnt[w];
        blk[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kThreads) compact_kernel(const double *t, const double *dt, int n,
                                                           nb_ctl *ctl, const int32_t *blk,
                                                           int32_t *act)
{
    __shared__ int s_w[kThreads / 32];
    __shared__ int s_prefix;
    const double tn = __longlong_as_double(static_cast<long long>(ctl->tnext_bits));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // counts of all earlier blocks
    int pre = 0;
    for (int b = threadIdx.x; b < static_cast<int>(blockIdx.x); b += blockDim.x)
        pre += blk[b];
    for (int off = 16; off > 0; off >>= 1)
        pre += __shfl_xor_sync(0xffffffffu, pre, off);
    if (lane == 0)
        s_w[warp] = pre;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kThreads / 32; ++w)
            s += s_w[w];
        s_prefix = s;
    }
    __syncthreads();

    const int base = blockIdx.x * kPerBlock + threadIdx.x * kPerThread;
    bool f[kPerThread];
    int c = 0;
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
        f[q] = base + q < n && due(t, dt, base + q, tn);
        c += f[q] ? 1 : 0;
    }
    // exclusive scan of c over the block: warp inclusive scan, then warp totals
    int incl = c;
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off)
            incl += o;
    }
    if (lane == 31)
        s_w[warp] = incl;
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w)
        wbase += s_w[w];
    int pos = s_prefix + wbase + incl - c;
#pragma unroll
    for (int q = 0; q < kPerThread; ++q)
        if (f[q])
            act[pos++] = base + q;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kThreads - 1)
        ctl->n_act = pos;
}

__global__ void iota_kernel(int32_t *act, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        act[i] = i;
}

}  // namespace

cudaError_t nb_launch_schedule(nb_ctx *c)
{
    const int n = static_cast<int>(c->n);
    cudaError_t e = cudaMemsetAsync(&c->ctl->tnext_bits, 0xff, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess)
        return e;
    int g1 = (n + kThreads - 1) / kThreads;
    g1 = g1 < c->sm_count * 8 ? g1 : c->sm_count * 8;
    tmin_kernel<<<g1, kThreads, 0, c->stream>>>(c->t, c->dt, n, c->ctl);
    const int nb = (n + kPerBlock - 1) / kPerBlock;
    count_kernel<<<nb, kThreads, 0, c->stream>>>(c->t, c->dt, n, c->ctl, c->blk);
    compact_kernel<<<nb, kThreads, 0, c->stream>>>(c->t, c->dt, n, c->ctl, c->blk, c->act_next);
    c->launches += 3;
    return cudaGetLastError();
}

cudaError_t nb_launch_iota(nb_ctx *c, int n, int32_t *dst)
{
    iota_kernel<<<(n + 255) / 256, 256, 0, c->stream>>>(dst, n);
    c->launches += 1;
    return cudaGetLastError();
}
