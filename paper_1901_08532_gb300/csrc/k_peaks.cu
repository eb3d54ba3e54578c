// Throughput probes of the CUDA-core pipes the evaluation kernels run on:
// scalar and packed (f32x2) FP32 fused multiply-add, FP64 fused multiply-add,
// and the special-function estimates R^(-1/2) and 1/R, alone and mixed with
// packed FMAs in the proportion of the mixed pair term.  They give the
// measured denominators of the evaluation kernels' roofline: the pair sum is
// not a contraction, so its ceiling is the plain FP32 / FP64 pipe, not the
// tensor cores.
//
// Each thread runs NCH independent dependency chains, so that latency is
// hidden and the pipe, not the chain, sets the rate.  Every block records
// its own elapsed SM cycles (clock64), so the per-clock rate does not depend
// on the clock the GPU ran at; CUDA events give the per-second rate.
#include <algorithm>
#include <vector>

#include "nb_internal.cuh"

namespace {

constexpr int NCH = 8;  // independent chains per thread

__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_ftz(float x)
{
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_noftz(float x)
{
    float y;
    asm volatile("rsqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Operations (FMA = one operation, one estimate = one operation) a thread
// performs per loop iteration, by kind.
__host__ __device__ constexpr int probe_ops(int kind)
{
    // kinds: 0 FFMA, 1 FFMA2 (2 per instruction), 2 DFMA, 3 rsqrt, 4 rcp (+ 1 add each),
    // 5 FFMA2 + rsqrt (ftz), 6 FFMA2 + rsqrt (no ftz), 7 FFMA2 + rsqrt + rcp (ftz),
    // 8 FFMA2 with three distinct register operands
    return kind == 8 ? NCH * 12 * 2
         : kind == 0 ? NCH * 16
         : kind == 1 ? NCH * 16 * 2
         : kind == 2 ? NCH * 16
         : kind == 3 || kind == 4 ? NCH * 4
         : kind == 5 || kind == 6 ? NCH * (13 * 2)        // + NCH estimates, counted apart
         : NCH * (13 * 2 + 1);                              // + 2 NCH estimates (1 add per rcp)
}

__host__ __device__ constexpr int probe_est(int kind)
{
    return kind == 5 || kind == 6 ? NCH : kind == 7 ? 2 * NCH : 0;
}

// Kind 1 (packed FMAs alone) is the explicit specialisation below.
template <int KIND>
__global__ void peak_kernel(int iters, float seed, float *sink, long long *cycles)
{
    __syncthreads();
    const long long c0 = clock64();
    const float s = seed + 1e-3f * static_cast<float>(threadIdx.x & 7);
    if (KIND == 0) {
        float acc[NCH];
#pragma unroll
        for (int k = 0; k < NCH; ++k) acc[k] = s + k;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < 16; ++u)
#pragma unroll
                for (int k = 0; k < NCH; ++k) acc[k] = __fmaf_rn(acc[k], 0.999f, 1e-3f);
        float r = 0.f;
#pragma unroll
        for (int k = 0; k < NCH; ++k) r += acc[k];
        if (r == 12345.f) sink[threadIdx.x] = r;
    } else if (KIND == 2) {
        double acc[NCH];
#pragma unroll
        for (int k = 0; k < NCH; ++k) acc[k] = s + k;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < 16; ++u)
#pragma unroll
                for (int k = 0; k < NCH; ++k) acc[k] = __fma_rn(acc[k], 0.999, 1e-3);
        double r = 0.0;
#pragma unroll
        for (int k = 0; k < NCH; ++k) r += acc[k];
        if (r == 12345.0) sink[threadIdx.x] = static_cast<float>(r);
    } else if (KIND == 3 || KIND == 4) {
        float y[NCH];
#pragma unroll
        for (int k = 0; k < NCH; ++k) y[k] = s + 0.5f + k;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int k = 0; k < NCH; ++k)
                    // the 1/R chain adds 1 after each estimate (it converges to the golden
                    // ratio): a bare chain of reciprocals would let the compiler cancel
                    // them in pairs
                    y[k] = KIND == 3 ? rsqrt_ftz(y[k]) : rcp_ftz(y[k]) + 1.0f;
        float r = 0.f;
#pragma unroll
        for (int k = 0; k < NCH; ++k) r += y[k];
        if (r == 12345.f) sink[threadIdx.x] = r;
    } else if (KIND == 8) {
        // every f32x2 FMA reads three different register pairs, none of them
        // a loop constant: the register-operand bandwidth case of the pair
        // term (the values grow and overflow; the rate does not depend on them)
        float2 p[NCH], q[NCH], r[NCH];
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            p[k] = make_float2(s + k, s - k);
            q[k] = make_float2(0.5f * s, 0.25f * k);
            r[k] = make_float2(1.0f - s, 0.125f * k);
        }
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    p[k] = __ffma2_rn(q[k], r[k], p[k]);
                    q[k] = __ffma2_rn(r[k], p[k], q[k]);
                    r[k] = __ffma2_rn(p[k], q[k], r[k]);
                }
        float x = 0.f;
#pragma unroll
        for (int k = 0; k < NCH; ++k) x += p[k].x + q[k].y + r[k].x;
        if (x == 12345.f) sink[threadIdx.x] = x;
    } else {
        // packed FMAs with estimates interleaved: per chain and iteration 13
        // f32x2 FMAs (26 operations) and one (kinds 5, 6) or two (kind 7)
        // estimates on an independent chain, the proportion of the mixed
        // pair term (53 f32x2 operations and 4 estimates per two pairs)
        float2 acc[NCH];
        float y[NCH], z[NCH];
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            acc[k] = make_float2(s + k, s - k);
            y[k] = s + 0.5f + k;
            z[k] = s + 0.25f + k;
        }
        const float2 a2 = make_float2(0.999f, 0.998f), b2 = make_float2(1e-3f, 2e-3f);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
#pragma unroll
                for (int u = 0; u < 13; ++u) acc[k] = __ffma2_rn(acc[k], a2, b2);
                if (KIND == 5 || KIND == 7) y[k] = rsqrt_ftz(y[k]);
                if (KIND == 6) y[k] = rsqrt_noftz(y[k]);
                if (KIND == 7) z[k] = rcp_ftz(z[k]) + 1.0f;
            }
        float r = 0.f;
#pragma unroll
        for (int k = 0; k < NCH; ++k) r += acc[k].x + acc[k].y + y[k] + z[k];
        if (r == 12345.f) sink[threadIdx.x] = r;
    }
    __syncthreads();
    const long long c1 = clock64();
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = c1 - c0;
}

template <>
__global__ void peak_kernel<1>(int iters, float seed, float *sink, long long *cycles)
{
    __syncthreads();
    const long long c0 = clock64();
    const float s = seed + 1e-3f * static_cast<float>(threadIdx.x & 7);
    float2 acc[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) acc[k] = make_float2(s + k, s - k);
    const float2 a2 = make_float2(0.999f, 0.998f), b2 = make_float2(1e-3f, 2e-3f);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < NCH; ++k) acc[k] = __ffma2_rn(acc[k], a2, b2);
    float r = 0.f;
#pragma unroll
    for (int k = 0; k < NCH; ++k) r += acc[k].x + acc[k].y;
    if (r == 12345.f) sink[threadIdx.x] = r;
    __syncthreads();
    const long long c1 = clock64();
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = c1 - c0;
}

cudaError_t launch_probe(int kind, dim3 grid, dim3 block, int iters, float *sink, long long *cyc,
                         cudaStream_t s)
{
    switch (kind) {
    case 0: peak_kernel<0><<<grid, block, 0, s>>>(iters, 1.0f, sink, cyc); break;
    case 1: peak_kernel<1><<<grid, block, 0, s>>>(iters, 1.0f, sink, cyc); break;
    case 2: peak_kernel<2><<<grid, block, 0, s>>>(iters, 1.0f, sink, cyc); break;
    case 3: peak_kernel<3><<<grid, block, 0, s>>>(iters, 1.0f, sink, cyc); break;
    case 4: peak_kernel<4><<<grid, block, 0, s>>>(iters, 1.0f, sink, cyc); break;
    case 5: peak_kernel<5><<<grid, block, 0, s>>>(iters, 1.0f, sink, cyc); break;
    case 6: peak_kernel<6><<<grid, block, 0, s>>>(iters, 1.0f, sink, cyc); break;
    case 7: peak_kernel<7><<<grid, block, 0, s>>>(iters, 1.0f, sink, cyc); break;
    default: peak_kernel<8><<<grid, block, 0, s>>>(iters, 1.0f, sink, cyc); break;
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" nb_status nb_peak_probe(int32_t kind, int32_t blocks_per_sm, int32_t threads, int32_t iters,
                                   double *ops_per_clk_sm, double *ops_per_s, double *est_per_clk_sm,
                                   double *sm_mhz)
{
    if (kind < 0 || kind > 8 || blocks_per_sm < 1 || blocks_per_sm > 32 || threads < 32 ||
        threads > 1024 || threads % 32 || iters < 1 || iters > (1 << 24)) {
        nb_set_thread_error("nb_peak_probe: invalid argument");
        return NB_EINVAL;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nblk = sms * blocks_per_sm;
    float *sink = nullptr;
    long long *cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    std::vector<long long> hc(static_cast<size_t>(nblk));
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float) * 1024);
    if (e == cudaSuccess) e = cudaMalloc(&cyc, sizeof(long long) * nblk);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // warm-up launch (clocks up, code loaded), then the timed one
    if (e == cudaSuccess) e = launch_probe(kind, nblk, threads, std::max(1, iters / 8), sink, cyc, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_probe(kind, nblk, threads, iters, sink, cyc, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess)
        e = cudaMemcpy(hc.data(), cyc, sizeof(long long) * nblk, cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    cudaFree(cyc);
    if (e != cudaSuccess) {
        nb_set_thread_error(cudaGetErrorString(e));
        return NB_ECUDA;
    }
    // every SM holds blocks_per_sm blocks at once; the slowest block's
    // cycles bound the SM's time
    const double cycles = static_cast<double>(*std::max_element(hc.begin(), hc.end()));
    const double per_thread = static_cast<double>(iters) * probe_ops(kind);
    const double est_thread = static_cast<double>(iters) * probe_est(kind);
    const double per_sm = per_thread * threads * blocks_per_sm;
    if (ops_per_clk_sm) *ops_per_clk_sm = per_sm / cycles;
    if (est_per_clk_sm) *est_per_clk_sm = est_thread * threads * blocks_per_sm / cycles;
    if (ops_per_s) *ops_per_s = per_sm * sms / (ms * 1e-3);
    if (sm_mhz) *sm_mhz = cycles / (ms * 1e-3) / 1e6;
    return NB_OK;
}
