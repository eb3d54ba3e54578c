// Energy and angular momentum of the current state (paper, section 3 item 3:
// both are evaluated on the device and checked periodically; Eq. 1 defines
// their relative errors).  FP64 throughout, deterministic: per-block sums in
// a fixed tree order, then one block adds the block sums in index order.
//   E_kin = sum 1/2 m_i |v_i|^2
//   E_pot = -sum_{i<j} m_i m_j / sqrt(|r_ij|^2 + eps^2)
//         = 1/2 sum_i m_i phi_i,  phi_i = -sum_{j != i} m_j / sqrt(...)
//   L     = sum m_i x_i cross v_i,  and sum m_i |x_i cross v_i|
#include "nb_internal.cuh"

namespace {

constexpr int kT = 256;
constexpr int kTile = 256;

template <int NV>
__device__ void block_sum(double (&v)[NV], double *out)
{
    __shared__ double s[NV][kT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = v[q];
        for (int off = 16; off > 0; off >>= 1)
            x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0)
            s[q][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double x = 0.0;
            for (int w = 0; w < kT / 32; ++w)
                x += s[q][w];
            out[q] = x;
        }
    }
}

__global__ void __launch_bounds__(kT) energy_kernel(const double *st, const double *m, int n,
                                                    double eps2, double *blocksums)
{
    __shared__ double sx[kTile], sy[kTile], sz[kTile], sm[kTile];
    const size_t N = static_cast<size_t>(n);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const int ii = valid ? i : 0;
    const double xi = st[(F_X * 3 + 0) * N + ii], yi = st[(F_X * 3 + 1) * N + ii],
                 zi = st[(F_X * 3 + 2) * N + ii];
    double phi = 0.0;
    for (int j0 = 0; j0 < n; j0 += kTile) {
        __syncthreads();
        for (int q = threadIdx.x; q < kTile; q += blockDim.x) {
            const int j = j0 + q;
            const bool ok = j < n;
            sx[q] = ok ? st[(F_X * 3 + 0) * N + j] : 0.0;
            sy[q] = ok ? st[(F_X * 3 + 1) * N + j] : 0.0;
            sz[q] = ok ? st[(F_X * 3 + 2) * N + j] : 0.0;
            sm[q] = ok ? m[j] : 0.0;
        }
        __syncthreads();
        const int len = min(kTile, n - j0);
        double part = 0.0;
        for (int q = 0; q < len; ++q) {
            const double dx = sx[q] - xi, dy = sy[q] - yi, dz = sz[q] - zi;
            const double r = sqrt(fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2))));
            part += (j0 + q == i) ? 0.0 : sm[q] / r;
        }
        phi += part;
    }
    double v[2] = {0.0, 0.0};
    if (valid) {
        const double vx = st[(F_V * 3 + 0) * N + i], vy = st[(F_V * 3 + 1) * N + i],
                     vz = st[(F_V * 3 + 2) * N + i];
        v[0] = 0.5 * m[i] * fma(vx, vx, fma(vy, vy, vz * vz));
        v[1] = -0.5 * m[i] * phi;
    }
    block_sum<2>(v, blocksums + 2 * blockIdx.x);
}

__global__ void __launch_bounds__(kT) angmom_kernel(const double *st, const double *m, int n,
                                                    double *blocksums)
{
    const size_t N = static_cast<size_t>(n);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < n) {
        const double x = st[(F_X * 3 + 0) * N + i], y = st[(F_X * 3 + 1) * N + i],
                     z = st[(F_X * 3 + 2) * N + i];
        const double vx = st[(F_V * 3 + 0) * N + i], vy = st[(F_V * 3 + 1) * N + i],
                     vz = st[(F_V * 3 + 2) * N + i];
        const double lx = y * vz - z * vy, ly = z * vx - x * vz, lz = x * vy - y * vx;
        v[0] = m[i] * lx;
        v[1] = m[i] * ly;
        v[2] = m[i] * lz;
        v[3] = m[i] * sqrt(lx * lx + ly * ly + lz * lz);
    }
    block_sum<4>(v, blocksums + 4 * blockIdx.x);
}

// Sum nv interleaved block sums in block order (one thread per value).
__global__ void final_sum_kernel(const double *blocksums, int nblocks, int nv, double *out)
{
    const int q = threadIdx.x;
    if (q >= nv)
        return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b)
        s += blocksums[b * nv + q];
    out[q] = s;
}

cudaError_t ensure_red(nb_ctx *c, size_t doubles)
{
    if (doubles <= c->red_cap)
        return cudaSuccess;
    cudaFree(c->red);
    c->red = nullptr;
    c->red_cap = 0;
    cudaError_t e = cudaMalloc(&c->red, doubles * sizeof(double));
    if (e == cudaSuccess)
        c->red_cap = doubles;
    return e;
}

}  // namespace

// out_dev[0] = E_kin, out_dev[1] = E_pot (device memory, 2 doubles).
cudaError_t nb_launch_energy(nb_ctx *c, double *out_dev)
{
    const int n = static_cast<int>(c->n);
    const int nb = (n + kT - 1) / kT;
    cudaError_t e = ensure_red(c, static_cast<size_t>(2) * nb);
    if (e != cudaSuccess)
        return e;
    energy_kernel<<<nb, kT, 0, c->stream>>>(c->st, c->m, n, c->eps * c->eps, c->red);
    final_sum_kernel<<<1, 32, 0, c->stream>>>(c->red, nb, 2, out_dev);
    c->launches += 2;
    return cudaGetLastError();
}

// out_dev[0..2] = L, out_dev[3] = sum m |x cross v|.
cudaError_t nb_launch_angmom(nb_ctx *c, double *out_dev)
{
    const int n = static_cast<int>(c->n);
    const int nb = (n + kT - 1) / kT;
    cudaError_t e = ensure_red(c, static_cast<size_t>(4) * nb);
    if (e != cudaSuccess)
        return e;
    angmom_kernel<<<nb, kT, 0, c->stream>>>(c->st, c->m, n, c->red);
    final_sum_kernel<<<1, 32, 0, c->stream>>>(c->red, nb, 4, out_dev);
    c->launches += 2;
    return cudaGetLastError();
}
