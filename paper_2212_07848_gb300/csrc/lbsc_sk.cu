// Density structure factor S(k) = <|delta n(k)|^2> (defined after Eq. (12)
// of arXiv:2212.07848) accumulated on the device.
//
// One sample: delta rho [ny][nx] (written by the step kernel on sampling
// steps) -> row FFTs (two real rows packed into one complex transform) ->
// half spectrum [ny][ldx] -> column FFTs over tiles of adjacent columns ->
// acc[ky][kx] += |X(k)|^2 / (nx ny) in FP64.  The transforms are iterative
// radix-2 decimation-in-time FFTs in shared memory over power-of-two sizes,
// with twiddle tables computed once in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lbsc_fft.cuh"
#include "lbsc_internal.cuh"

namespace lbsc {

// Twiddles e^{-2 pi i m / n}, m < n/2, evaluated in FP64.
template <typename T>
__global__ void twiddle_kernel(typename C2<T>::t *tw, int n) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n / 2) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    typename C2<T>::t v;
    v.x = (T)c;
    v.y = (T)(-s);
    tw[m] = v;
}

cudaError_t launch_twiddles(int precision, void *tw, int n, cudaStream_t s) {
    const int blocks = (n / 2 + 255) / 256;
    if (precision == 0)
        twiddle_kernel<float><<<blocks, 256, 0, s>>>((float2 *)tw, n);
    else
        twiddle_kernel<double><<<blocks, 256, 0, s>>>((double2 *)tw, n);
    return cudaGetLastError();
}

template <typename T>
__global__ void sk_rows_kernel(const T *__restrict__ drho, typename C2<T>::t *__restrict__ spec,
                               const typename C2<T>::t *__restrict__ tw, int nx, int log2nx,
                               int ldx) {
    sk_rows_block<T>(drho, spec, tw, nx, log2nx, ldx, blockIdx.x);
}

template <typename T>
__global__ void sk_cols_kernel(const typename C2<T>::t *__restrict__ spec, double *__restrict__ acc,
                               const typename C2<T>::t *__restrict__ tw, int nx, int ny,
                               int log2ny, int ldx, int cpb, double inv_n) {
    sk_cols_block<T>(spec, acc, tw, nx, ny, log2ny, ldx, cpb, inv_n, blockIdx.x * cpb);
}

template <typename T>
static cudaError_t sk_sample_t(const SkArgs &a, cudaStream_t s) {
    using CT = typename C2<T>::t;
    const int lx = ilog2(a.nx), ly = ilog2(a.ny);
    const size_t row_smem = (size_t)a.nx * sizeof(CT);
    const int cpb = cols_per_block(a.ny, sizeof(CT));
    const size_t col_smem = (size_t)cpb * a.ny * sizeof(CT);
    cudaError_t e;
    e = cudaFuncSetAttribute(sk_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)row_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sk_cols_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)col_smem);
    if (e != cudaSuccess) return e;
    const int rthreads = a.nx / 2 < 512 ? (a.nx / 2 < 32 ? 32 : a.nx / 2) : 512;
    sk_rows_kernel<T><<<a.ny / 2, rthreads, row_smem, s>>>(
        (const T *)a.drho, (CT *)a.spec, (const CT *)a.tw_x, a.nx, lx, a.ldx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int hx = a.nx / 2 + 1;
    const int cblocks = (hx + cpb - 1) / cpb;
    sk_cols_kernel<T><<<cblocks, 512, col_smem, s>>>((const CT *)a.spec, a.acc,
                                                     (const CT *)a.tw_y, a.nx, a.ny, ly,
                                                     a.ldx, cpb, 1.0 / ((double)a.nx * a.ny));
    return cudaGetLastError();
}

cudaError_t launch_sk_sample(int precision, const SkArgs &a, cudaStream_t s) {
    return precision == 0 ? sk_sample_t<float>(a, s) : sk_sample_t<double>(a, s);
}

// Mean over samples on the half plane, host layout [ny][nx/2+1]; k = 0 -> 0.
__global__ void sk_readout_kernel(const double *__restrict__ acc, double inv_count,
                                  double *__restrict__ out, int nx, int ny, int ldx) {
    const int hx = nx / 2 + 1;
    const size_t total = (size_t)hx * ny;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int ky = (int)(e / hx), kx = (int)(e % hx);
        out[e] = (kx == 0 && ky == 0) ? 0.0 : acc[(size_t)ky * ldx + kx] * inv_count;
    }
}

cudaError_t launch_sk_readout(const double *acc, double inv_count, double *out, int nx, int ny,
                              int ldx, cudaStream_t s) {
    const size_t total = (size_t)(nx / 2 + 1) * ny;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    sk_readout_kernel<<<blocks, 256, 0, s>>>(acc, inv_count, out, nx, ny, ldx);
    return cudaGetLastError();
}

// Radial bins over the full plane: bin b = round(|k| / dk), dk = 2 pi / max(nx, ny);
// a half-plane column 0 < kx < nx/2 stands for two modes (k and -k).
__global__ void sk_bins_kernel(const double *__restrict__ acc, double inv_count,
                               double *__restrict__ bins, double *__restrict__ counts, int nbins,
                               int nx, int ny, int ldx) {
    const int hx = nx / 2 + 1;
    const size_t total = (size_t)hx * ny;
    const double L = (double)(nx > ny ? nx : ny);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int ky = (int)(e / hx), kx = (int)(e % hx);
        if (kx == 0 && ky == 0) continue;
        const int my = ky <= ny / 2 ? ky : ky - ny;
        const double qx = (double)kx * (L / nx), qy = (double)my * (L / ny);
        const int b = (int)rint(sqrt(qx * qx + qy * qy));
        if (b >= nbins) continue;
        const double w = (kx == 0 || 2 * kx == nx) ? 1.0 : 2.0;
        atomicAdd(&bins[b], w * acc[(size_t)ky * ldx + kx] * inv_count);
        atomicAdd(&counts[b], w);
    }
}

cudaError_t launch_sk_bins(const double *acc, double inv_count, double *bins, double *counts,
                           int nbins, int nx, int ny, int ldx, cudaStream_t s) {
    const size_t total = (size_t)(nx / 2 + 1) * ny;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    sk_bins_kernel<<<blocks, 256, 0, s>>>(acc, inv_count, bins, counts, nbins, nx, ny, ldx);
    return cudaGetLastError();
}

}  // namespace lbsc

namespace lbsc {

// First moments of the mean S(k) over the full plane (k = 0 excluded):
// out = (sum_k S(k), sum_k |k| S(k)), |k| = 2 pi sqrt((kx/nx)^2 + (ky/ny)^2)
// with folded indices; a half-plane column 0 < kx < nx/2 counts twice.  One
// block, fixed summation order.
__global__ void __launch_bounds__(256)
sk_moments_kernel(const double *__restrict__ acc, double inv_count, int nx, int ny, int ldx,
                  double *__restrict__ out) {
    const int hx = nx / 2 + 1;
    double s0 = 0.0, s1 = 0.0;
    for (int e = threadIdx.x; e < hx * ny; e += blockDim.x) {
        const int ky = e / hx, kx = e % hx;
        if (kx == 0 && ky == 0) continue;
        const int my = ky <= ny / 2 ? ky : ky - ny;
        const double w = (kx == 0 || 2 * kx == nx) ? 1.0 : 2.0;
        const double S = acc[(size_t)ky * ldx + kx] * inv_count;
        const double qx = (double)kx / nx, qy = (double)my / ny;
        s0 += w * S;
        s1 += w * S * 6.283185307179586 * sqrt(qx * qx + qy * qy);
    }
    __shared__ double sh0[256], sh1[256];
    sh0[threadIdx.x] = s0;
    sh1[threadIdx.x] = s1;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh0[threadIdx.x] += sh0[threadIdx.x + o];
            sh1[threadIdx.x] += sh1[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh0[0];
        out[1] = sh1[0];
    }
}

cudaError_t launch_sk_moments(const double *acc, double inv_count, int nx, int ny, int ldx,
                              double *out2, cudaStream_t s) {
    sk_moments_kernel<<<1, 256, 0, s>>>(acc, inv_count, nx, ny, ldx, out2);
    return cudaGetLastError();
}

}  // namespace lbsc
