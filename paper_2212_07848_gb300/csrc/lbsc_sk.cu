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

#include "lbsc_internal.cuh"

namespace lbsc {

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <typename CT>
__device__ __forceinline__ CT cmul(CT a, CT b) {
    CT r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

static inline int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// In-place radix-2 DIT over `nfft` independent transforms of length n stored
// contiguously in shared memory (input already in bit-reversed order).
template <typename CT>
__device__ void fft_smem(CT *s, int n, int log2n, int nfft, const CT *__restrict__ tw) {
    const int half = n >> 1;
    const int total = nfft * half;
    for (int l = 0; l < log2n; ++l) {
        const int m = 1 << l;                 // half-size of the butterflies
        const int stride = half >> l;         // twiddle index stride: n / (2m)
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int f = b / half;
            const int t = b - f * half;
            const int j = t & (m - 1);
            const int base = f * n + ((t >> l) << (l + 1)) + j;
            const CT w = tw[j * stride];
            const CT u = s[base];
            const CT v = cmul(s[base + m], w);
            CT a, c;
            a.x = u.x + v.x; a.y = u.y + v.y;
            c.x = u.x - v.x; c.y = u.y - v.y;
            s[base] = a;
            s[base + m] = c;
        }
        __syncthreads();
    }
}

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

// Row pass: block b transforms rows 2b and 2b+1 packed as z = a + i b and
// separates X_a(k) = (Z(k) + conj Z(n-k)) / 2, X_b(k) = (Z(k) - conj Z(n-k)) / 2i.
template <typename T>
__global__ void sk_rows_kernel(const T *__restrict__ drho, typename C2<T>::t *__restrict__ spec,
                               const typename C2<T>::t *__restrict__ tw, int nx, int log2nx,
                               int ldx) {
    using CT = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *s = reinterpret_cast<CT *>(smem_raw);
    const int ya = 2 * blockIdx.x, yb = ya + 1;
    const T *ra = drho + (size_t)ya * nx;
    const T *rb = drho + (size_t)yb * nx;
    for (int j = threadIdx.x; j < nx; j += blockDim.x) {
        CT v;
        v.x = ra[j];
        v.y = rb[j];
        s[__brev((unsigned)j) >> (32 - log2nx)] = v;
    }
    __syncthreads();
    fft_smem<CT>(s, nx, log2nx, 1, tw);
    CT *oa = spec + (size_t)ya * ldx;
    CT *ob = spec + (size_t)yb * ldx;
    for (int k = threadIdx.x; k <= nx / 2; k += blockDim.x) {
        const CT z = s[k];
        const CT zc = s[(nx - k) & (nx - 1)];
        CT xa, xb;
        xa.x = T(0.5) * (z.x + zc.x);
        xa.y = T(0.5) * (z.y - zc.y);
        // (z - conj(zc)) / (2i) = -(i/2) (z - conj(zc))
        xb.x = T(0.5) * (z.y + zc.y);
        xb.y = T(-0.5) * (z.x - zc.x);
        oa[k] = xa;
        ob[k] = xb;
    }
}

// Column pass: block b transforms columns kx0 .. kx0+cpb-1 (length ny) and
// accumulates |X|^2 / N.
template <typename T>
__global__ void sk_cols_kernel(const typename C2<T>::t *__restrict__ spec, double *__restrict__ acc,
                               const typename C2<T>::t *__restrict__ tw, int nx, int ny,
                               int log2ny, int ldx, int cpb, double inv_n) {
    using CT = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *s = reinterpret_cast<CT *>(smem_raw);
    const int hx = nx / 2 + 1;
    const int kx0 = blockIdx.x * cpb;
    const int total = cpb * ny;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int c = e % cpb, y = e / cpb;
        CT v;
        if (kx0 + c < hx) {
            v = spec[(size_t)y * ldx + kx0 + c];
        } else {
            v.x = T(0);
            v.y = T(0);
        }
        s[c * ny + (__brev((unsigned)y) >> (32 - log2ny))] = v;
    }
    __syncthreads();
    fft_smem<CT>(s, ny, log2ny, cpb, tw);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int c = e % cpb, ky = e / cpb;
        if (kx0 + c >= hx) continue;
        const CT v = s[c * ny + ky];
        const double re = (double)v.x, im = (double)v.y;
        acc[(size_t)ky * ldx + kx0 + c] += (re * re + im * im) * inv_n;
    }
}

static int cols_per_block(int ny, size_t csize) {
    int cpb = 4;
    while (cpb > 1 && (size_t)cpb * ny * csize > 128 * 1024) cpb >>= 1;
    return cpb;
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
