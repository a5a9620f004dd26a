// Shared-memory FFT blocks of the structure-factor sample (used by the
// single-lattice and the batched ensemble kernels): iterative radix-2
// decimation-in-time transforms over power-of-two sizes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbsc {

inline int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

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

// Row pass: block b transforms rows 2b and 2b+1 packed as z = a + i b and
// separates X_a(k) = (Z(k) + conj Z(n-k)) / 2, X_b(k) = (Z(k) - conj Z(n-k)) / 2i.
template <typename T>
__device__ __forceinline__ void sk_rows_block(const T *__restrict__ drho,
                                              typename C2<T>::t *__restrict__ spec,
                                              const typename C2<T>::t *__restrict__ tw, int nx,
                                              int log2nx, int ldx, int pair) {
    using CT = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *s = reinterpret_cast<CT *>(smem_raw);
    const int ya = 2 * pair, yb = ya + 1;
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
__device__ __forceinline__ void sk_cols_block(const typename C2<T>::t *__restrict__ spec,
                                              double *__restrict__ acc,
                                              const typename C2<T>::t *__restrict__ tw, int nx,
                                              int ny, int log2ny, int ldx, int cpb, double inv_n,
                                              int kx0) {
    using CT = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *s = reinterpret_cast<CT *>(smem_raw);
    const int hx = nx / 2 + 1;
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


inline int cols_per_block(int ny, size_t csize) {
    int cpb = 4;
    while (cpb > 1 && (size_t)cpb * ny * csize > 128 * 1024) cpb >>= 1;
    return cpb;
}

}  // namespace lbsc
