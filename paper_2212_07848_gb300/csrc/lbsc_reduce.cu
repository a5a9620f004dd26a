// Conserved moments of the stored state: total mass sum_x rho and momentum
// sum_x j in FP64 (the collision and the zero-noise conserved modes keep
// them constant, so their drift is the conservation check of Eq. (12) with
// the noise of the paragraph after Eq. (16)).
//
// Two passes with a fixed launch shape, so the summation order -- and the
// FP64 result -- is the same on every call: a grid-stride pass with warp
// shuffles and a shared-memory tree writes one partial triple per block; one
// block then adds the partials in a fixed order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbsc_internal.cuh"

namespace lbsc {

constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 152 * 8;

int conserved_blocks(int nx, int ny) {
    const size_t n = (size_t)nx * ny;
    size_t b = (n + kRedThreads - 1) / kRedThreads;
    return (int)(b < (size_t)kRedMaxBlocks ? b : (size_t)kRedMaxBlocks);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide fixed-order sum of three values; result valid in thread 0.
__device__ __forceinline__ void block_sum3(double &a, double &b, double &c) {
    __shared__ double sh[3][kRedThreads / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = a;
        sh[1][wid] = b;
        sh[2][wid] = c;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? sh[0][lane] : 0.0;
        b = lane < nw ? sh[1][lane] : 0.0;
        c = lane < nw ? sh[2][lane] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_sum(c);
    }
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
conserved_partials_kernel(const T *__restrict__ df, size_t plane, double *__restrict__ partials) {
    double m = 0.0, jx = 0.0, jy = 0.0;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < plane;
         s += (size_t)gridDim.x * blockDim.x) {
        double g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = (double)df[i * plane + s];
        m += ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
        jx += (g[1] - g[3]) + (g[5] - g[7]) + (g[8] - g[6]);
        jy += (g[2] - g[4]) + (g[5] - g[7]) + (g[6] - g[8]);
    }
    block_sum3(m, jx, jy);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = m;
        partials[3 * blockIdx.x + 1] = jx;
        partials[3 * blockIdx.x + 2] = jy;
    }
}

// out = (N rho0 + sum delta rho, sum jx, sum jy); rho0 term added on the host.
__global__ void __launch_bounds__(kRedThreads)
conserved_final_kernel(const double *__restrict__ partials, int nblocks, double *__restrict__ out3) {
    double m = 0.0, jx = 0.0, jy = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        m += partials[3 * b + 0];
        jx += partials[3 * b + 1];
        jy += partials[3 * b + 2];
    }
    block_sum3(m, jx, jy);
    if (threadIdx.x == 0) {
        out3[0] = m;
        out3[1] = jx;
        out3[2] = jy;
    }
}

cudaError_t launch_conserved(int precision, const void *df, double *partials, int nblocks,
                             double *out3, int nx, int ny, cudaStream_t s) {
    const size_t plane = (size_t)nx * ny;
    if (precision == 0)
        conserved_partials_kernel<float><<<nblocks, kRedThreads, 0, s>>>((const float *)df, plane,
                                                                         partials);
    else
        conserved_partials_kernel<double><<<nblocks, kRedThreads, 0, s>>>((const double *)df,
                                                                          plane, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    conserved_final_kernel<<<1, kRedThreads, 0, s>>>(partials, nblocks, out3);
    return cudaGetLastError();
}

}  // namespace lbsc
