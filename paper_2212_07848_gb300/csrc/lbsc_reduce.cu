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

#include <mutex>

#include "lbsc.h"
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

// Mass and momentum deviations of one site added to FP64 running sums.  An
// FP32 state combines its nine deviations in FP32 (the rounding of that
// 9-term sum, ~2^-24 of the deviations, is at the storage precision itself)
// and only the three site totals go through FP64, whose throughput on this
// GPU is a small fraction of FP32's; an FP64 state is summed in FP64.
__device__ __forceinline__ void add_site_moments(const float *__restrict__ df, size_t plane,
                                                 size_t s, double &m, double &jx, double &jy) {
    float g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = df[i * plane + s];
    m += (double)(((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8])));
    jx += (double)((g[1] - g[3]) + (g[5] - g[7]) + (g[8] - g[6]));
    jy += (double)((g[2] - g[4]) + (g[5] - g[7]) + (g[6] - g[8]));
}
__device__ __forceinline__ void add_site_moments(const double *__restrict__ df, size_t plane,
                                                 size_t s, double &m, double &jx, double &jy) {
    double g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = df[i * plane + s];
    m += ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
    jx += (g[1] - g[3]) + (g[5] - g[7]) + (g[8] - g[6]);
    jy += (g[2] - g[4]) + (g[5] - g[7]) + (g[6] - g[8]);
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
conserved_partials_kernel(const T *__restrict__ df, size_t plane, double *__restrict__ partials) {
    double m = 0.0, jx = 0.0, jy = 0.0;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < plane;
         s += (size_t)gridDim.x * blockDim.x) {
        add_site_moments(df, plane, s, m, jx, jy);
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

// ---------------------------------------------------------------------------
// Allocation-free variant for callers that must not call cudaMalloc (for
// example a host application whose device memory is all owned by its own
// pool, or a loop that cannot accept the device-wide synchronisation an
// allocation implies).  The per-block partial sums live in a fixed device
// array inside this library instead of a context buffer.
// ---------------------------------------------------------------------------
namespace lbsc {

constexpr int kStaticSitesPerBlock = kRedThreads * 16;      // 4096 sites per block
constexpr int kStaticMaxBlocks = 4096;                      // up to 4096 x 4096 sites
static __device__ __align__(256) double g_conserved_scratch[3 * kStaticMaxBlocks];

// One block per contiguous chunk of kStaticSitesPerBlock sites; every block
// writes its own partial triple, so no slot has to start at zero.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
conserved_chunk_kernel(const T *__restrict__ df, size_t plane, double *__restrict__ partials) {
    double m = 0.0, jx = 0.0, jy = 0.0;
    const size_t begin = (size_t)blockIdx.x * kStaticSitesPerBlock;
    size_t end = begin + kStaticSitesPerBlock;
    if (end > plane) end = plane;
    for (size_t s = begin + threadIdx.x; s < end; s += kRedThreads) {
        add_site_moments(df, plane, s, m, jx, jy);
    }
    block_sum3(m, jx, jy);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = m;
        partials[3 * blockIdx.x + 1] = jx;
        partials[3 * blockIdx.x + 2] = jy;
    }
}

__global__ void __launch_bounds__(kRedThreads)
conserved_static_final_kernel(const double *__restrict__ partials, int nblocks, double mass0,
                              double *__restrict__ out3) {
    double m = 0.0, jx = 0.0, jy = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        m += partials[3 * b + 0];
        jx += partials[3 * b + 1];
        jy += partials[3 * b + 2];
    }
    block_sum3(m, jx, jy);
    if (threadIdx.x == 0) {
        out3[0] = mass0 + m;
        out3[1] = jx;
        out3[2] = jy;
    }
}

namespace {
// Device address of g_conserved_scratch, looked up once per device with that
// device current (in host code the symbol names a host-side stand-in).  It is
// kept until the process exits; a reset of the device's primary context makes
// it stale (the header says so).
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double *g_scratch_addr[kMaxDevices] = {nullptr};

int scratch_for_current_device(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_conserved_scratch) != cudaSuccess || !p) return LB_ERR_CUDA;
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return LB_OK;
}
}  // namespace

}  // namespace lbsc

extern "C" int lb_conserved_static(const void *d_df, int precision, int nx, int ny, double rho0,
                                   double *d_out3, void *stream) {
    using namespace lbsc;
    if (!d_df || !d_out3 || nx < 1 || ny < 1) return LB_ERR_ARG;
    if (precision != LB_FP32 && precision != LB_FP64) return LB_ERR_ARG;
    const size_t plane = (size_t)nx * (size_t)ny;
    if (plane > (size_t)kStaticSitesPerBlock * kStaticMaxBlocks) return LB_ERR_UNSUPPORTED;
    double *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != LB_OK) return rc;
    const int nblocks = (int)((plane + kStaticSitesPerBlock - 1) / kStaticSitesPerBlock);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == LB_FP32)
        conserved_chunk_kernel<float><<<nblocks, kRedThreads, 0, s>>>((const float *)d_df, plane,
                                                                      scratch);
    else
        conserved_chunk_kernel<double><<<nblocks, kRedThreads, 0, s>>>((const double *)d_df,
                                                                       plane, scratch);
    if (cudaGetLastError() != cudaSuccess) return LB_ERR_CUDA;
    conserved_static_final_kernel<<<1, kRedThreads, 0, s>>>(scratch, nblocks,
                                                           (double)plane * rho0, d_out3);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}
