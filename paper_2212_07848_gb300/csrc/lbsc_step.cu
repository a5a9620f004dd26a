// Fused fluctuating Shan-Chen D2Q9 time step (Eq. (12) of arXiv:2212.07848):
// pull streaming -> density -> pseudopotential on the tile and its halo ->
// Shan-Chen force, Eq. (1) -> moments -> BGK + Guo source -> Philox noise on
// the non-conserved moments -> inverse transform -> store.
//
// Layout: populations are stored as deviations delta f_i = f_i - w_i rho0,
// structure of arrays [9][ny][nx] (x fastest), two buffers swapped per step.
// Storing deviations keeps the relative precision of density fluctuations of
// size sqrt(kT) in FP32.
//
// Work decomposition: a CTA owns a strip of columns and sweeps strip_h rows
// downwards.  Each iteration pulls one new row (one thread per column),
// writes the pseudopotential deviation of that row into a shared-memory ring
// of rows, and collides the row H above it, whose 2H+1 pseudopotential rows
// are then complete.  The pulled populations of the last H+1 rows stay in
// registers, so every population is read from DRAM once per step (halo rows
// and columns are re-read from L2 only at strip boundaries).  Two layouts
// of the halo columns: step_kernel (128 columns per CTA and a fifth warp
// that only pulls the 2H halo columns) and step_kernel_ov (128 threads per
// CTA covering 128 - 2H interior columns plus their halo, so every warp
// collides and 8 CTAs of 4 warps fit an SM; the faster one on GB300).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lbsc_collide.cuh"
#include "lbsc_device.cuh"
#include "lbsc_internal.cuh"
#include "lbsc_strip.cuh"

namespace lbsc {

template <typename T, int ORDER, bool SAMPLE, bool UNIT = false>
__global__ void __launch_bounds__(kStepTX + 32) step_kernel(const KParams<T> p) {
    const int y0 = blockIdx.y * p.strip_h;
    step_strip<T, ORDER, SAMPLE, false, UNIT>(p, p.rk, blockIdx.x * kStepTX, y0,
                                              min(y0 + p.strip_h, p.ny));
}


// Overlapped layout: kStepTX threads per CTA, kStepTX - 2H interior columns,
// the halo pseudopotentials recomputed by the CTA's own edge threads.
template <typename T, int ORDER, bool SAMPLE, bool UNIT = false>
__global__ void __launch_bounds__(kStepTX) step_kernel_ov(const KParams<T> p) {
    const int y0 = blockIdx.y * p.strip_h;
    step_strip_ov<T, ORDER, SAMPLE, false, UNIT>(p, p.rk, blockIdx.x * ov_cols<ORDER>(), y0,
                                                 min(y0 + p.strip_h, p.ny));
}

template <typename T, int ORDER>
static cudaError_t launch_ov_t(const StepArgs &a, cudaStream_t s) {
    KParams<T> k = make_params<T>(a);
    constexpr int C = ov_cols<ORDER>();
    dim3 grid((a.nx + C - 1) / C, (a.ny + a.strip_h - 1) / a.strip_h);
    const bool unit =
        std::is_same<T, float>::value && a.gamma == 0.0 && a.gamma_b == 0.0 && a.gamma_g == 0.0;
    if (unit) {
        if (a.drho_out) step_kernel_ov<T, ORDER, true, true><<<grid, kStepTX, 0, s>>>(k);
        else step_kernel_ov<T, ORDER, false, true><<<grid, kStepTX, 0, s>>>(k);
    } else {
        if (a.drho_out) step_kernel_ov<T, ORDER, true><<<grid, kStepTX, 0, s>>>(k);
        else step_kernel_ov<T, ORDER, false><<<grid, kStepTX, 0, s>>>(k);
    }
    return cudaGetLastError();
}

template <typename T, int ORDER>
static cudaError_t launch_t(const StepArgs &a, cudaStream_t s) {
    if (a.layout == 1) return launch_ov_t<T, ORDER>(a, s);
    KParams<T> k = make_params<T>(a);
    dim3 grid((a.nx + kStepTX - 1) / kStepTX, (a.ny + a.strip_h - 1) / a.strip_h);
    // FP32 with every relaxation rate 1 (tau = 1 BGK, the usual setting) takes
    // the kernel that skips the unused moments
    if constexpr (std::is_same<T, float>::value) {
        if (a.gamma == 0.0 && a.gamma_b == 0.0 && a.gamma_g == 0.0) {
            if (a.drho_out)
                step_kernel<T, ORDER, true, true><<<grid, kStepTX + 32, 0, s>>>(k);
            else
                step_kernel<T, ORDER, false, true><<<grid, kStepTX + 32, 0, s>>>(k);
            return cudaGetLastError();
        }
    }
    if (a.drho_out) {
        step_kernel<T, ORDER, true><<<grid, kStepTX + 32, 0, s>>>(k);
    } else {
        step_kernel<T, ORDER, false><<<grid, kStepTX + 32, 0, s>>>(k);
    }
    return cudaGetLastError();
}

cudaError_t launch_step(int precision, int stencil, const StepArgs &a, cudaStream_t s) {
    if (precision == 0) {
        if (stencil == 4) return launch_t<float, 4>(a, s);
        if (stencil == 6) return launch_t<float, 6>(a, s);
        if (stencil == 8) return launch_t<float, 8>(a, s);
    } else {
        if (stencil == 4) return launch_t<double, 4>(a, s);
        if (stencil == 6) return launch_t<double, 6>(a, s);
        if (stencil == 8) return launch_t<double, 8>(a, s);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Initial state: delta f_i = w_i * amp * z(site), z from Philox block 2 of
// step 0 (amp = 0: the homogeneous state at rest).
// ---------------------------------------------------------------------------
struct InitKeys {
    uint32_t rk[20];
};

template <typename T>
__global__ void init_kernel(T *__restrict__ df, int nx, int ny, T amp, InitKeys keys,
                            uint32_t replica) {
    const size_t plane = (size_t)nx * ny;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < plane;
         s += (size_t)gridDim.x * blockDim.x) {
        T d = T(0);
        if (amp != T(0)) {
            uint4 r = philox4x32_10(make_uint4((uint32_t)s, 0u, replica, 2u), keys.rk);
            T z0, z1;
            box_muller(uniform01<T>(r.x), uniform01<T>(r.y), z0, z1);
            d = amp * z0;
        }
        df[0 * plane + s] = T(4.0 / 9.0) * d;
#pragma unroll
        for (int i = 1; i < 5; ++i) df[i * plane + s] = T(1.0 / 9.0) * d;
#pragma unroll
        for (int i = 5; i < 9; ++i) df[i * plane + s] = T(1.0 / 36.0) * d;
    }
}

cudaError_t launch_init(int precision, void *df, int nx, int ny, double amp,
                        const uint32_t round_keys[20], uint32_t replica, cudaStream_t s) {
    InitKeys k;
    for (int i = 0; i < 20; ++i) k.rk[i] = round_keys[i];
    const size_t plane = (size_t)nx * ny;
    int blocks = (int)((plane + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (precision == 0)
        init_kernel<float><<<blocks, 256, 0, s>>>((float *)df, nx, ny, (float)amp, k, replica);
    else
        init_kernel<double><<<blocks, 256, 0, s>>>((double *)df, nx, ny, amp, k, replica);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Density of the stored state: rho = rho0 + sum_i delta f_i (FP64 output),
// and the delta rho field in storage precision for an unscheduled S(k) sample.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void density_kernel(const T *__restrict__ df, double rho0, double *__restrict__ out,
                               size_t plane) {
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < plane;
         s += (size_t)gridDim.x * blockDim.x) {
        T g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = df[i * plane + s];
        out[s] = rho0 + (double)sum9(g);
    }
}

template <typename T>
__global__ void drho_kernel(const T *__restrict__ df, T *__restrict__ out, size_t plane) {
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < plane;
         s += (size_t)gridDim.x * blockDim.x) {
        T g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = df[i * plane + s];
        out[s] = sum9(g);
    }
}

cudaError_t launch_density(int precision, const void *df, double rho0, double *out, int nx,
                           int ny, cudaStream_t s) {
    const size_t plane = (size_t)nx * ny;
    int blocks = (int)((plane + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (precision == 0)
        density_kernel<float><<<blocks, 256, 0, s>>>((const float *)df, rho0, out, plane);
    else
        density_kernel<double><<<blocks, 256, 0, s>>>((const double *)df, rho0, out, plane);
    return cudaGetLastError();
}

cudaError_t launch_drho(int precision, const void *df, void *drho, int nx, int ny,
                        cudaStream_t s) {
    const size_t plane = (size_t)nx * ny;
    int blocks = (int)((plane + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (precision == 0)
        drho_kernel<float><<<blocks, 256, 0, s>>>((const float *)df, (float *)drho, plane);
    else
        drho_kernel<double><<<blocks, 256, 0, s>>>((const double *)df, (double *)drho, plane);
    return cudaGetLastError();
}

}  // namespace lbsc
