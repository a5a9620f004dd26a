// Test-only probe: evaluates the library's FP32 device math (expm1, the
// Box-Muller pair from two 32-bit words, and the ring Box-Muller of the step
// kernels from a radius word and an angle index) on host-given inputs.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbsc_device.cuh"

__global__ void expm1_probe(const float *x, float *y, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = lbsc::dev_expm1(x[i]);
}

__global__ void bm_probe(const uint32_t *r, float *z, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float a, b;
        lbsc::box_muller(lbsc::uniform01<float>(r[2 * i]), lbsc::uniform01<float>(r[2 * i + 1]), a, b);
        z[2 * i] = a;
        z[2 * i + 1] = b;
    }
}

// r[2i] = radius word, r[2i+1] = angle index; rho = 1: z = rad (c, s)
__global__ void ring_probe(const uint32_t *r, float *z, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float rad, c, s;
        lbsc::box_ring_polar(lbsc::uniform01<float>(r[2 * i]), r[2 * i + 1] & 1023u, 1.0f, rad, c, s);
        z[2 * i] = rad * c;
        z[2 * i + 1] = rad * s;
    }
}

template <typename T>
static int run(void (*k)(const T *, float *, int), const T *hin, size_t in_bytes, float *hout,
               size_t out_bytes, int n) {
    T *din = nullptr;
    float *dout = nullptr;
    if (cudaMalloc(&din, in_bytes) != cudaSuccess) return 1;
    if (cudaMalloc(&dout, out_bytes) != cudaSuccess) return 1;
    cudaMemcpy(din, hin, in_bytes, cudaMemcpyHostToDevice);
    k<<<(n + 255) / 256, 256>>>(din, dout, n);
    cudaError_t e = cudaMemcpy(hout, dout, out_bytes, cudaMemcpyDeviceToHost);
    cudaFree(din);
    cudaFree(dout);
    return e == cudaSuccess ? 0 : 2;
}

extern "C" int probe_expm1(const float *x, float *y, int n) {
    return run<float>(expm1_probe, x, n * sizeof(float), y, n * sizeof(float), n);
}

extern "C" int probe_box_muller(const uint32_t *r, float *z, int npairs) {
    return run<uint32_t>(bm_probe, r, 2 * npairs * sizeof(uint32_t), z, 2 * npairs * sizeof(float),
                         npairs);
}

extern "C" int probe_box_ring(const uint32_t *r, float *z, int npairs) {
    return run<uint32_t>(ring_probe, r, 2 * npairs * sizeof(uint32_t), z, 2 * npairs * sizeof(float),
                         npairs);
}
