// Test-only probe: the first outputs of cuRAND's device Philox4_32_10
// generator, used to pin the oracle's Philox4x32-10 against a library.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void philox_probe(unsigned long long seed, unsigned long long subseq, uint4 *out) {
    curandStatePhilox4_32_10_t s;
    curand_init(seed, subseq, 0, &s);
    out[0] = curand4(&s);
    out[1] = curand4(&s);
}

extern "C" int curand_philox_first(unsigned long long seed, unsigned long long subseq,
                                   unsigned int *host8) {
    uint4 *d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(uint4)) != cudaSuccess) return 1;
    philox_probe<<<1, 1>>>(seed, subseq, d);
    cudaError_t e = cudaMemcpy(host8, d, 2 * sizeof(uint4), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : 2;
}
