// Forward 3x3 convolution of the learned surrogate on the fifth-generation
// tensor cores: tcgen05.mma (BF16 operands from shared memory, FP32
// accumulator in tensor memory), one elected thread issuing, completion
// tracked on mbarriers.
//
// Implicit GEMM per CTA: M = 128 consecutive output pixels of one image row
// (TMEM lane m = pixel m), N = BN output channels (TMEM columns), K = 9 taps x
// Cin.  The CTA stages the three input rows it needs (130 columns, periodic
// wrap, 16-byte cp.async copies) once in shared memory, with consecutive
// pixels 16 bytes apart: each tap's A operand is then the same staged rows
// seen through a descriptor whose start address is shifted by the tap's
// pixel offset, so the input is read about 3x per output tile instead of 9x.
// The weights of all nine taps are staged beside it.  The MMAs of tap row r
// are issued as soon as input row r and its weights have landed (three
// cp.async groups); one commit on an mbarrier (bounded wait) releases the
// epilogue.
// The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31), adds the bias, applies ReLU and stores BF16.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbsc.h"

namespace lbsc {

int nn_conv_path = 0;   // 0: auto, 1: mma.sync, 2: tcgen05 wherever it has a kernel
__device__ int g_nn_status;               // bit 0: an mbarrier wait gave up;
                                          // bit 1: tensor memory left allocated
constexpr unsigned long long kTcWaitNs = 1000000000ull;   // default bound: 1 s
__device__ unsigned long long g_nn_wait_ns = kTcWaitNs;   // lb_nn_set_wait_ns

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the completion of the phase with the given parity; false if it has
// not completed within limit_ns (0: give up at the first unfinished check,
// which does not block).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_test_wait(bar, parity)) return true;
    if (limit_ns == 0) return false;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem)
                 : "memory");
}

// Shared-memory matrix descriptor (K-major, no swizzle): start address,
// leading (K) and stride (8-row group) byte offsets, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t r[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory plan of one CTA: the three input rows y-1, y, y+1 over the
// 130 columns x0-1 .. x0+128 (A, staged once), and the weights of all nine
// taps for BN output channels (B).  A is laid out so that consecutive pixels
// are 16 bytes apart (8-row groups SBO = 128 B) and 8-channel K chunks
// LBO = 130 x 16 B apart: shifting a tap by one pixel is then a 16-byte shift
// of the descriptor's start address, and the nine taps read the same staged
// rows.  B is canonical K-major per tap: 8-row groups SBO = Cin/8 x 128 B,
// K chunks 128 B apart.
template <int BN, int CIN>
struct RowCfg {
    static constexpr int KC = CIN / 8;                    // 16-byte chunks per pixel
    static constexpr uint32_t LBO_A = 130 * 16;           // between K chunks of a row
    static constexpr int ROW_BYTES = KC * LBO_A;          // one staged input row
    static constexpr int A_BYTES = 3 * ROW_BYTES;
    static constexpr int TAP_BYTES = BN * CIN * 2;
    static constexpr int B_BYTES = 9 * TAP_BYTES;
    static constexpr int SMEM = A_BYTES + B_BYTES;
    static constexpr uint32_t SBO_B = KC * 128;
    static constexpr uint32_t NCOLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
};

template <int BN, int CIN>
__global__ void __launch_bounds__(128)
conv3x3_tc_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ w,
                  const float *__restrict__ bias, bf16 *__restrict__ y, int H, int W, int Cout,
                  int relu) {
    using C = RowCfg<BN, CIN>;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_per_row = W / 128;
    const int yrow = blockIdx.x / tiles_per_row;
    const int x0 = (blockIdx.x - yrow * tiles_per_row) * 128;
    const size_t img = (size_t)blockIdx.y * H * W;
    const int n0 = blockIdx.z * BN;
    constexpr uint32_t IDESC = idesc_bf16(128, BN);
    uint8_t *sA = smem;
    uint8_t *sB = smem + C::A_BYTES;

    // three cp.async groups: input row y-1+r and the weights of taps 3r .. 3r+2
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int ys = wrapi(yrow + r - 1, H);
        const bf16 *src = x + (img + (size_t)ys * W) * CIN;
        uint8_t *dst = sA + r * C::ROW_BYTES;
        for (int v = tid; v < 130 * C::KC; v += 128) {
            const int col = v / C::KC, kc = v - col * C::KC;
            int xs = x0 - 1 + col;
            xs = xs < 0 ? xs + W : (xs >= W ? xs - W : xs);
            cp_async16(dst + kc * C::LBO_A + col * 16, src + (size_t)xs * CIN + kc * 8);
        }
        for (int v = tid; v < 3 * BN * C::KC; v += 128) {
            const int tl = v / (BN * C::KC), rem = v - tl * (BN * C::KC);
            const int n = rem / C::KC, kc = rem - n * C::KC;
            const int tap = 3 * r + tl;
            cp_async16(sB + tap * C::TAP_BYTES + (n >> 3) * C::SBO_B + kc * 128 + (n & 7) * 16,
                       w + ((size_t)tap * Cout + n0 + n) * CIN + kc * 8);
        }
        cp_async_commit();
    }
    if (warp == 0) tmem_alloc(&s_tmem, C::NCOLS);
    if (tid == 32) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // the MMAs of tap row r start once its input row and weights have landed
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        if (r == 0) cp_async_wait_group<2>();
        else if (r == 1) cp_async_wait_group<1>();
        else cp_async_wait_group<0>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t arow = smem_u32(sA + r * C::ROW_BYTES);
#pragma unroll
            for (int tx = 0; tx < 3; ++tx) {   // dx = tx - 1: staged column tx is pixel x0 + dx
                const uint32_t btap = smem_u32(sB + (3 * r + tx) * C::TAP_BYTES);
#pragma unroll
                for (int j = 0; j < CIN / 16; ++j)
                    tc_mma(tmem, smem_desc(arow + tx * 16 + 2 * j * C::LBO_A, C::LBO_A, 128),
                           smem_desc(btap + j * 256, 128, C::SBO_B), IDESC,
                           (r > 0 || tx > 0 || j > 0) ? 1u : 0u);
            }
            if (r == 2) tc_commit(&bar);
        }
    }
    const bool done = mbar_wait(&bar, 0, g_nn_wait_ns);
    const bool ok = !__syncthreads_or(!done);
    __shared__ int s_drained;
    if (ok) {
        tc_fence_after();
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        bf16 *yout = y + (img + (size_t)yrow * W + x0 + warp * 32 + lane) * Cout + n0;
#pragma unroll
        for (int col = 0; col < BN; col += 16) {
            uint32_t rr[16];
            tmem_ld16(lane_base + col, rr);
            uint32_t packed[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float v0 = __uint_as_float(rr[2 * q]), v1 = __uint_as_float(rr[2 * q + 1]);
                if (bias) {
                    v0 += bias[n0 + col + 2 * q];
                    v1 += bias[n0 + col + 2 * q + 1];
                }
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                packed[q] = *reinterpret_cast<uint32_t *>(&h);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(yout + col);
            dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
    } else if (tid == 0) {
        atomicOr(&g_nn_status, 1);
        // the committed MMAs must finish before their accumulator is freed:
        // wait for them again with the default bound
        s_drained = mbar_wait(&bar, 0, kTcWaitNs) ? 1 : 0;
        if (!s_drained) atomicOr(&g_nn_status, 2);
    }
    tc_fence_before();
    __syncthreads();
    // never free tensor memory under MMAs that may still be in flight
    if (warp == 0 && (ok || s_drained)) tmem_dealloc(tmem, C::NCOLS);
}

template <int BN, int CIN>
cudaError_t launch_tc(const bf16 *x, const bf16 *w, const float *bias, bf16 *y, int nb, int h,
                      int wd, int cout, int relu, cudaStream_t s) {
    using C = RowCfg<BN, CIN>;
    static_assert(C::SMEM <= 220 * 1024, "shared-memory plan too large");
    static bool attr_set = false;   // per instantiation; set before the first launch
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel<BN, CIN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((unsigned)((size_t)h * (wd / 128)), nb, cout / BN);
    conv3x3_tc_kernel<BN, CIN><<<grid, 128, C::SMEM, s>>>(x, w, bias, y, h, wd, cout, relu);
    return cudaGetLastError();
}

}  // namespace

// Forward convolution on tcgen05 when the path selection and the shape allow
// (rows a multiple of 128 pixels, 16/32/64/128 channels);
// cudaErrorNotSupported otherwise so that the caller takes the mma.sync kernel.
cudaError_t launch_conv3x3_tc(const void *x, const void *w, const float *bias, void *y, int nb,
                              int h, int wd, int cin, int cout, int relu, cudaStream_t s) {
    if (wd % 128) return cudaErrorNotSupported;   // a tile is 128 pixels of one row
    // auto: tcgen05 where it measured faster than mma.sync on GB300 (32 and 64
    // input channels); 16 channels are gather-latency-bound and 128 channels
    // limit the CTA to one per SM, where the mma.sync kernel is as fast or faster
    if (nn_conv_path == 0 && (cin == 16 || cin == 128)) return cudaErrorNotSupported;
    const bf16 *xb = (const bf16 *)x, *wb = (const bf16 *)w;
    bf16 *yb = (bf16 *)y;
#define TC(BN, CIN) return launch_tc<BN, CIN>(xb, wb, bias, yb, nb, h, wd, cout, relu, s)
    // output-channel block per CTA: all of cout where A and the nine taps of B fit
    if (cin == 16) {
        if (cout == 16) TC(16, 16);
        if (cout == 32) TC(32, 16);
        if (cout == 64) TC(64, 16);
        if (cout == 128) TC(128, 16);
    } else if (cin == 32) {
        if (cout == 16) TC(16, 32);
        if (cout == 32) TC(32, 32);
        if (cout == 64) TC(64, 32);
        if (cout == 128) TC(128, 32);
    } else if (cin == 64) {
        if (cout == 16) TC(16, 64);
        if (cout == 32) TC(32, 64);
        if (cout == 64) TC(64, 64);
        if (cout == 128) TC(128, 64);
    } else if (cin == 128) {
        if (cout % 32 == 0) TC(32, 128);
        if (cout == 16) TC(16, 128);
    }
#undef TC
    return cudaErrorNotSupported;
}

}  // namespace lbsc

extern "C" int lb_nn_set_conv_path(int path) {
    if (path < 0 || path > 2) return LB_ERR_ARG;
    lbsc::nn_conv_path = path;
    return LB_OK;
}

extern "C" int lb_nn_status(void) {
    int v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return LB_ERR_CUDA;
    if (cudaMemcpyFromSymbol(&v, lbsc::g_nn_status, sizeof(int)) != cudaSuccess) return LB_ERR_CUDA;
    if (v) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(lbsc::g_nn_status, &zero, sizeof(int)) != cudaSuccess)
            return LB_ERR_CUDA;
        return (v & 2) ? LB_ERR_CUDA : LB_ERR_TIMEOUT;
    }
    return LB_OK;
}

extern "C" int lb_nn_set_wait_ns(long long ns) {
    const unsigned long long v = ns < 0 ? lbsc::kTcWaitNs : (unsigned long long)ns;
    if (cudaDeviceSynchronize() != cudaSuccess) return LB_ERR_CUDA;
    if (cudaMemcpyToSymbol(lbsc::g_nn_wait_ns, &v, sizeof(v)) != cudaSuccess) return LB_ERR_CUDA;
    return LB_OK;
}
