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
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lbsc.h"

namespace lbsc {

int nn_conv_path = 0;   // 0: auto, 1: mma.sync, 2: tcgen05 per-tile kernel wherever it
                        // has one, 3: persistent tcgen05 kernel wherever it has one
__device__ int g_nn_status;               // bit 0: an mbarrier wait gave up;
                                          // bit 1: tensor memory left allocated
constexpr unsigned long long kTcWaitNs = 1000000000ull;   // default bound: 1 s
__device__ unsigned long long g_nn_wait_ns = kTcWaitNs;   // lb_nn_set_wait_ns
extern const int kWgTcMaxChunks = 192;   // bound on the SMs a weight-gradient launch plans for

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
// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout that TMA writes with CU_TENSOR_MAP_SWIZZLE_128B: rows of
// 64 BF16 (128 bytes) whose 16-byte chunks are permuted by the row's index
// within each 8-row, 1024-byte group (SBO = 1024), layout type 2 at bits
// 61-63.  The permutation follows the absolute shared-memory address (the
// groups start on 1024-byte boundaries), so an operand may start at any row
// of a group, or 32 bytes into a row for the next K step, with the base
// offset field left at 0 (checked against the CPU reference on GB300; the
// field set to the start row's index gave wrong results).
// (The same holds for rows of SP = 32 or 64 bytes, 16 or 32 BF16, with the
// matching 32- or 64-byte pattern: 8-row groups 8 SP bytes apart, layout type
// 6 or 4.)
// Its low word: start address / 16 (bits 0-13) and the LBO field (unused for
// swizzled K-major, 1); its high word: SBO = 8 rows (bits 32-45), version 1
// (bit 46), layout type (bits 61-63).
__device__ __forceinline__ uint32_t desc_sw_lo(uint32_t saddr) {
    return ((saddr & 0x3FFFFu) >> 4) | (1u << 16);
}
template <int SP> __host__ __device__ constexpr uint32_t desc_sw_hi() {
    static_assert(SP == 32 || SP == 64 || SP == 128, "swizzle span");
    return ((8u * SP) >> 4) | (1u << 14) | ((uint32_t)(SP == 128 ? 2 : SP == 64 ? 4 : 6) << 29);
}
template <int SP>
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t saddr) {
    return ((uint64_t)desc_sw_hi<SP>() << 32) | desc_sw_lo(saddr);
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
// The same with each descriptor given as its two 32-bit words (low words
// differing, high words shared).
__device__ __forceinline__ void tc_mma_lo(uint32_t dtmem, uint32_t alo, uint32_t ahi, uint32_t blo,
                                          uint32_t bhi, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n .reg .b64 ad, bd;\n setp.ne.b32 p, %6, 0;\n"
        " mov.b64 ad, {%1, %2};\n mov.b64 bd, {%3, %4};\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], ad, bd, %5, p;\n}\n" ::"r"(dtmem),
        "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(accumulate)
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

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
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

// ---------------------------------------------------------------------------
// Persistent, warp-specialised variant.  One CTA per SM (192 threads):
//   warp 4  producer: stages the nine taps' weights of the CTA's output-channel
//           block once, then input rows into a ring of R slots (cp.async,
//           completion tracked on mbarriers), as far ahead as free slots allow;
//   warp 5  MMA issuer (one thread): for each output row (128 pixels of one
//           image row) the 9 x CIN/16 tcgen05.mma of its three input rows
//           into one of two tensor-memory accumulators, then tcgen05.commit
//           to release the accumulator to the epilogue and the input rows
//           that no later row needs back to the producer;
//   warps 0-3 epilogue: tcgen05.ld of the accumulator (warp w owns lanes
//           32w .. 32w+31 = pixels), bias, ReLU, BF16 stores, then release
//           the accumulator.
// A CTA walks runs of consecutive output rows down a 128-pixel column band,
// so each input row is staged once per run.  DG: the input gradient of a
// forward layer (weights read transposed, taps mirrored), so the same kernel
// serves forward and backward.  Every wait is bounded; a timeout stops every
// role, and tensor memory is freed only after the committed MMAs finished.
// ---------------------------------------------------------------------------
template <int BN, int CIN>
struct PCfg {
    // Input channels are staged in blocks of BC = min(CIN, 64) channels, one
    // TMA box each, whose pixel rows of SP = 2 BC bytes carry the matching
    // 32-, 64- or 128-byte swizzle: a block of one input row holds pixels
    // x0-8 .. x0+135 as 144 rows; column c (pixel x0-1+c) is row c + 7.
    static constexpr int BC = CIN < 64 ? CIN : 64;
    static constexpr int SP = 2 * BC;                     // bytes per pixel row of a block
    static constexpr int KB = CIN / BC;                   // channel blocks
    static constexpr int KS = SP / 32;                    // K = 16 steps per block
    static constexpr uint32_t LBO_A = 144 * SP;           // block stride of a staged row
    static constexpr uint32_t COL0 = 7 * SP;
    static constexpr uint32_t PIX = SP;                   // bytes between pixels
    static constexpr int ROW_BYTES = KB * 144 * SP;
    static constexpr int TAP_BYTES = BN * CIN * 2;
    static constexpr int B_BYTES = 9 * TAP_BYTES;
    static constexpr int R0 = (220 * 1024 - B_BYTES) / ROW_BYTES;
    static constexpr int R = R0 < 4 ? 4 : (R0 > 8 ? 8 : R0);   // ring slots
    static constexpr int A_BYTES = R * ROW_BYTES;
    static constexpr int SMEM = A_BYTES + B_BYTES;
    // B per tap: channel block kb of output channel n at kb * BN * SP + n * SP
    // (16-byte chunks swizzled as TMA writes them)
    static constexpr uint32_t LBO_B = BN * SP;
    static constexpr uint32_t ROW_TX = (uint32_t)CIN * 144 * 2;   // bytes landing per row
    static constexpr int ALIGN = 1024;                            // staging alignment
    static constexpr uint32_t NCOLS = 2 * BN <= 32 ? 32 : (2 * BN <= 64 ? 64 : (2 * BN <= 128 ? 128 : 256));
};
constexpr int kTcpThreads = 192;

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, int c0, int c1,
                                          int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
// Bounded wait that also gives up when another role has aborted.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                             const volatile int *abort) {
    if (mbar_test_wait(bar, parity)) return true;
    if (limit_ns == 0) return false;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// tm_x: the input as [nb*H][W][CIN] with a box of 8 channels x 128 pixels
// (tm_xh: 8 channels x 8 pixels, the halo copies); tm_w: the weights as
// [9][Cout][CIN] with a box of 8 channels x BN output channels (forward only;
// the input gradient transposes the weights while staging them).
template <int BN, int CIN, bool DG>
__global__ void __launch_bounds__(kTcpThreads, 1)
conv3x3_tcp_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_xh,
                   const __grid_constant__ CUtensorMap tm_w, const bf16 *__restrict__ w,
                   const float *__restrict__ bias, bf16 *__restrict__ y, int nb, int H, int W,
                   int Cout, int relu, int ctas_per_block, int units_per_cta) {
    using C = PCfg<BN, CIN>;
    constexpr int R = C::R;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[R], slot_free[R], acc_full[2], acc_empty[2], wfull;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort, s_drained;
    __shared__ float s_bias[BN];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // aligned base for the bulk copies (128 bytes, 1024 for the swizzled
    // layout; the launch adds that much slack)
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + (C::ALIGN - 1)) &
        ~static_cast<uintptr_t>(C::ALIGN - 1));
    uint8_t *sA = smem;
    uint8_t *sB = smem + C::A_BYTES;
    constexpr uint32_t IDESC = idesc_bf16(128, BN);
    const int bands = W / 128;
    // this CTA's output-channel block and its share of that block's rows
    const int n0 = (blockIdx.x / ctas_per_block) * BN;
    const long units = (long)nb * H * bands;
    const long u_begin = (long)(blockIdx.x % ctas_per_block) * units_per_cta;
    const long u_end = min(units, u_begin + units_per_cta);
    const uint64_t limit = g_nn_wait_ns;
    volatile int *abort = &s_abort;

    if (warp == 0) tmem_alloc(&s_tmem, C::NCOLS);
    for (int i = tid; i < BN; i += kTcpThreads) s_bias[i] = bias ? bias[n0 + i] : 0.f;
    if (DG) {
        // w holds the forward layer's [9][CIN][Cout]; B[n][c] = w[8 - tap][c][n0 + n],
        // staged by every thread (16-byte loads of 8 n, scattered 2-byte stores)
        for (int v = tid; v < 9 * CIN * (BN / 8); v += kTcpThreads) {
            const int tap = v / (CIN * (BN / 8)), rem = v - tap * (CIN * (BN / 8));
            const int c = rem / (BN / 8), nc = rem - c * (BN / 8);
            const uint4 q = *reinterpret_cast<const uint4 *>(
                w + ((size_t)(8 - tap) * CIN + c) * Cout + n0 + nc * 8);
            const bf16 *e = reinterpret_cast<const bf16 *>(&q);
            // row n = nc * 8 + j of block c / BC; its 16-byte chunk ch = (c % BC) / 8
            // sits at chunk index ch ^ sw(n), the swizzle of an SP-byte row
            // (128: n % 8; 64: (n / 2) % 4; 32: (n / 4) % 2)
            uint8_t *d = sB + tap * C::TAP_BYTES + (c / C::BC) * C::LBO_B + nc * 8 * C::SP +
                         (c & 7) * 2;
            const int ch = (c % C::BC) >> 3;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n = nc * 8 + j;
                const int sw = C::SP == 128 ? (n & 7) : (C::SP == 64 ? ((n >> 1) & 3) : ((n >> 2) & 1));
                *reinterpret_cast<bf16 *>(d + j * C::SP + ((ch ^ sw) << 4)) = e[j];
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (tid == kTcpThreads - 1) {
        for (int i = 0; i < R; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&slot_free[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 4);
        }
        mbar_init(&wfull, 1);
        s_abort = 0;
        s_drained = 1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // unit u -> (image, band, row); rows vary fastest.  A run: consecutive
    // rows of one (image, band), at most to the end of the CTA's share.
    auto run_at = [&](long u, int &b, int &x0, int &row0, int &len) {
        row0 = (int)(u % H);
        const long r = u / H;
        x0 = (int)(r % bands) * 128;
        b = (int)(r / bands);
        len = (int)min(u_end - u, (long)(H - row0));
    };

    if (warp == 4) {
        // ---------------- producer (one thread issues the bulk copies) ----------------
        long seq = 0;
        if (lane == 0) {
            if (!DG) {
                mbar_expect_tx(&wfull, (uint32_t)C::B_BYTES);
                constexpr int NBLK = C::KB, BCH = C::BC;      // boxes per tap, channels per box
                for (int tap = 0; tap < 9; ++tap)
                    for (int kc = 0; kc < NBLK; ++kc)
                        tma_load3(sB + tap * C::TAP_BYTES + kc * C::LBO_B, &tm_w, kc * BCH, n0, tap,
                                  &wfull);
            }
            for (long u = u_begin; u < u_end && !*abort;) {
                int b, x0, row0, len;
                run_at(u, b, x0, row0, len);
                const int xl = x0 == 0 ? W - 8 : x0 - 8;          // left halo (periodic)
                const int xr = x0 + 128 == W ? 0 : x0 + 128;      // right halo
                bool stop = false;
                for (int j = 0; j < len + 2; ++j, ++seq) {
                    const int slot = (int)(seq % R);
                    if (seq >= R &&
                        !mbar_wait_ab(&slot_free[slot], (uint32_t)((seq / R - 1) & 1), limit, abort)) {
                        *abort = 1;
                        stop = true;
                        break;
                    }
                    int ys = row0 - 1 + j;
                    ys = ys < 0 ? ys + H : (ys >= H ? ys - H : ys);
                    const int yy = b * H + ys;
                    uint8_t *dst = sA + slot * C::ROW_BYTES;
                    mbar_expect_tx(&full[slot], C::ROW_TX);
                    constexpr int NBLK = C::KB, BCH = C::BC;      // channel blocks, channels per block
                    for (int kc = 0; kc < NBLK; ++kc) {
                        uint8_t *ch = dst + kc * C::LBO_A;
                        // x0-8 .. x0-1, x0 .. x0+127, x0+128 .. x0+135
                        tma_load3(ch, &tm_xh, kc * BCH, xl, yy, &full[slot]);
                        tma_load3(ch + 8 * C::PIX, &tm_x, kc * BCH, x0, yy, &full[slot]);
                        tma_load3(ch + 136 * C::PIX, &tm_xh, kc * BCH, xr, yy, &full[slot]);
                    }
                }
                if (stop) break;
                u += len;
            }
            // every copy must land before the CTA exits (the barriers and the
            // buffers live in its shared memory): wait, with the default
            // bound, for the weights and the last R rows issued
            if (!DG) mbar_wait(&wfull, 0, kTcWaitNs);
            for (long sq = seq > R ? seq - R : 0; sq < seq; ++sq)
                mbar_wait(&full[sq % R], (uint32_t)((sq / R) & 1), kTcWaitNs);
        }
        __syncwarp();
    } else if (warp == 5) {
        // ---------------- MMA issuer ----------------
        // One thread issues, and per MMA it adds one constant to each
        // operand's descriptor: the start-address field of a swizzled K-major
        // descriptor (bits 0-13, address / 16) cannot carry for shared
        // addresses below 2^18, so the descriptor of addr + off (off a
        // multiple of 16) is the one of addr with off / 16 added to its low
        // word, and the high word is the same for every operand.
        int t = 0, nfree = 0;   // output rows issued; input rows whose slot was released
        bool ok = true;
        if (lane == 0) {
            constexpr uint32_t DHI = desc_sw_hi<C::SP>();
            const uint32_t a_lo = desc_sw_lo(smem_u32(sA) + C::COL0);
            const uint32_t b_lo = desc_sw_lo(smem_u32(sB));
            if (!DG) ok = mbar_wait_ab(&wfull, 0, limit, abort);
            int seq0 = 0;
            for (long u = u_begin; u < u_end && ok;) {
                int b, x0, row0, len;
                run_at(u, b, x0, row0, len);
                for (int tt = 0; tt < len && ok; ++tt, ++t) {
                    // the three input rows of output row tt: sequence numbers
                    // seq0 + tt .. seq0 + tt + 2 (the first two were waited for
                    // with the previous row, except at the start of a run)
                    for (int q = tt == 0 ? 0 : 2; q < 3 && ok; ++q) {
                        const int sq = seq0 + tt + q;
                        ok = mbar_wait_ab(&full[sq % R], (uint32_t)((sq / R) & 1), limit, abort);
                    }
                    if (ok && t >= 2)
                        ok = mbar_wait_ab(&acc_empty[t & 1], (uint32_t)(((t - 2) >> 1) & 1), limit,
                                          abort);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t acc = tmem + (uint32_t)((t & 1) * BN);
                    const int s0 = (seq0 + tt) % R;
                    const int s1 = s0 + 1 == R ? 0 : s0 + 1;
                    const int s2 = s1 + 1 == R ? 0 : s1 + 1;
                    constexpr uint32_t kRow = (uint32_t)C::ROW_BYTES >> 4;
                    const uint32_t arow[3] = {a_lo + (uint32_t)s0 * kRow, a_lo + (uint32_t)s1 * kRow,
                                              a_lo + (uint32_t)s2 * kRow};
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                            for (int j = 0; j < CIN / 16; ++j) {
                                // K step j: block j / KS, 32 bytes per step within it
                                const uint32_t oa =
                                    (uint32_t)(dx * C::SP + (j / C::KS) * C::LBO_A + (j % C::KS) * 32) >> 4;
                                const uint32_t ob =
                                    (uint32_t)((3 * dy + dx) * C::TAP_BYTES + (j / C::KS) * C::LBO_B +
                                               (j % C::KS) * 32) >> 4;
                                tc_mma_lo(acc, arow[dy] + oa, DHI, b_lo + ob, DHI, IDESC,
                                          (dy > 0 || dx > 0 || j > 0) ? 1u : 0u);
                            }
                        }
                        if (dy == 0) {
                            // the row above is read by no later output row: hand
                            // its slot back as soon as these MMAs finish
                            tc_commit(&slot_free[s0]);
                            ++nfree;
                        }
                    }
                    tc_commit(&acc_full[t & 1]);
                    if (tt + 1 == len) {
                        // end of the run: its last two input rows are free too
                        tc_commit(&slot_free[s1]);
                        tc_commit(&slot_free[s2]);
                        nfree += 2;
                    }
                }
                seq0 += len + 2;
                u += len;
            }
            if (!ok) {
                *abort = 1;
                atomicOr(&g_nn_status, 1);
            }
            // drain: every MMA committed must finish before the accumulator
            // is freed, and every commit's arrival must land before the CTA
            // exits: wait (default bound) for the last phase of each barrier
            // this thread committed to.  The slot releases went to input rows
            // 0 .. nfree - 1 in order, so slot i took (nfree - 1 - i) / R + 1.
            bool drained = true;
            for (int g = t > 2 ? t - 2 : 0; g < t; ++g)
                drained = mbar_wait(&acc_full[g & 1], (uint32_t)((g >> 1) & 1), kTcWaitNs) && drained;
            for (int i = 0; i < R && i < nfree; ++i) {
                const int n = (nfree - 1 - i) / R + 1;
                drained = mbar_wait(&slot_free[i], (uint32_t)((n - 1) & 1), kTcWaitNs) && drained;
            }
            if (!drained) {
                s_drained = 0;
                atomicOr(&g_nn_status, 2);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 0-3) ----------------
        long t = 0;
        for (long u = u_begin; u < u_end && !*abort;) {
            int b, x0, row0, len;
            run_at(u, b, x0, row0, len);
            for (int tt = 0; tt < len; ++tt, ++t) {
                if (!mbar_wait_ab(&acc_full[t & 1], (uint32_t)((t >> 1) & 1), limit, abort)) {
                    *abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t lane_base =
                    tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((t & 1) * BN);
                bf16 *yout = y + (((size_t)b * H + row0 + tt) * W + x0 + warp * 32 + lane) * Cout + n0;
                constexpr int CH = BN < 32 ? BN : 32;   // columns per tensor-memory load
#pragma unroll
                for (int col = 0; col < BN; col += CH) {
                    uint32_t rr[CH];
                    if constexpr (CH == 32) tmem_ld32(lane_base + col, rr);
                    else tmem_ld16(lane_base + col, rr);
                    uint32_t packed[CH / 2];
#pragma unroll
                    for (int q = 0; q < CH / 2; ++q) {
                        float v0 = __uint_as_float(rr[2 * q]) + s_bias[col + 2 * q];
                        float v1 = __uint_as_float(rr[2 * q + 1]) + s_bias[col + 2 * q + 1];
                        if (relu) {
                            v0 = fmaxf(v0, 0.f);
                            v1 = fmaxf(v1, 0.f);
                        }
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
                        packed[q] = *reinterpret_cast<uint32_t *>(&h2);
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(yout + col);
#pragma unroll
                    for (int q = 0; q < CH / 8; ++q)
                        dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2],
                                            packed[4 * q + 3]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[t & 1]);
            }
            if (*abort) break;
            u += len;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && s_drained) tmem_dealloc(tmem, C::NCOLS);
}

// Resident CTAs of kTcpThreads threads per SM: registers are allocated per
// warp in units of 256, and the warps of B resident CTAs are spread over the
// SM's four schedulers, each holding a quarter of the register file, so B
// fits while ceil(B warps / 4) warps' registers fit a quarter; every CTA also
// takes its shared memory plus 1 KB reserved by the system.  (This reproduces
// the limits the profiler reports for this kernel and for the ensemble's
// persistent kernel.)
int tcp_slots_per_sm(int regs, int smem_cta, int smem_sm, int regs_sm, int tmem_slots) {
    const int warps = kTcpThreads / 32;
    const int warp_regs = (regs * 32 + 255) / 256 * 256;
    int by_regs = 0;
    while ((((by_regs + 1) * warps + 3) / 4) * warp_regs <= regs_sm / 4) ++by_regs;
    const int by_smem = smem_sm / (smem_cta + 1024);
    return std::max(1, std::min(tmem_slots, std::min(by_regs, by_smem)));
}

// Tensor maps of the persistent convolution (cuTensorMapEncodeTiled through
// the runtime's driver entry point).
PFN_cuTensorMapEncodeTiled_v12000 tcp_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

// A BF16 tensor [d2][d1][d0] (d0 innermost) with a box of b0 x b1 x 1, copied
// with the swizzle pattern of `span`-byte rows (32, 64 or 128: the box's b0
// channels make one row).
bool tcp_map_span(CUtensorMap *m, const void *base, uint64_t d0, uint64_t d1, uint64_t d2,
                  uint32_t b0, uint32_t b1, int span) {
    auto fn = tcp_encode_fn();
    if (!fn || b0 * 2 != (uint32_t)span) return false;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {d0 * 2, d0 * d1 * 2};
    const cuuint32_t box[3] = {b0, b1, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapSwizzle sw = span == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : span == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                               : CU_TENSOR_MAP_SWIZZLE_32B;
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int CIN, bool DG>
cudaError_t launch_tcp(const bf16 *x, const bf16 *w, const float *bias, bf16 *y, int nb, int h,
                       int wd, int cout, int relu, cudaStream_t s) {
    using C = PCfg<BN, CIN>;
    static_assert(C::SMEM + C::ALIGN <= 226 * 1024, "shared-memory plan too large");
    // at most 512 / NCOLS CTAs may share an SM's 512 tensor-memory columns:
    // the shared-memory request is padded so that no more fit
    constexpr int kPerSm = 512 / (int)C::NCOLS;
    constexpr int kMinSmem = 233472 / (kPerSm + 1) + 1;   // 228 KB of shared memory per SM
    constexpr int kSmem = C::SMEM + C::ALIGN > kMinSmem ? C::SMEM + C::ALIGN : kMinSmem;
    // TMA: 16-byte aligned base addresses
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(w)) & 15)
        return cudaErrorNotSupported;
    CUtensorMap mx, mxh, mw;
    if (!tcp_map_span(&mx, x, CIN, wd, (uint64_t)nb * h, C::BC, 128, C::SP) ||
        !tcp_map_span(&mxh, x, CIN, wd, (uint64_t)nb * h, C::BC, 8, C::SP))
        return cudaErrorNotSupported;
    if (!DG) {
        if (!tcp_map_span(&mw, w, CIN, cout, 9, C::BC, BN, C::SP)) return cudaErrorNotSupported;
    } else {
        mw = mx;   // unused by the input gradient
    }
    // CTAs resident per SM: a narrow layer's output rows are short chains of
    // copies, MMAs and a read-out whose latency one CTA per SM cannot hide, so
    // the grid fills every resident slot.  The slots are counted here from the
    // kernel's registers and shared memory (and the tensor-memory padding
    // above) because the runtime's occupancy query answered one CTA per SM for
    // plans of which two were measured resident together on GB300 (47 and
    // 110 KB of shared memory, about 100 registers).
    static int nsm = 0, per_sm = 1;
    if (!nsm) {
        int dev = 0, smem_sm = 0, regs_sm = 0;
        cudaFuncAttributes fa;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv3x3_tcp_kernel<BN, CIN, DG>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, conv3x3_tcp_kernel<BN, CIN, DG>);
        if (e != cudaSuccess) {
            nsm = 0;
            return e;
        }
        per_sm = tcp_slots_per_sm(fa.numRegs, (int)fa.sharedSizeBytes + kSmem, smem_sm, regs_sm,
                                  kPerSm);
    }
    const int nblk = cout / BN;
    const long units = (long)nb * h * (wd / 128);
    int per_blk = std::max(1, nsm * per_sm / nblk);
    if (per_blk > units) per_blk = (int)units;
    const int per = (int)((units + per_blk - 1) / per_blk);
    conv3x3_tcp_kernel<BN, CIN, DG><<<nblk * per_blk, kTcpThreads, kSmem, s>>>(
        mx, mxh, mw, w, bias, y, nb, h, wd, cout, relu, per_blk, per);
    return cudaGetLastError();
}

// Channel block per CTA: all of cout where the weights and the ring fit,
// else 32 (128 input channels).
template <bool DG>
cudaError_t launch_tcp_shape(const bf16 *x, const bf16 *w, const float *bias, bf16 *y, int nb,
                             int h, int wd, int cin, int cout, int relu, cudaStream_t s) {
#define TCP(BN, CIN) return launch_tcp<BN, CIN, DG>(x, w, bias, y, nb, h, wd, cout, relu, s)
    if (cin == 16) {
        if (cout == 16) TCP(16, 16);
        if (cout == 32) TCP(32, 16);
        if (cout == 64) TCP(64, 16);
        if (cout == 128) TCP(128, 16);
    } else if (cin == 32) {
        if (cout == 16) TCP(16, 32);
        if (cout == 32) TCP(32, 32);
        if (cout == 64) TCP(64, 32);
        if (cout == 128) TCP(128, 32);
    } else if (cin == 64) {
        if (cout == 16) TCP(16, 64);
        if (cout == 32) TCP(32, 64);
        if (cout == 64) TCP(64, 64);
        if (cout == 128) TCP(128, 64);
    } else if (cin == 128) {
        if (cout == 16) TCP(16, 128);
        if (cout % 32 == 0) TCP(32, 128);
    }
#undef TCP
    return cudaErrorNotSupported;
}


// ---------------------------------------------------------------------------
// Weight gradient on tcgen05: dw[tap][n][c] += sum_p x[p + off(tap)][c] dy[p][n]
// as GEMMs over 128-pixel tiles of one image row (K = the tile's pixels).
// Both operands are staged straight from the NHWC tensors by TMA, one pixel
// per row with its channels contiguous (the forward kernel's row layout), so
// they are MN-major operands; a tap's pixel shift is a row shift of the x
// operand's descriptor.  M = 128 rows of the operand with more channels (AC
// real ones; the rows beyond them read other staged data or slack and land in
// accumulator rows that are discarded), N = the other's NC channels.  A CTA
// holds TP accumulators (all nine taps when 9 NC tensor-memory columns fit,
// else the three of one tap row), sums a chunk of tiles into them, and writes
// them once to its slice of the caller's workspace; a separate kernel adds the
// chunks in a fixed order.  Warp 4 issues the copies into a ring of S slots,
// one thread of warp 5 the MMAs, warps 0-3 read the accumulators at the end.
// Every wait is bounded, as in the forward kernel.
// ---------------------------------------------------------------------------
// CTAs per SM for a weight gradient with cin input and cout output channels
// and tp taps per CTA: two when their accumulators (at most 256
// tensor-memory columns each) and a ring of at least two slots plus the
// padding slack fit twice (a narrow layer's tiles are short chains of copies
// and MMAs whose latency a second CTA hides), else one.
__host__ __device__ constexpr int wg_ctas(int tp, int cin, int cout) {
    const bool ax = cin > cout;
    const int ac = ax ? cin : cout, nc = ax ? cout : cin;
    const int xr = tp == 9 ? 3 : 1;
    const int slot = xr * ((144 * cin * 2 + 1023) / 1024 * 1024) + (128 * cout * 2 + 1023) / 1024 * 1024;
    const int slack = (128 - ac) * (ax ? 144 : 128) * 2;
    return tp * nc <= 256 && (110 * 1024 - slack) / slot >= 2 ? 2 : 1;
}
// Taps per CTA: all nine (their accumulators take 9 nc tensor-memory
// columns, and three staged x rows must fit) unless one tap row per CTA gives
// two CTAs per SM where nine do not.
__host__ __device__ constexpr int wg_taps(int cin, int cout) {
    const int nc = cin < cout ? cin : cout;
    const bool nine = 9 * nc <= 512 && 3 * 144 * cin * 2 <= 80 * 1024;
    return nine && wg_ctas(9, cin, cout) == 2 ? 9 : (wg_ctas(3, cin, cout) == 2 ? 3 : (nine ? 9 : 3));
}
__host__ __device__ constexpr int wg_per_sm(int cin, int cout) {
    return wg_ctas(wg_taps(cin, cout), cin, cout);
}

template <int AC, int NC, bool AX>
struct WCfg {
    static constexpr int TP = wg_taps(AX ? AC : NC, AX ? NC : AC);   // taps per CTA
    static constexpr int PER_SM = wg_per_sm(AX ? AC : NC, AX ? NC : AC);
    static constexpr int TG = 9 / TP;                   // tap groups
    static constexpr int XR = TP == 9 ? 3 : 1;          // x rows staged per tile
    static constexpr int XC = AX ? AC : NC;             // channels of x
    static constexpr int DC = AX ? NC : AC;             // channels of dy
    // channels per staged block (a TMA box; rows of XSP / DSP bytes, swizzled
    // with the matching 32-, 64- or 128-byte pattern)
    static constexpr int XBC = XC < 64 ? XC : 64, DBC = DC < 64 ? DC : 64;
    static constexpr int XSP = 2 * XBC, DSP = 2 * DBC;
    static constexpr int XROW = 144, DROW = 128;        // pixel rows: x0-8 .. x0+135, x0 .. x0+127
    static constexpr int X_BYTES = XROW * XC * 2;       // one staged x row (what lands)
    static constexpr int D_BYTES = DROW * DC * 2;
    static constexpr int X_STRIDE = (X_BYTES + 1023) / 1024 * 1024;
    static constexpr int D_STRIDE = (D_BYTES + 1023) / 1024 * 1024;
    static constexpr int A_BYTES = AX ? XR * X_STRIDE : D_STRIDE;   // per slot
    static constexpr int B_BYTES = AX ? D_STRIDE : XR * X_STRIDE;
    // what the MMAs read of the A operand past its AC channels (M = 128)
    static constexpr int SLACK = (128 - AC) * (AX ? XROW : DROW) * 2;
    static constexpr int S0 = ((PER_SM == 2 ? 110 : 200) * 1024 - SLACK) / (A_BYTES + B_BYTES);
    static constexpr int S = S0 > 4 ? 4 : S0;           // ring slots
    static constexpr int SMEM = S * (A_BYTES + B_BYTES) + SLACK;
    static constexpr uint32_t NCOLS = TP * NC <= 32 ? 32 : TP * NC <= 64 ? 64
                                    : TP * NC <= 128 ? 128 : TP * NC <= 256 ? 256 : 512;
    static constexpr uint32_t TX = XR * X_BYTES + D_BYTES;   // bytes landing per slot
    static_assert(S >= 2, "shared-memory plan too small");
};
constexpr int kWgtThreads = 192;

// Descriptor of an MN-major operand staged as pixel rows of SP bytes (SP / 2
// channels: 16, 32 or 64), swizzled with the SP-byte pattern that TMA writes:
// blocks of SP / 2 channels `rows` rows apart (LBO), 8-row groups 8 SP bytes
// apart (SBO), layout type 6 / 4 / 2 for 32 / 64 / 128 bytes; starting at
// pixel row `row`.  As for the K-major operands, the swizzle follows the
// absolute shared-memory address, so any start row works with the base
// offset field at 0.  The high word is desc_sw_hi<SP>(); the low word at row
// 0 is mn_desc_lo, and starting `row` rows further adds row SP / 16 to it
// (the start-address field cannot carry for shared addresses below 2^18).
template <int SP>
__device__ __forceinline__ uint32_t mn_desc_lo(uint32_t base, int rows) {
    static_assert(SP == 32 || SP == 64 || SP == 128, "swizzle span");
    return ((base & 0x3FFFFu) >> 4) | ((((uint32_t)(rows * SP) >> 4) & 0x3FFFu) << 16);
}

// tm_x / tm_xh: x as [nb*H][W][Cin], boxes of XB channels x 128 / 8 pixels;
// tm_dy: dy as [nb*H][W][Cout], box DB channels x 128 pixels.  part: this
// launch's partial sums [chunk][9][Cout][Cin].
template <int AC, int NC, bool AX>
__global__ void __launch_bounds__(kWgtThreads, 1)
wgrad_tc_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_xh,
                const __grid_constant__ CUtensorMap tm_dy, float *__restrict__ part, int nb, int H,
                int W, int Cin, int Cout, int tiles_per_chunk) {
    using C = WCfg<AC, NC, AX>;
    constexpr int S = C::S, TP = C::TP;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[S], slot_free[S], done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort, s_drained;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t *sB = smem;                          // S slots of the B operand
    uint8_t *sA = smem + S * C::B_BYTES;         // S slots of the A operand, then the slack
    auto xreg = [&](int slot, int q) {
        return (AX ? sA + slot * C::A_BYTES : sB + slot * C::B_BYTES) + q * C::X_STRIDE;
    };
    auto dreg = [&](int slot) { return AX ? sB + slot * C::B_BYTES : sA + slot * C::A_BYTES; };
    // both operands MN-major (bits 15 and 16)
    constexpr uint32_t IDESC = idesc_bf16(128, NC) | (1u << 15) | (1u << 16);
    const int tg = blockIdx.x % C::TG, chunk = blockIdx.x / C::TG;
    const int bands = W / 128;
    const long ntiles = (long)nb * bands * H;
    const long t_begin = (long)chunk * tiles_per_chunk;
    const long t_end = min(ntiles, t_begin + tiles_per_chunk);
    const int n = (int)(t_end - t_begin);   // >= 1 by the launch plan
    const uint64_t limit = g_nn_wait_ns;
    volatile int *abort = &s_abort;
    // tile t -> image b, band x0, row y (rows fastest: consecutive tiles share x rows)
    auto tile_at = [&](long t, int &b, int &x0, int &y) {
        y = (int)(t % H);
        const long r = t / H;
        x0 = (int)(r % bands) * 128;
        b = (int)(r / bands);
    };

    if (warp == 0) tmem_alloc(&s_tmem, C::NCOLS);
    if (tid == kWgtThreads - 1) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&slot_free[i], 1);
        }
        mbar_init(&done, 1);
        s_abort = 0;
        s_drained = 1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 4) {
        // ---------------- producer ----------------
        if (lane == 0) {
            constexpr int XB = C::XBC, DB = C::DBC;     // channels per box
            constexpr int XP = C::XSP, DP = C::DSP;     // bytes per pixel row
            int t = 0;
            for (; t < n && !*abort; ++t) {
                const int slot = t % S;
                if (t >= S &&
                    !mbar_wait_ab(&slot_free[slot], (uint32_t)((t / S - 1) & 1), limit, abort)) {
                    *abort = 1;
                    break;
                }
                int b, x0, y;
                tile_at(t_begin + t, b, x0, y);
                const int xl = x0 == 0 ? W - 8 : x0 - 8;        // left halo (periodic)
                const int xr = x0 + 128 == W ? 0 : x0 + 128;    // right halo
                mbar_expect_tx(&full[slot], C::TX);
                for (int q = 0; q < C::XR; ++q) {
                    const int ys = wrapi(y + (TP == 9 ? q : tg) - 1, H);
                    uint8_t *dst = xreg(slot, q);
                    for (int kc = 0; kc < C::XC / XB; ++kc) {
                        uint8_t *ch = dst + kc * C::XROW * XP;
                        tma_load3(ch, &tm_xh, kc * XB, xl, b * H + ys, &full[slot]);
                        tma_load3(ch + 8 * XP, &tm_x, kc * XB, x0, b * H + ys, &full[slot]);
                        tma_load3(ch + 136 * XP, &tm_xh, kc * XB, xr, b * H + ys, &full[slot]);
                    }
                }
                for (int kc = 0; kc < C::DC / DB; ++kc)
                    tma_load3(dreg(slot) + kc * C::DROW * DP, &tm_dy, kc * DB, x0, b * H + y,
                              &full[slot]);
            }
            // every copy issued must land before the CTA exits
            for (int sq = t > S ? t - S : 0; sq < t; ++sq)
                mbar_wait(&full[sq % S], (uint32_t)((sq / S) & 1), kTcWaitNs);
        }
        __syncwarp();
    } else if (warp == 5) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            // descriptor low words built once per tile, a constant added per MMA
            constexpr uint32_t DHI = desc_sw_hi<C::DSP>(), XHI = desc_sw_hi<C::XSP>();
            constexpr int NQ = TP == 9 ? 3 : 1;
            int ncommit = 0;   // tiles whose slot release was committed (in order)
            bool ok = true;
            for (int t = 0; t < n && ok; ++t) {
                const int slot = t % S;
                ok = mbar_wait_ab(&full[slot], (uint32_t)((t / S) & 1), limit, abort);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d_lo = mn_desc_lo<C::DSP>(smem_u32(dreg(slot)), C::DROW);
                uint32_t x_lo[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) x_lo[q] = mn_desc_lo<C::XSP>(smem_u32(xreg(slot, q)), C::XROW);
                // K steps outer, taps inner: consecutive MMAs go to different
                // accumulators, so none waits for the one before it
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t dd = d_lo + (uint32_t)((16 * j * C::DSP) >> 4);
#pragma unroll
                    for (int tl = 0; tl < TP; ++tl) {
                        // pixels 16j .. 16j+15 of the tile; x shifted by the tap
                        // (staged row 8 is pixel x0, so the tap's row 7 + dx + p)
                        const int q = TP == 9 ? tl / 3 : 0, dx = tl % 3;
                        const uint32_t xd = x_lo[q] + (uint32_t)(((7 + dx + 16 * j) * C::XSP) >> 4);
                        if constexpr (AX)
                            tc_mma_lo(tmem + (uint32_t)(tl * NC), xd, XHI, dd, DHI, IDESC,
                                      (t > 0 || j > 0) ? 1u : 0u);
                        else
                            tc_mma_lo(tmem + (uint32_t)(tl * NC), dd, DHI, xd, XHI, IDESC,
                                      (t > 0 || j > 0) ? 1u : 0u);
                    }
                }
                tc_commit(&slot_free[slot]);
                ++ncommit;
            }
            if (!ok) {
                *abort = 1;
                atomicOr(&g_nn_status, 1);
            }
            // done: every MMA issued has finished (also after an abort, so that
            // tensor memory is freed only then); wait for it and for the last
            // arrival on each slot barrier before the CTA may exit
            // (slot i took (ncommit - 1 - i) / S + 1 of the slot releases)
            tc_commit(&done);
            bool drained = mbar_wait(&done, 0, kTcWaitNs);
            for (int i = 0; i < S && i < ncommit; ++i) {
                const int k = (ncommit - 1 - i) / S + 1;
                drained = mbar_wait(&slot_free[i], (uint32_t)((k - 1) & 1), kTcWaitNs) && drained;
            }
            if (!drained) {
                s_drained = 0;
                atomicOr(&g_nn_status, 2);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 0-3): lanes 32w .. 32w+31 = rows m ----------------
        if (!mbar_wait_ab(&done, 0, limit, abort)) *abort = 1;
        if (!*abort) {
            tc_fence_after();
            const int m = warp * 32 + lane;
            const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
            constexpr int CH = NC < 32 ? NC : 32;   // columns per tensor-memory load
#pragma unroll 1
            for (int tl = 0; tl < TP; ++tl) {
                const int tap = TP == 9 ? tl : tg * 3 + tl;
                float *dst = part + ((size_t)chunk * 9 + tap) * Cout * Cin;
#pragma unroll
                for (int col = 0; col < NC; col += CH) {
                    uint32_t rr[CH];
                    if constexpr (CH == 32) tmem_ld32(lane_base + (uint32_t)(tl * NC + col), rr);
                    else tmem_ld16(lane_base + (uint32_t)(tl * NC + col), rr);
                    if (n <= 0)   // no tile (the launch plan avoids it): a zero partial sum
                        for (int k = 0; k < CH; ++k) rr[k] = 0u;
                    if (m < AC) {
                        if constexpr (!AX) {
                            // row m = output channel, column = input channel
                            float4 *o = reinterpret_cast<float4 *>(dst + (size_t)m * Cin + col);
#pragma unroll
                            for (int k = 0; k < CH / 4; ++k)
                                o[k] = make_float4(__uint_as_float(rr[4 * k]), __uint_as_float(rr[4 * k + 1]),
                                                   __uint_as_float(rr[4 * k + 2]),
                                                   __uint_as_float(rr[4 * k + 3]));
                        } else {
                            // row m = input channel, column = output channel
#pragma unroll
                            for (int k = 0; k < CH; ++k)
                                dst[(size_t)(col + k) * Cin + m] = __uint_as_float(rr[k]);
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && s_drained) tmem_dealloc(tmem, C::NCOLS);
}

template <int AC, int NC, bool AX>
cudaError_t launch_wgrad_t(const bf16 *x, const bf16 *dy, float *part, int nb, int h, int wd,
                           int cin, int cout, int nchunk, cudaStream_t s) {
    using C = WCfg<AC, NC, AX>;
    // at most 512 / NCOLS CTAs may share an SM's tensor memory: pad the
    // shared-memory request so that no more fit
    constexpr int kPerSm = 512 / (int)C::NCOLS;
    constexpr int kMinSmem = 233472 / (kPerSm + 1) + 1;
    constexpr int kSmem = C::SMEM + 1024 > kMinSmem ? C::SMEM + 1024 : kMinSmem;
    static_assert(C::SMEM + 1024 <= 226 * 1024, "shared-memory plan too large");
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(dy)) & 15)
        return cudaErrorNotSupported;
    CUtensorMap mx, mxh, mdy;
    if (!tcp_map_span(&mx, x, cin, wd, (uint64_t)nb * h, C::XBC, 128, C::XSP) ||
        !tcp_map_span(&mxh, x, cin, wd, (uint64_t)nb * h, C::XBC, 8, C::XSP) ||
        !tcp_map_span(&mdy, dy, cout, wd, (uint64_t)nb * h, C::DBC, 128, C::DSP))
        return cudaErrorNotSupported;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel<AC, NC, AX>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long ntiles = (long)nb * h * (wd / 128);
    const int per = (int)((ntiles + nchunk - 1) / nchunk);
    wgrad_tc_kernel<AC, NC, AX><<<C::TG * nchunk, kWgtThreads, kSmem, s>>>(
        mx, mxh, mdy, part, nb, h, wd, cin, cout, per);
    return cudaGetLastError();
}

// NC <= AC channels of the N operand (NC < AC when the A operand is x).
template <int AC, bool AX>
cudaError_t launch_wgrad_nc(int nc, const bf16 *x, const bf16 *dy, float *part, int nb, int h,
                            int wd, int cin, int cout, int nchunk, cudaStream_t s) {
    if constexpr (AC > 16 || !AX)
        if (nc == 16) return launch_wgrad_t<AC, 16, AX>(x, dy, part, nb, h, wd, cin, cout, nchunk, s);
    if constexpr (AC > 32 || (AC == 32 && !AX))
        if (nc == 32) return launch_wgrad_t<AC, 32, AX>(x, dy, part, nb, h, wd, cin, cout, nchunk, s);
    if constexpr (AC > 64 || (AC == 64 && !AX))
        if (nc == 64) return launch_wgrad_t<AC, 64, AX>(x, dy, part, nb, h, wd, cin, cout, nchunk, s);
    if constexpr (AC == 128 && !AX)
        if (nc == 128) return launch_wgrad_t<AC, 128, AX>(x, dy, part, nb, h, wd, cin, cout, nchunk, s);
    return cudaErrorNotSupported;
}

template <bool AX>
cudaError_t launch_wgrad_ac(int ac, int nc, const bf16 *x, const bf16 *dy, float *part, int nb,
                            int h, int wd, int cin, int cout, int nchunk, cudaStream_t s) {
    switch (ac) {
    case 16: return launch_wgrad_nc<16, AX>(nc, x, dy, part, nb, h, wd, cin, cout, nchunk, s);
    case 32: return launch_wgrad_nc<32, AX>(nc, x, dy, part, nb, h, wd, cin, cout, nchunk, s);
    case 64: return launch_wgrad_nc<64, AX>(nc, x, dy, part, nb, h, wd, cin, cout, nchunk, s);
    case 128: return launch_wgrad_nc<128, AX>(nc, x, dy, part, nb, h, wd, cin, cout, nchunk, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace

// Persistent tcgen05 convolution (forward, or the input gradient with dgrad)
// for rows a multiple of 128 pixels and 16/32/64/128 channels;
// cudaErrorNotSupported otherwise so that the caller takes the mma.sync kernel.
cudaError_t launch_conv3x3_tcp(const void *x, const void *w, const float *bias, void *y, int nb,
                               int h, int wd, int cin, int cout, int relu, int dgrad,
                               cudaStream_t s) {
    if (wd % 128 || h < 2) return cudaErrorNotSupported;
    const bf16 *xb = (const bf16 *)x, *wb = (const bf16 *)w;
    bf16 *yb = (bf16 *)y;
    return dgrad ? launch_tcp_shape<true>(xb, wb, bias, yb, nb, h, wd, cin, cout, relu, s)
                 : launch_tcp_shape<false>(xb, wb, bias, yb, nb, h, wd, cin, cout, relu, s);
}

// Weight gradient on tcgen05 (see wgrad_tc_kernel): the chunk count for a
// launch (CTAs = tap groups x chunks, one or two per SM), or 0 where the kernel does
// not apply (image rows not a multiple of 128 pixels, channel counts other
// than 16, 32, 64, 128).
int wgrad_tc_chunks(int nb, int h, int wd, int cin, int cout, int nsm) {
    auto ok = [](int c) { return c == 16 || c == 32 || c == 64 || c == 128; };
    if (wd % 128 || h < 2 || !ok(cin) || !ok(cout) || nsm < 1) return 0;
    const int tg = 9 / wg_taps(cin, cout), per_sm = wg_per_sm(cin, cout);
    const long ntiles = (long)nb * h * (wd / 128);
    long k = (long)nsm * per_sm / tg;
    if (k > (long)kWgTcMaxChunks * per_sm / tg) k = (long)kWgTcMaxChunks * per_sm / tg;
    if (k > ntiles) k = ntiles;
    if (k < 1) k = 1;
    // chunks of ceil(ntiles / k) tiles: keep only those that get a tile
    const long per = (ntiles + k - 1) / k;
    return (int)((ntiles + per - 1) / per);
}

// Partial sums [nchunk][9][cout][cin] of the weight gradient into part.
cudaError_t launch_wgrad_tc(const void *x, const void *dy, float *part, int nb, int h, int wd,
                            int cin, int cout, int nchunk, cudaStream_t s) {
    const bf16 *xb = (const bf16 *)x, *db = (const bf16 *)dy;
    // M = 128 rows of the operand with more channels (dy on a tie)
    if (cout >= cin)
        return launch_wgrad_ac<false>(cout, cin, xb, db, part, nb, h, wd, cin, cout, nchunk, s);
    return launch_wgrad_ac<true>(cin, cout, xb, db, part, nb, h, wd, cin, cout, nchunk, s);
}

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
    if (path < 0 || path > 3) return LB_ERR_ARG;
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
