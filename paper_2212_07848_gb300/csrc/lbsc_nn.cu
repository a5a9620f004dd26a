// Learned surrogate building blocks: BF16 tensor-core 3x3 convolutions on
// periodic NHWC fields (forward, input gradient, weight gradient) with FP32
// accumulation, and the elementwise pieces of a small convolutional
// operator (pooling, upsampling, skip sums, ReLU mask, coarse-graining of the
// lattice density, MSE loss, Adam).  The surrogate advances the coarse
// density of a quench by a fixed stride; the plain lattice Boltzmann step
// stays the reference it is scored against.
//
// The forward convolution runs on tcgen05 (lbsc_nn_tc.cu) for its output
// channel counts; the mma.sync kernels here serve the input gradient, the
// weight gradient and the forward path when it is selected for comparison.
// They are implicit GEMMs on mma.sync m16n8k16 (BF16 in, FP32 accumulate):
// M = output pixels (128 consecutive pixels per CTA), N = output channels,
// K = 9 taps x input channels; the im2col tile is gathered with circular
// (periodic) padding straight from NHWC into shared memory.
// The input gradient is the same kernel run on dY with the taps mirrored and
// the weight matrix transposed; the weight gradient is a GEMM over pixels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lbsc.h"

namespace lbsc {

// tcgen05 forward convolution (lbsc_nn_tc.cu) and the path selection.
extern int nn_conv_path;
cudaError_t launch_conv3x3_tcp(const void *x, const void *w, const float *bias, void *y, int nb,
                               int h, int wd, int cin, int cout, int relu, int dgrad,
                               cudaStream_t s);
extern const int kWgTcMaxChunks;
int wgrad_tc_chunks(int nb, int h, int wd, int cin, int cout, int nsm);
cudaError_t launch_wgrad_tc(const void *x, const void *dy, float *part, int nb, int h, int wd,
                            int cin, int cout, int nchunk, cudaStream_t s);
cudaError_t launch_conv3x3_tc(const void *x, const void *w, const float *bias, void *y, int nb,
                              int h, int wd, int cin, int cout, int relu, cudaStream_t s);

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void mma_bf16_16816(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// ---------------------------------------------------------------------------
// Forward / input-gradient convolution.
//   forward: y[p][n] = act( bias[n] + sum_{tap, c} x[p + off(tap)][c] w[tap][n][c] )
//   dgrad  : dx[p][c] = sum_{tap, n} dy[p + off(tap)][n] w[8 - tap][n][c]
// CTA: 128 consecutive pixels of one image (row-major, may span rows) x BN
// channels; 4 warps, each 32 pixels x BN.
// ---------------------------------------------------------------------------
template <int BN, int BK, bool DGRAD>
__global__ void __launch_bounds__(128)
conv3x3_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ w, const float *__restrict__ bias,
               bf16 *__restrict__ y, int H, int W, int Cin, int Cout, int relu) {
    // GEMM view: K = 9 * Kc (Kc = channels of x), N = Nc (channels of y)
    constexpr int P = BK + 8;                      // smem row pitch (elements)
    __shared__ __align__(16) bf16 As[128 * P];
    __shared__ __align__(16) bf16 Bs[BN * P];
    const int Kc = Cin, Nc = Cout;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int pix0 = blockIdx.x * 128;            // first pixel of the tile in its image
    const int b = blockIdx.y;
    const int n0 = blockIdx.z * BN;
    const size_t img = (size_t)b * H * W;

    float acc[2][BN / 8][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < BN / 8; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        for (int c0 = 0; c0 < Kc; c0 += BK) {
            // A: 128 pixels x BK channels, 16-byte vectors (8 bf16)
            constexpr int AV = 128 * BK / 8;
            for (int v = tid; v < AV; v += 128) {
                const int px = v / (BK / 8), cv = v % (BK / 8);
                const int pix = pix0 + px;
                const int ys = wrapi(pix / W + dy, H), xs = wrapi(pix % W + dx, W);
                const uint4 val = *reinterpret_cast<const uint4 *>(
                    x + (img + (size_t)ys * W + xs) * Kc + c0 + cv * 8);
                *reinterpret_cast<uint4 *>(&As[px * P + cv * 8]) = val;
            }
            // B: BN output channels x BK input channels
            if (!DGRAD) {
                constexpr int BV = BN * BK / 8;
                for (int v = tid; v < BV; v += 128) {
                    const int nn = v / (BK / 8), cv = v % (BK / 8);
                    const uint4 val = *reinterpret_cast<const uint4 *>(
                        w + ((size_t)tap * Nc + n0 + nn) * Kc + c0 + cv * 8);
                    *reinterpret_cast<uint4 *>(&Bs[nn * P + cv * 8]) = val;
                }
            } else {
                // w is [9][Kc][Nc] of the forward layer (Kc = its Cout, Nc = its Cin):
                // B[nn][kk] = w[8 - tap][kk][nn]
                for (int e = tid; e < BN * BK; e += 128) {
                    const int kk = e / BN, nn = e % BN;
                    Bs[nn * P + kk] = w[((size_t)(8 - tap) * Kc + c0 + kk) * Nc + n0 + nn];
                }
            }
            __syncthreads();
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                uint32_t af[2][4];
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) {
                    const int r = warp * 32 + mi * 16 + g;
                    const int k = ks * 16 + 2 * t;
                    af[mi][0] = *reinterpret_cast<const uint32_t *>(&As[r * P + k]);
                    af[mi][1] = *reinterpret_cast<const uint32_t *>(&As[(r + 8) * P + k]);
                    af[mi][2] = *reinterpret_cast<const uint32_t *>(&As[r * P + k + 8]);
                    af[mi][3] = *reinterpret_cast<const uint32_t *>(&As[(r + 8) * P + k + 8]);
                }
#pragma unroll
                for (int ni = 0; ni < BN / 8; ++ni) {
                    const int nn = ni * 8 + g;
                    const int k = ks * 16 + 2 * t;
                    uint32_t bfr[2];
                    bfr[0] = *reinterpret_cast<const uint32_t *>(&Bs[nn * P + k]);
                    bfr[1] = *reinterpret_cast<const uint32_t *>(&Bs[nn * P + k + 8]);
#pragma unroll
                    for (int mi = 0; mi < 2; ++mi) mma_bf16_16816(acc[mi][ni], af[mi], bfr);
                }
            }
            __syncthreads();
        }
    }
    // epilogue: bias, ReLU, BF16 store (channel pairs)
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < BN / 8; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int px = warp * 32 + mi * 16 + g + h * 8;
                const int n = n0 + ni * 8 + 2 * t;
                float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
                if (bias) {
                    v0 += bias[n];
                    v1 += bias[n + 1];
                }
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                *reinterpret_cast<__nv_bfloat162 *>(y + (img + pix0 + px) * Nc + n) =
                    __floats2bfloat162_rn(v0, v1);
            }
}

// ---------------------------------------------------------------------------
// Weight gradient: dw[tap][n][c] += sum_p x[p + off(tap)][c] dy[p][n].
// GEMM per tap with M = n, N = c and K = pixels, split over chunks of
// 128-pixel tiles: each CTA writes its chunk's partial sums of all nine taps
// to a workspace with plain stores, and a second kernel adds the chunks into
// dw in a fixed order (no atomics, so the result is deterministic).
// A CTA covers BM output channels x BC input channels with one warp per
// 16 x 16 block.  Per tile it stages dY [128][BM] and, one tap row (dy) at a
// time, the three shifted input tiles x[p + off][BC] in shared memory with
// 16-byte cp.async copies; both operands are K-major there (pixels are rows),
// so the fragments come from ldmatrix with the .trans qualifier.
// ---------------------------------------------------------------------------
constexpr int kWgTile = 128;            // pixels per tile (one GEMM K block)
constexpr int kWgTargetCtas = 152 * 8;  // CTAs a launch aims for

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t r[4], const void *smem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(sa));
}

template <int BM, int BC>
__global__ void __launch_bounds__(32 * (BM / 16) * (BC / 16))
wgrad_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ dy, float *__restrict__ part,
             int H, int W, int Cin, int Cout, int ntiles, int tiles_per_chunk) {
    constexpr int NT = 32 * (BM / 16) * (BC / 16);
    constexpr int PD = BM + 8, PX = BC + 8;        // row pitches (16-byte padded)
    __shared__ __align__(16) bf16 sDy[kWgTile * PD];
    __shared__ __align__(16) bf16 sX[3][kWgTile * PX];
    __shared__ int sYX[kWgTile][2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int nw = (warp % (BM / 16)) * 16, cw = (warp / (BM / 16)) * 16;
    const int n0 = blockIdx.x * BM, c0 = blockIdx.y * BC;
    const int chunk = blockIdx.z;
    const int tile_begin = chunk * tiles_per_chunk;
    const int tile_end = min(tile_begin + tiles_per_chunk, ntiles);
    const int tiles_per_img = H * W / kWgTile;

    float acc[9][2][4];
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    // ldmatrix row addresses: lane -> (pixel offset, channel offset) of its 8x8 matrix
    const int mat = lane >> 3, r8 = lane & 7;
    const int a_pix = r8 + ((mat & 2) ? 8 : 0), a_col = nw + ((mat & 1) ? 8 : 0);
    const int b_pix = r8 + ((mat & 1) ? 8 : 0), b_col = cw + ((mat & 2) ? 8 : 0);

    for (int tile = tile_begin; tile < tile_end; ++tile) {
        const int b = tile / tiles_per_img;
        const int pix0 = (tile - b * tiles_per_img) * kWgTile;
        const size_t img = (size_t)b * H * W;
        for (int px = tid; px < kWgTile; px += NT) {
            sYX[px][0] = (pix0 + px) / W;
            sYX[px][1] = (pix0 + px) % W;
        }
        constexpr int DV = kWgTile * BM / 8;
        for (int v = tid; v < DV; v += NT) {
            const int px = v / (BM / 8), cv = v % (BM / 8);
            cp_async16(&sDy[px * PD + cv * 8], dy + (img + pix0 + px) * Cout + n0 + cv * 8);
        }
        __syncthreads();   // sYX visible
        for (int ty = 0; ty < 3; ++ty) {
            const int ddy = ty - 1;
            constexpr int XV = kWgTile * BC / 8;
#pragma unroll
            for (int tx = 0; tx < 3; ++tx) {
                const int ddx = tx - 1;
                for (int v = tid; v < XV; v += NT) {
                    const int px = v / (BC / 8), cv = v % (BC / 8);
                    const int ys = wrapi(sYX[px][0] + ddy, H), xs = wrapi(sYX[px][1] + ddx, W);
                    cp_async16(&sX[tx][px * PX + cv * 8],
                               x + (img + (size_t)ys * W + xs) * Cin + c0 + cv * 8);
                }
            }
            cp_async_wait_all();
            __syncthreads();
#pragma unroll 2
            for (int k0 = 0; k0 < kWgTile; k0 += 16) {
                uint32_t af[4];
                ldsm_x4_trans(af, &sDy[(k0 + a_pix) * PD + a_col]);
#pragma unroll
                for (int tx = 0; tx < 3; ++tx) {
                    uint32_t bf[4];
                    ldsm_x4_trans(bf, &sX[tx][(k0 + b_pix) * PX + b_col]);
                    mma_bf16_16816(acc[ty * 3 + tx][0], af, &bf[0]);
                    mma_bf16_16816(acc[ty * 3 + tx][1], af, &bf[2]);
                }
            }
            __syncthreads();   // before the next tap row (or tile) overwrites sX / sDy
        }
    }
    // partial sums of this chunk: part[chunk][tap][n][c]
#pragma unroll
    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int n = n0 + nw + g + h * 8;
                const int c = c0 + cw + ni * 8 + 2 * t;
                float2 v = make_float2(acc[tap][ni][2 * h], acc[tap][ni][2 * h + 1]);
                *reinterpret_cast<float2 *>(
                    part + (((size_t)chunk * 9 + tap) * Cout + n) * Cin + c) = v;
            }
}

// dw[i] += sum over chunks of part[chunk][i], chunks added in order.
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, float *__restrict__ dw, size_t n,
                                    int nchunk) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int ch = 0; ch < nchunk; ++ch) s += part[(size_t)ch * n + i];
        dw[i] += s;
    }
}

// Chunking of a weight-gradient launch (shared by the workspace query).
struct WgPlan {
    int bm, bc, ntiles, tiles_per_chunk, nchunk;
};
WgPlan wgrad_plan(int nb, int h, int w, int cin, int cout) {
    WgPlan p;
    p.bm = cout % 32 == 0 ? 32 : 16;
    p.bc = cin % 32 == 0 ? 32 : 16;
    p.ntiles = (int)((size_t)nb * h * w / kWgTile);
    const int blocks = (cout / p.bm) * (cin / p.bc);
    int want = (kWgTargetCtas + blocks - 1) / blocks;
    if (want > p.ntiles) want = p.ntiles;
    if (want < 1) want = 1;
    p.tiles_per_chunk = (p.ntiles + want - 1) / want;
    p.nchunk = (p.ntiles + p.tiles_per_chunk - 1) / p.tiles_per_chunk;
    return p;
}

// Chunks of partial sums a workspace must hold: the mma.sync plan's or the
// tcgen05 kernel's largest.
int wgrad_max_chunks(int nb, int h, int w, int cin, int cout) {
    const int a = wgrad_plan(nb, h, w, cin, cout).nchunk;
    const int b = wgrad_tc_chunks(nb, h, w, cin, cout, kWgTcMaxChunks);
    return a > b ? a : b;
}

// ---------------------------------------------------------------------------
// Elementwise pieces (NHWC BF16 activations, FP32 parameters and losses).
// ---------------------------------------------------------------------------
#define GRID_STRIDE(i, n) \
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

// Bias gradient db[c] += sum_p dy[p][c] in a fixed order: block (b, g) sums
// channel group g over its grid-stride share of pixels (each warp a strided
// subset, then the warps in order) into part[b][c]; bias_reduce_kernel adds
// the kBiasBlocks partials of each channel in order.
constexpr int kBiasBlocks = 1216;   // eight 256-thread blocks per SM
__global__ void __launch_bounds__(256) bias_grad_kernel(const bf16 *__restrict__ dy,
                                                        float *__restrict__ part, size_t P, int C) {
    // thread t: channel group g = t % G (8 channels, one 16-byte load), pixel
    // slot t / G of the block's PB pixels per sweep; fixed order throughout
    const int G = C / 8, PB = 256 / G;
    const int g = threadIdx.x % G, slot = threadIdx.x / G;
    float s[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] = 0.f;
    if (slot < PB) {
#pragma unroll 4
        for (size_t p = (size_t)blockIdx.x * PB + slot; p < P; p += (size_t)gridDim.x * PB) {
            const uint4 q = *reinterpret_cast<const uint4 *>(dy + p * C + g * 8);
            const __nv_bfloat162 *e = reinterpret_cast<const __nv_bfloat162 *>(&q);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = __bfloat1622float2(e[k]);
                s[2 * k] += f.x;
                s[2 * k + 1] += f.y;
            }
        }
    }
    __shared__ float red[256][9];   // padded: conflict-free column reads
#pragma unroll
    for (int k = 0; k < 8; ++k) red[threadIdx.x][k] = s[k];
    __syncthreads();
    // channel c = 8 g' + k: the PB slots of group g', in slot order
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const int gg = c / 8, k = c % 8;
        float a = 0.f;
        for (int sl = 0; sl < PB; ++sl) a += red[sl * G + gg][k];
        part[(size_t)blockIdx.x * C + c] = a;
    }
}
// db[c] += the partials of channel c (block c): thread t adds partials t,
// t + 256, ... in order, then a fixed tree over the threads.
__global__ void __launch_bounds__(256) bias_reduce_kernel(const float *__restrict__ part,
                                                          float *__restrict__ db, int C,
                                                          int nblocks) {
    const int c = blockIdx.x;
    float a = 0.f;
    for (int b = threadIdx.x; b < nblocks; b += 256) a += part[(size_t)b * C + c];
    __shared__ float red[256];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] += red[0];
}

__global__ void relu_mask_kernel(const bf16 *__restrict__ dy, const bf16 *__restrict__ y,
                                 bf16 *__restrict__ dz, size_t n) {
    GRID_STRIDE(i, n) dz[i] = __bfloat162float(y[i]) > 0.f ? dy[i] : __float2bfloat16(0.f);
}

__global__ void pool2_fwd_kernel(const bf16 *__restrict__ x, bf16 *__restrict__ y, int NB, int H,
                                 int W, int C) {
    const int h = H / 2, w = W / 2;
    GRID_STRIDE(i, (size_t)NB * h * w * C) {
        const int c = (int)(i % C);
        size_t r = i / C;
        const int X = (int)(r % w), Y = (int)((r / w) % h), b = (int)(r / ((size_t)w * h));
        const size_t base = (((size_t)b * H + 2 * Y) * W + 2 * X) * C + c;
        const float s = __bfloat162float(x[base]) + __bfloat162float(x[base + C]) +
                        __bfloat162float(x[base + (size_t)W * C]) +
                        __bfloat162float(x[base + (size_t)W * C + C]);
        y[i] = __float2bfloat16(0.25f * s);
    }
}

__global__ void pool2_bwd_kernel(const bf16 *__restrict__ dy, bf16 *__restrict__ dx, int NB, int H,
                                 int W, int C) {
    GRID_STRIDE(i, (size_t)NB * H * W * C) {
        const int c = (int)(i % C);
        size_t r = i / C;
        const int x = (int)(r % W), yy = (int)((r / W) % H), b = (int)(r / ((size_t)W * H));
        dx[i] = __float2bfloat16(
            0.25f * __bfloat162float(dy[(((size_t)b * (H / 2) + yy / 2) * (W / 2) + x / 2) * C + c]));
    }
}

__global__ void up2_fwd_kernel(const bf16 *__restrict__ x, bf16 *__restrict__ y, int NB, int H,
                               int W, int C) {
    // x: [NB][H][W][C] -> y: [NB][2H][2W][C]
    GRID_STRIDE(i, (size_t)NB * 4 * H * W * C) {
        const int c = (int)(i % C);
        size_t r = i / C;
        const int X = (int)(r % (2 * W)), Y = (int)((r / (2 * W)) % (2 * H)),
                  b = (int)(r / ((size_t)4 * W * H));
        y[i] = x[(((size_t)b * H + Y / 2) * W + X / 2) * C + c];
    }
}

__global__ void up2_bwd_kernel(const bf16 *__restrict__ dy, bf16 *__restrict__ dx, int NB, int H,
                               int W, int C) {
    // dy: [NB][2H][2W][C] -> dx: [NB][H][W][C]
    GRID_STRIDE(i, (size_t)NB * H * W * C) {
        const int c = (int)(i % C);
        size_t r = i / C;
        const int x = (int)(r % W), yy = (int)((r / W) % H), b = (int)(r / ((size_t)W * H));
        const size_t base = (((size_t)b * 2 * H + 2 * yy) * 2 * W + 2 * x) * C + c;
        const size_t row = (size_t)2 * W * C;
        dx[i] = __float2bfloat16(__bfloat162float(dy[base]) + __bfloat162float(dy[base + C]) +
                                 __bfloat162float(dy[base + row]) +
                                 __bfloat162float(dy[base + row + C]));
    }
}

__global__ void add_kernel(const bf16 *__restrict__ a, const bf16 *__restrict__ b,
                           bf16 *__restrict__ y, size_t n) {
    GRID_STRIDE(i, n) y[i] = __float2bfloat16(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

// Coarse-grain the density of a lattice state (FP32 deviations [9][ny][nx])
// by f x f block averages: out [ny/f][nx/f] = (block mean of rho - rho0) / scale.
__global__ void coarse_kernel(const float *__restrict__ df, int nx, int ny, int f, float scale,
                              float *__restrict__ out) {
    const int cx = nx / f, cy = ny / f;
    const size_t plane = (size_t)nx * ny;
    GRID_STRIDE(i, (size_t)cx * cy) {
        const int X = (int)(i % cx), Y = (int)(i / cx);
        float s = 0.f;
        for (int yy = 0; yy < f; ++yy)
            for (int xx = 0; xx < f; ++xx) {
                const size_t site = (size_t)(Y * f + yy) * nx + X * f + xx;
                float d = 0.f;
#pragma unroll
                for (int k = 0; k < 9; ++k) d += df[k * plane + site];
                s += d;
            }
        out[i] = s / (f * f) / scale;
    }
}

// dst[.][dch] += src[.][sch] (BF16 channels of two [n][C] buffers).
__global__ void add_channel_kernel(bf16 *__restrict__ dst, int dc, int dch,
                                   const bf16 *__restrict__ src, int sc, int sch, size_t n) {
    GRID_STRIDE(i, n) dst[i * dc + dch] = __float2bfloat16(__bfloat162float(dst[i * dc + dch]) +
                                                            __bfloat162float(src[i * sc + sch]));
}

// Block MSE: the residual d = base + y[.][0] - target averaged over each
// B x B block of each image [nb][h][w]; loss += weight * mean over blocks of
// (block mean)^2 and dy[.][0] += its gradient, 2 weight mean_b / (nblocks B^2),
// on every pixel of block b.  One CTA per block (blocks are disjoint, so the
// read-modify-write of dy needs no atomics).
__global__ void __launch_bounds__(256) mse_block_kernel(const bf16 *__restrict__ y, int C,
                                                        const float *__restrict__ tgt,
                                                        const float *__restrict__ base, int H,
                                                        int W, int B, float weight,
                                                        float inv_nblocks, float *__restrict__ loss,
                                                        bf16 *__restrict__ dy) {
    const int bw = W / B, bh = H / B;
    const int blk = blockIdx.x;
    const int img = blk / (bw * bh), r = blk % (bw * bh);
    const int by = r / bw, bx = r % bw;
    const size_t img0 = (size_t)img * H * W;
    const int npx = B * B;
    float s = 0.f;
    for (int t = threadIdx.x; t < npx; t += blockDim.x) {
        const size_t p = img0 + (size_t)(by * B + t / B) * W + bx * B + t % B;
        s += base[p] + __bfloat162float(y[p * C]) - tgt[p];
    }
    __shared__ float red[8];
    __shared__ float mean_s;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
        const float m = a / (float)npx;
        mean_s = m;
        atomicAdd(loss, weight * m * m * inv_nblocks);
    }
    __syncthreads();
    if (!dy) return;
    const float g = 2.f * weight * mean_s * inv_nblocks / (float)npx;
    for (int t = threadIdx.x; t < npx; t += blockDim.x) {
        const size_t p = img0 + (size_t)(by * B + t / B) * W + bx * B + t % B;
        dy[p * C] = __float2bfloat16(__bfloat162float(dy[p * C]) + g);
    }
}

// Coarse-grained momentum j = sum_i c_i df_i (D2Q9 order 0:(0,0) 1:(1,0)
// 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)); the w_i rho0
// part of the populations carries no momentum.
__global__ void coarse_mom_kernel(const float *__restrict__ df, int nx, int ny, int f, float scale,
                                  float *__restrict__ jx_out, float *__restrict__ jy_out) {
    const int cx = nx / f, cy = ny / f;
    const size_t plane = (size_t)nx * ny;
    GRID_STRIDE(i, (size_t)cx * cy) {
        const int X = (int)(i % cx), Y = (int)(i / cx);
        float sx = 0.f, sy = 0.f;
        for (int yy = 0; yy < f; ++yy)
            for (int xx = 0; xx < f; ++xx) {
                const size_t site = (size_t)(Y * f + yy) * nx + X * f + xx;
                const float f1 = df[plane + site], f2 = df[2 * plane + site];
                const float f3 = df[3 * plane + site], f4 = df[4 * plane + site];
                const float f5 = df[5 * plane + site], f6 = df[6 * plane + site];
                const float f7 = df[7 * plane + site], f8 = df[8 * plane + site];
                sx += (f1 - f3) + (f5 - f7) + (f8 - f6);
                sy += (f2 - f4) + (f5 - f7) + (f6 - f8);
            }
        jx_out[i] = sx / (f * f) / scale;
        jy_out[i] = sy / (f * f) / scale;
    }
}

// One more channel of a network input: out[.][ch] = BF16(src), and with
// prev out[.][ch + 2] = BF16(src - prev) (the layout lb_nn_residual keeps).
__global__ void expand_ch_kernel(const float *__restrict__ src, const float *__restrict__ prev,
                                 bf16 *__restrict__ out, int C, int ch, size_t n) {
    GRID_STRIDE(i, n) {
        out[i * C + ch] = __float2bfloat16(src[i]);
        if (prev) out[i * C + ch + 2] = __float2bfloat16(src[i] - prev[i]);
    }
}

// Weighted residual MSE of one output channel: prediction = base + y[.][ch],
// loss += weight * mean((prediction - target)^2), dy[.][ch] = its gradient
// (no other channel of dy is touched).
__global__ void mse_ch_kernel(const bf16 *__restrict__ y, int C, int ch,
                              const float *__restrict__ tgt, const float *__restrict__ base,
                              size_t n, float weight, float *__restrict__ loss,
                              bf16 *__restrict__ dy) {
    float s = 0.f;
    GRID_STRIDE(i, n) {
        const float d = base[i] + __bfloat162float(y[i * C + ch]) - tgt[i];
        s += d * d;
        if (dy) dy[i * C + ch] = __float2bfloat16(2.f * weight * d / (float)n);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, weight * s / (float)n);
}

// Residual MSE: prediction = base + y[.][0] (FP32 base, BF16 increment),
// loss += mean((prediction - target)^2), dy = d loss / d y (channel 0; 0 elsewhere).
__global__ void mse_kernel(const bf16 *__restrict__ y, int C, const float *__restrict__ tgt,
                           const float *__restrict__ base, size_t n, float *__restrict__ loss,
                           bf16 *__restrict__ dy) {
    float s = 0.f;
    GRID_STRIDE(i, n) {
        const float d = base[i] + __bfloat162float(y[i * C]) - tgt[i];
        s += d * d;
        if (dy) {
            dy[i * C] = __float2bfloat16(2.f * d / (float)n);
            for (int c = 1; c < C; ++c) dy[i * C + c] = __float2bfloat16(0.f);
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s / (float)n);
}

// Mean of channel 0 of y [n][C] in two passes with a fixed summation order:
// block b writes the sum of its grid-stride share to part[b]; one block then
// adds the nb partial sums and writes part[-1] = sum / n (part = buf + 1).
constexpr int kMeanBlocks = 512;
__device__ __forceinline__ float block_sum256(float s) {
    __shared__ float red[8];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    s = 0.f;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;   // valid in thread 0
}
__global__ void __launch_bounds__(256) mean_part_kernel(const bf16 *__restrict__ y, int C, size_t n,
                                                       float *__restrict__ part) {
    float s = 0.f;
    GRID_STRIDE(i, n) s += __bfloat162float(y[i * C]);
    s = block_sum256(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void __launch_bounds__(256) mean_final_kernel(const float *__restrict__ part, int nb,
                                                        size_t n, float *__restrict__ out) {
    float s = 0.f;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b];
    s = block_sum256(s);
    if (threadIdx.x == 0) out[0] = s / (float)n;
}

// Rollout update: state (FP32) += y[.][0] - mean (mean = *mean_in, or 0
// without it: the increment projected to zero mean conserves the mass of the
// field); the next network input x [n][Cx] gets channel 0 = BF16(state) and
// channel 2 = the increment just applied; its other channels are untouched.
__global__ void residual_kernel(float *__restrict__ state, const bf16 *__restrict__ y, int C,
                                bf16 *__restrict__ x, int Cx, size_t n,
                                const float *__restrict__ mean_in) {
    const float mu = mean_in ? mean_in[0] : 0.f;
    GRID_STRIDE(i, n) {
        const float d = __bfloat162float(y[i * C]) - mu;
        const float v = state[i] + d;
        state[i] = v;
        x[i * Cx] = __float2bfloat16(v);
        if (Cx > 2) x[i * Cx + 2] = __float2bfloat16(d);
    }
}

__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, bf16 *__restrict__ wb, size_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    GRID_STRIDE(i, n) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
    }
}

// Network input from an FP32 field: out[i][0] = BF16(src[i]), out[i][1] = gfeat,
// out[i][2] = BF16(src[i] - prev[i]) (the last increment; 0 without prev),
// out[i][3..C) = 0.
__global__ void expand_kernel(const float *__restrict__ src, const float *__restrict__ prev,
                              float gfeat, bf16 *__restrict__ out, int C, size_t n) {
    GRID_STRIDE(i, n) {
        bf16 *o = out + i * C;
        o[0] = __float2bfloat16(src[i]);
        if (C > 1) o[1] = __float2bfloat16(gfeat);
        if (C > 2) o[2] = __float2bfloat16(prev ? src[i] - prev[i] : 0.f);
        for (int c = 3; c < C; ++c) o[c] = __float2bfloat16(0.f);
    }
}

// Increment as the divergence of a flux: J = (y[..][0], y[..][1]) on the
// pixels of [nb][h][w], backward differences with periodic wrap,
//   inc[b][i][j] = -(Jx[i][j] - Jx[i][j-1] + Jy[i][j] - Jy[i-1][j]),
// so every increment conserves the field's mass pixel by pixel (a sum over
// the periodic image telescopes to zero).
__global__ void flux_div_kernel(const bf16 *__restrict__ y, int C, bf16 *__restrict__ inc, int H,
                                int W, size_t n) {
    GRID_STRIDE(p, n) {
        const int j = (int)(p % W);
        const size_t row = p / W;
        const int i = (int)(row % H);
        const size_t img = (row - i) * W;
        const size_t pxm = img + (size_t)i * W + (j == 0 ? W - 1 : j - 1);
        const size_t pym = img + (size_t)(i == 0 ? H - 1 : i - 1) * W + j;
        const float jx = __bfloat162float(y[p * C]), jxm = __bfloat162float(y[pxm * C]);
        const float jy = __bfloat162float(y[p * C + 1]), jym = __bfloat162float(y[pym * C + 1]);
        inc[p] = __float2bfloat16(-((jx - jxm) + (jy - jym)));
    }
}
// Its adjoint: dy[..][0] = -(dinc[i][j] - dinc[i][j+1]),
// dy[..][1] = -(dinc[i][j] - dinc[i+1][j]), the other channels 0.
__global__ void flux_div_bwd_kernel(const bf16 *__restrict__ dinc, bf16 *__restrict__ dy, int C,
                                    int H, int W, size_t n) {
    GRID_STRIDE(p, n) {
        const int j = (int)(p % W);
        const size_t row = p / W;
        const int i = (int)(row % H);
        const size_t img = (row - i) * W;
        const size_t pxp = img + (size_t)i * W + (j == W - 1 ? 0 : j + 1);
        const size_t pyp = img + (size_t)(i == H - 1 ? 0 : i + 1) * W + j;
        const float d = __bfloat162float(dinc[p]);
        bf16 *o = dy + p * C;
        o[0] = __float2bfloat16(-(d - __bfloat162float(dinc[pxp])));
        o[1] = __float2bfloat16(-(d - __bfloat162float(dinc[pyp])));
        for (int c = 2; c < C; ++c) o[c] = __float2bfloat16(0.f);
    }
}

__global__ void f2bf_kernel(const float *__restrict__ a, bf16 *__restrict__ b, size_t n) {
    GRID_STRIDE(i, n) b[i] = __float2bfloat16(a[i]);
}

int blocks_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : b < 152 * 32 ? b : 152 * 32);
}

}  // namespace
}  // namespace lbsc

using namespace lbsc;

#define NN_RET() return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA

extern "C" {

int lb_nn_conv3x3(const void *x, const void *w, const float *bias, void *y, int nb, int h, int wd,
                  int cin, int cout, int relu, int dgrad, void *stream) {
    if (!x || !w || !y || nb < 1 || h < 2 || wd < 2 || ((size_t)h * wd) % 128 || cin % 16 ||
        cout % 16 || cin < 16 || cout < 16)
        return LB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (dgrad && (bias || relu)) return LB_ERR_ARG;
    // automatic choice: the persistent tcgen05 kernel wherever it has one
    // (rows a multiple of 128 pixels), forward and input gradient; it measured
    // fastest on GB300 for every layer of the surrogate
    if (nn_conv_path == 0 || nn_conv_path == 3) {
        const cudaError_t e = launch_conv3x3_tcp(x, w, bias, y, nb, h, wd, cin, cout, relu, dgrad, s);
        if (e == cudaSuccess) return LB_OK;
        if (e != cudaErrorNotSupported) return LB_ERR_CUDA;
    }
    if (!dgrad && nn_conv_path != 1 && nn_conv_path != 3) {
        const cudaError_t e = launch_conv3x3_tc(x, w, bias, y, nb, h, wd, cin, cout, relu, s);
        if (e == cudaSuccess) return LB_OK;
        if (e != cudaErrorNotSupported) return LB_ERR_CUDA;
    }
    // GEMM K channels = channels of the kernel's input, N = of its output
    dim3 grid((unsigned)((size_t)h * wd / 128), nb, 1);
    const bf16 *xb = (const bf16 *)x, *wb = (const bf16 *)w;
    bf16 *yb = (bf16 *)y;
    const int bn = cout % 64 == 0 ? 64 : (cout % 32 == 0 ? 32 : 16);
    grid.z = cout / bn;
    const bool k32 = cin % 32 == 0;
#define LAUNCH(BN, BK, DG) \
    conv3x3_kernel<BN, BK, DG><<<grid, 128, 0, s>>>(xb, wb, bias, yb, h, wd, cin, cout, relu)
    if (!dgrad) {
        if (bn == 64) { if (k32) LAUNCH(64, 32, false); else LAUNCH(64, 16, false); }
        else if (bn == 32) { if (k32) LAUNCH(32, 32, false); else LAUNCH(32, 16, false); }
        else { if (k32) LAUNCH(16, 32, false); else LAUNCH(16, 16, false); }
    } else {
        if (bias || relu) return LB_ERR_ARG;
        if (bn == 64) { if (k32) LAUNCH(64, 32, true); else LAUNCH(64, 16, true); }
        else if (bn == 32) { if (k32) LAUNCH(32, 32, true); else LAUNCH(32, 16, true); }
        else { if (k32) LAUNCH(16, 32, true); else LAUNCH(16, 16, true); }
    }
#undef LAUNCH
    NN_RET();
}

size_t lb_nn_wgrad_workspace(int nb, int h, int wd, int cin, int cout) {
    if (nb < 1 || h < 1 || wd < 1 || cin < 16 || cout < 16 || cin % 16 || cout % 16 ||
        ((size_t)h * wd) % kWgTile)
        return 0;
    // chunk partials of dw (for either kernel), then the bias partials
    // [kBiasBlocks][cout]
    return ((size_t)wgrad_max_chunks(nb, h, wd, cin, cout) * 9 * cout * cin +
            (size_t)kBiasBlocks * cout) *
           sizeof(float);
}

int lb_nn_conv3x3_wgrad(const void *x, const void *dy, float *dw, float *dbias, int nb, int h,
                        int wd, int cin, int cout, void *workspace, size_t workspace_bytes,
                        void *stream) {
    if (!x || !dy || !dw || !workspace || nb < 1 || h < 1 || wd < 1 || cin < 16 || cout < 16 ||
        cin % 16 || cout % 16 || ((size_t)h * wd) % kWgTile)
        return LB_ERR_ARG;
    if (workspace_bytes < lb_nn_wgrad_workspace(nb, h, wd, cin, cout)) return LB_ERR_ARG;
    if ((((uintptr_t)workspace) | ((uintptr_t)x) | ((uintptr_t)dy)) % 16) return LB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const WgPlan p = wgrad_plan(nb, h, wd, cin, cout);
    const bf16 *xb = (const bf16 *)x, *db = (const bf16 *)dy;
    float *part = (float *)workspace;
    const size_t n = (size_t)9 * cout * cin;
    float *bpart = part + (size_t)wgrad_max_chunks(nb, h, wd, cin, cout) * n;
    // tcgen05 kernel where it applies (and unless the mma.sync path is forced)
    int nchunk = 0;
    if (nn_conv_path != 1) {
        static int nsm = 0;
        if (!nsm) {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return LB_ERR_CUDA;
        }
        const int k = wgrad_tc_chunks(nb, h, wd, cin, cout, nsm);
        if (k > 0) {
            const cudaError_t e = launch_wgrad_tc(x, dy, part, nb, h, wd, cin, cout, k, s);
            if (e == cudaSuccess) nchunk = k;
            else if (e != cudaErrorNotSupported) return LB_ERR_CUDA;
        }
    }
    if (nchunk == 0) {   // the mma.sync kernel
        dim3 grid(cout / p.bm, cin / p.bc, p.nchunk);
#define WG(BM, BC)                                                                           \
    wgrad_kernel<BM, BC><<<grid, 32 * (BM / 16) * (BC / 16), 0, s>>>(xb, db, part, h, wd,   \
                                                                     cin, cout, p.ntiles,   \
                                                                     p.tiles_per_chunk)
        if (p.bm == 32) { if (p.bc == 32) WG(32, 32); else WG(32, 16); }
        else { if (p.bc == 32) WG(16, 32); else WG(16, 16); }
#undef WG
        if (cudaGetLastError() != cudaSuccess) return LB_ERR_CUDA;
        nchunk = p.nchunk;
    }
    wgrad_reduce_kernel<<<blocks_for(n), 256, 0, s>>>(part, dw, n, nchunk);
    if (cudaGetLastError() != cudaSuccess) return LB_ERR_CUDA;
    if (dbias) {
        bias_grad_kernel<<<kBiasBlocks, 256, 0, s>>>(db, bpart, (size_t)nb * h * wd, cout);
        if (cudaGetLastError() != cudaSuccess) return LB_ERR_CUDA;
        bias_reduce_kernel<<<cout, 256, 0, s>>>(bpart, dbias, cout, kBiasBlocks);
    }
    NN_RET();
}

int lb_nn_relu_mask(const void *dy, const void *y, void *dz, size_t n, void *stream) {
    relu_mask_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(
        (const bf16 *)dy, (const bf16 *)y, (bf16 *)dz, n);
    NN_RET();
}

int lb_nn_pool2(const void *x, void *y, int nb, int h, int w, int c, int backward, void *stream) {
    if (h % 2 || w % 2) return LB_ERR_ARG;
    const size_t n = backward ? (size_t)nb * h * w * c : (size_t)nb * (h / 2) * (w / 2) * c;
    if (!backward)
        pool2_fwd_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, (bf16 *)y, nb, h, w, c);
    else
        pool2_bwd_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, (bf16 *)y, nb, h, w, c);
    NN_RET();
}

int lb_nn_up2(const void *x, void *y, int nb, int h, int w, int c, int backward, void *stream) {
    // (h, w): the coarse size
    const size_t n = backward ? (size_t)nb * h * w * c : (size_t)nb * 4 * h * w * c;
    if (!backward)
        up2_fwd_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, (bf16 *)y, nb, h, w, c);
    else
        up2_bwd_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, (bf16 *)y, nb, h, w, c);
    NN_RET();
}

int lb_nn_add(const void *a, const void *b, void *y, size_t n, void *stream) {
    add_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>((const bf16 *)a, (const bf16 *)b, (bf16 *)y, n);
    NN_RET();
}

int lb_nn_coarse_grain(const float *df, int nx, int ny, int f, double scale, float *out,
                       void *stream) {
    if (!df || !out || f < 1 || nx % f || ny % f || !(scale != 0.0)) return LB_ERR_ARG;
    coarse_kernel<<<blocks_for((size_t)(nx / f) * (ny / f)), 256, 0, (cudaStream_t)stream>>>(
        df, nx, ny, f, (float)scale, out);
    NN_RET();
}

int lb_nn_add_channel(void *dst, int dc, int dch, const void *src, int sc, int sch, size_t n,
                      void *stream) {
    if (!dst || !src || dch < 0 || dch >= dc || sch < 0 || sch >= sc) return LB_ERR_ARG;
    add_channel_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(
        (bf16 *)dst, dc, dch, (const bf16 *)src, sc, sch, n);
    NN_RET();
}

int lb_nn_mse_blocks(const void *y, int c, const float *target, const float *base, int nb, int h,
                     int w, int block, double weight, float *loss, void *dy, void *stream) {
    if (!y || !target || !base || !loss || c < 1 || nb < 1 || block < 1 || h % block ||
        w % block)
        return LB_ERR_ARG;
    const int nblocks = nb * (h / block) * (w / block);
    mse_block_kernel<<<nblocks, 256, 0, (cudaStream_t)stream>>>(
        (const bf16 *)y, c, target, base, h, w, block, (float)weight, 1.f / (float)nblocks, loss,
        (bf16 *)dy);
    NN_RET();
}

int lb_nn_coarse_momentum(const float *df, int nx, int ny, int f, double scale, float *jx,
                          float *jy, void *stream) {
    if (!df || !jx || !jy || f < 1 || nx % f || ny % f || !(scale != 0.0)) return LB_ERR_ARG;
    coarse_mom_kernel<<<blocks_for((size_t)(nx / f) * (ny / f)), 256, 0, (cudaStream_t)stream>>>(
        df, nx, ny, f, (float)scale, jx, jy);
    NN_RET();
}

int lb_nn_expand_channel(const float *src, const float *prev, void *out, int c, int ch, size_t n,
                         void *stream) {
    if (!src || !out || ch < 0 || ch >= c || (prev && ch + 2 >= c)) return LB_ERR_ARG;
    expand_ch_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(src, prev, (bf16 *)out, c,
                                                                      ch, n);
    NN_RET();
}

int lb_nn_mse_channel(const void *y, int c, int ch, const float *target, const float *base,
                      size_t n, double weight, float *loss, void *dy, void *stream) {
    if (!y || !target || !base || !loss || ch < 0 || ch >= c) return LB_ERR_ARG;
    mse_ch_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(
        (const bf16 *)y, c, ch, target, base, n, (float)weight, loss, (bf16 *)dy);
    NN_RET();
}

int lb_nn_mse(const void *y, int c, const float *target, const float *base, size_t n, float *loss,
              void *dy, void *stream) {
    if (!y || !target || !base || !loss || c < 1) return LB_ERR_ARG;
    mse_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(
        (const bf16 *)y, c, target, base, n, loss, (bf16 *)dy);
    NN_RET();
}

int lb_nn_residual(float *state, const void *y, int c, void *x, int cx, size_t n, float *mean_buf,
                   void *stream) {
    if (!state || !y || !x || c < 1 || cx < 1) return LB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (mean_buf) {
        size_t want = (n + 2047) / 2048;
        const int nb = (int)(want < 1 ? 1 : (want > (size_t)kMeanBlocks ? kMeanBlocks : want));
        mean_part_kernel<<<nb, 256, 0, s>>>((const bf16 *)y, c, n, mean_buf + 1);
        mean_final_kernel<<<1, 256, 0, s>>>(mean_buf + 1, nb, n, mean_buf);
        if (cudaGetLastError() != cudaSuccess) return LB_ERR_CUDA;
    }
    residual_kernel<<<blocks_for(n), 256, 0, s>>>(state, (const bf16 *)y, c, (bf16 *)x, cx, n,
                                                  mean_buf);
    NN_RET();
}

int lb_nn_adam(float *w, const float *g, float *m, float *v, void *w_bf16, size_t n, double lr,
               double b1, double b2, double eps, long long step, void *stream) {
    const float c1 = (float)(1.0 - pow(b1, (double)step)), c2 = (float)(1.0 - pow(b2, (double)step));
    adam_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, (bf16 *)w_bf16, n,
                                                                 (float)lr, (float)b1, (float)b2,
                                                                 (float)eps, c1, c2);
    NN_RET();
}

int lb_nn_expand(const float *src, const float *prev, double gfeat, void *out, int c, size_t n,
                 void *stream) {
    if (!src || !out || c < 1) return LB_ERR_ARG;
    expand_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(src, prev, (float)gfeat,
                                                                   (bf16 *)out, c, n);
    NN_RET();
}

int lb_nn_flux_div(const void *in, void *out, int c, int nb, int h, int w, int backward,
                   void *stream) {
    if (!in || !out || c < 2 || nb < 1 || h < 1 || w < 1) return LB_ERR_ARG;
    const size_t n = (size_t)nb * h * w;
    if (!backward)
        flux_div_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(
            (const bf16 *)in, c, (bf16 *)out, h, w, n);
    else
        flux_div_bwd_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(
            (const bf16 *)in, (bf16 *)out, c, h, w, n);
    NN_RET();
}

int lb_nn_to_bf16(const float *a, void *b, size_t n, void *stream) {
    f2bf_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(a, (bf16 *)b, n);
    NN_RET();
}

}  // extern "C"
