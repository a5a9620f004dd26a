// Fused D2Q9 step with TMA-staged rows (FP32, nx a multiple of 128).
//
// Same arithmetic as step_kernel (Eq. (12) with the force of Eq. (1)); only
// the data movement differs.  A CTA owns a strip of 128 columns and sweeps
// strip_h rows.  One producer thread brings each lattice row of the strip --
// all nine planes, columns x0-4 .. x0+131 -- into a shared-memory ring with a
// single three-dimensional bulk tensor copy (cp.async.bulk.tensor) that
// completes on an mbarrier, several rows ahead of use.  Every pull is then a
// shared-memory load with an immediate offset, so the streaming step costs no
// global address arithmetic and no register queue.  The new populations of a
// row are staged in shared memory and written back with a bulk tensor store.
//
// Columns outside [0, nx) arrive zero-filled (the copy starts at x0 - 4);
// in the first and last strip the halo warp overwrites them with the
// periodic images (plain loads) once the copy has landed.  Every wait is
// bounded in time (a per-context limit, 2 s by default): on expiry the
// kernel records LB_STEP_TIMEOUT in the flag, lets every thread leave
// through the same barrier, and waits (with the default bound) for its
// copies in flight before returning.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbsc_collide.cuh"
#include "lbsc_device.cuh"
#include "lbsc_internal.cuh"

namespace lbsc {

namespace {

constexpr int kTX = kStepTX;            // interior columns per CTA (128)
constexpr int kBox = kTX + 8;           // columns per staged row: x0-4 .. x0+131
constexpr int kSlot = 1248;             // floats per ring slot: 9 x 136 = 1224 padded to 128 B
constexpr uint64_t kWaitNs = 2000000000ull;   // default bound on a wait: 2 s

template <int H> struct TmaCfg {
    static constexpr int R = (H == 1) ? 6 : 8;            // ring rows (>= lookahead + H + 3)
    static constexpr int PSI_RING = (H == 1) ? 4 : 8;     // rows of the pseudopotential ring
    static constexpr int W = kTX + 2 * H;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
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
// Wait for the phase with the given parity; false if it has not completed
// within limit_ns (0: give up at the first unfinished check, which does not
// block).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_test_wait(bar, parity)) return true;
    if (limit_ns == 0) return false;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void tma_load_row(float *dst, const CUtensorMap *map, int x, int y,
                                             uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(0), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_row(const CUtensorMap *map, int x, int y,
                                              const float *src) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(x), "r"(y), "r"(0), "r"(smem_u32(src))
        : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Pull streaming from three staged rows (y-1, y, y+1) at smem column c of
// each row: g_i = f_i(x - c_i).  Plane i of a slot starts at i * kBox.
__device__ __forceinline__ void pull_smem(const float *rm, const float *rc, const float *rp,
                                          float g[9]) {
    g[0] = rc[0 * kBox];
    g[1] = rc[1 * kBox - 1];   // c = ( 1, 0): from x-1
    g[2] = rm[2 * kBox];       // c = ( 0, 1): from y-1
    g[3] = rc[3 * kBox + 1];   // c = (-1, 0)
    g[4] = rp[4 * kBox];       // c = ( 0,-1)
    g[5] = rm[5 * kBox - 1];   // c = ( 1, 1)
    g[6] = rm[6 * kBox + 1];   // c = (-1, 1)
    g[7] = rp[7 * kBox + 1];   // c = (-1,-1)
    g[8] = rp[8 * kBox - 1];   // c = ( 1,-1)
}

}  // namespace

template <int ORDER, bool SAMPLE>
__global__ void __launch_bounds__(kTX + 32)
step_kernel_tma(const __grid_constant__ CUtensorMap tm_src,
                const __grid_constant__ CUtensorMap tm_dst, const KParams<float> p,
                const unsigned long long wait_ns) {
    using S = Stencil<ORDER>;
    constexpr int H = S::H;
    using Cfg = TmaCfg<H>;
    constexpr int R = Cfg::R;
    constexpr int PR = Cfg::PSI_RING;
    constexpr int W = Cfg::W;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>(smem_raw);          // R x kSlot
    float *stage = ring + R * kSlot;                             // 2 x 9 x kTX
    float *spsi = stage + 2 * 9 * kTX;                           // PR x W
    uint64_t *bar = reinterpret_cast<uint64_t *>(spsi + PR * W);  // R mbarriers

    const int nx = p.nx, ny = p.ny;
    const int tx = threadIdx.x;
    const int x0 = blockIdx.x * kTX;
    const int y0 = blockIdx.y * p.strip_h;
    const int y1 = min(y0 + p.strip_h, ny);
    const int it_end = (y1 - y0) + 2 * H;
    const int nrows = it_end + 2;            // staged row k <-> lattice row y0 - H - 1 + k
    const bool interior = tx < kTX;
    const int hl = tx - kTX;
    const bool halo = !interior && hl < 2 * H;
    const bool producer = (tx == kTX + 31);
    const bool edge_l = (x0 == 0), edge_r = (x0 + kTX == nx);

    // column of this thread's site inside a staged row and inside the psi ring
    int col, pcol;
    if (interior) {
        col = tx + 4;
        pcol = tx + H;
    } else {
        const int h = min(hl, 2 * H - 1);
        col = h < H ? 4 - H + h : 4 + kTX + (h - H);
        pcol = h < H ? h : kTX + H + (h - H);
    }

    if (tx == 0) {
        for (int s = 0; s < R; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const uint32_t row_bytes = 9u * kBox * 4u;
    auto issue = [&](int k) {
        const int s = k % R;
        const int y = (y0 - H - 1 + k + 2 * ny) % ny;
        fence_proxy_async();
        mbar_expect_tx(&bar[s], row_bytes);
        tma_load_row(ring + s * kSlot, &tm_src, x0 - 4, y, &bar[s]);
    };
    auto slot_of = [&](int k) { return ring + (k % R) * kSlot; };
    auto parity_of = [&](int k) { return (uint32_t)((k / R) & 1); };

    // Periodic images of the zero-filled columns in the first and last strip.
    auto fixup = [&](int k) {
        if (!(edge_l || edge_r) || interior) return;
        const int y = (y0 - H - 1 + k + 2 * ny) % ny;
        float *slot = slot_of(k);
        const size_t plane = (size_t)nx * ny;
        const int nside = (edge_l ? 1 : 0) + (edge_r ? 1 : 0);
        for (int e = hl; e < 36 * nside; e += 32) {
            const bool left = edge_l && e < 36;
            const int ee = e % 36, i = ee / 4, c = ee % 4;
            const int gx = left ? nx - 4 + c : c;
            const int sc = left ? c : 4 + kTX + c;
            slot[i * kBox + sc] = __ldg(p.src + i * plane + (size_t)y * nx + gx);
        }
        fence_proxy_async();
    };

    // Lookahead: after the barrier of iteration it, row it + R - H - 1 is
    // issued into the slot of row it - H - 1, which no thread reads again.
    // Abort decisions are taken only through __syncthreads_or, so every
    // thread of the CTA leaves the loop at the same barrier.
    const int pre = min(R - H - 2, nrows - 1);
    int last_issued = -1;
    if (producer) {
        for (int k = 0; k <= pre; ++k) issue(k);
        last_issued = pre;
    }
    bool ok = true;
    // rows 0..2 are read in iteration 0 and must be in place (and fixed) first
    for (int k = 0; k < 3 && k < nrows; ++k)
        ok = ok && mbar_wait(&bar[k % R], parity_of(k), wait_ns);
    if (ok)
        for (int k = 0; k < 3 && k < nrows; ++k) fixup(k);
    bool aborted = __syncthreads_or(!ok) != 0;

    const float rho0 = p.rho0;
    for (int it = 0; it < it_end && !aborted; ++it) {
        // halo warp: fix the periodic columns of row it+3 (read from iteration it+1 on)
        if (!interior && (edge_l || edge_r) && it + 3 < nrows) {
            if (mbar_wait(&bar[(it + 3) % R], parity_of(it + 3), wait_ns))
                fixup(it + 3);
            else
                ok = false;
        }
        // newest row of this iteration's psi pulls
        if (!mbar_wait(&bar[(it + 2) % R], parity_of(it + 2), wait_ns)) ok = false;

        const int pslot = it & (PR - 1);
        if (interior || halo) {
            float g[9];
            pull_smem(slot_of(it) + col, slot_of(it + 1) + col, slot_of(it + 2) + col, g);
            spsi[pslot * W + pcol] = delta_psi<float>(sum9(g), p.psi_kind, rho0, p.psi_c, p.psi_b);
        }
        // the store of the row collided in the previous iteration must have
        // read its staging buffer before that buffer is written again
        if (producer) bulk_wait_read_all();
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        if (producer) {
            const int knew = it + R - H - 1;
            if (knew < nrows) {
                issue(knew);
                last_issued = knew;
            }
            if (it - 1 >= 2 * H) {
                const int yprev = y0 + (it - 1) - 2 * H;
                tma_store_row(&tm_dst, x0, yprev, stage + ((it - 1) & 1) * 9 * kTX);
            }
        }
        if (it < 2 * H || !interior) continue;

        // ---- collide row yr ------------------------------------------------
        const int yr = y0 + it - 2 * H;
        float sx = 0.f, sy = 0.f;
#pragma unroll
        for (int a = 0; a < S::N; ++a) {
            const HalfVec hv = S::v(a);
            const float dpl = spsi[((it - H + hv.ey) & (PR - 1)) * W + pcol + hv.ex];
            const float dmi = spsi[((it - H - hv.ey) & (PR - 1)) * W + pcol - hv.ex];
            const float d = float(hv.w) * (dpl - dmi);
            if (hv.ex != 0) sx += float(hv.ex) * d;
            if (hv.ey != 0) sy += float(hv.ey) * d;
        }
        const float psic = p.psi0 + spsi[((it - H) & (PR - 1)) * W + pcol];
        const float Fx = p.force_pref * psic * sx;
        const float Fy = p.force_pref * psic * sy;

        float g[9], f[9];
        pull_smem(slot_of(it - H) + col, slot_of(it - H + 1) + col, slot_of(it - H + 2) + col, g);
        collide(g, Fx, Fy, p, p.rk, (uint32_t)(x0 + tx) + (uint32_t)nx * (uint32_t)yr, step_of(p), f);
        float *st = stage + (it & 1) * 9 * kTX + tx;
#pragma unroll
        for (int i = 0; i < 9; ++i) st[i * kTX] = f[i];
        fence_proxy_async();
        if (SAMPLE) p.drho_out[(size_t)yr * nx + x0 + tx] = sum9(g);
        if (!isfinite(f[1] + f[5])) atomicOr(p.flag, LB_STEP_NONFINITE);
    }
    __syncthreads();
    if (producer) {
        if (!aborted && it_end - 1 >= 2 * H) {
            const int ylast = y0 + (it_end - 1) - 2 * H;
            tma_store_row(&tm_dst, x0, ylast, stage + ((it_end - 1) & 1) * 9 * kTX);
        }
        bulk_wait_all();
        if (aborted) {
            atomicOr(p.flag, LB_STEP_TIMEOUT);
            // let every copy this CTA issued land before its shared memory is
            // released (each wait bounded again, by the default bound)
            for (int k = max(0, last_issued - R + 1); k <= last_issued; ++k)
                mbar_wait(&bar[k % R], parity_of(k), kWaitNs);
        }
    }
}

// ---------------------------------------------------------------------------
// Host side: tensor maps over the [9][ny][nx] FP32 population buffers.
// ---------------------------------------------------------------------------
namespace {
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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

bool encode(CUtensorMap *m, void *base, int nx, int ny, uint32_t box_x) {
    auto fn = get_encode();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 9};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
    const cuuint32_t box[3] = {box_x, 1, 9};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int H> constexpr size_t tma_smem() {
    return (size_t)TmaCfg<H>::R * kSlot * 4 + 2 * 9 * kTX * 4 +
           (size_t)TmaCfg<H>::PSI_RING * TmaCfg<H>::W * 4 + TmaCfg<H>::R * 8;
}
}  // namespace

bool tma_eligible(int precision, int nx, int ny) {
    return precision == 0 && nx % kTX == 0 && nx >= kTX && ny >= 4 && get_encode() != nullptr;
}

bool tma_encode_maps(TmaMaps *m, void *buf0, void *buf1, int nx, int ny) {
    static_assert(sizeof(CUtensorMap) == sizeof(m->load[0]), "tensor map size");
    CUtensorMap *ld = reinterpret_cast<CUtensorMap *>(m->load);
    CUtensorMap *stv = reinterpret_cast<CUtensorMap *>(m->store);
    m->ok = encode(&ld[0], buf0, nx, ny, kBox) && encode(&ld[1], buf1, nx, ny, kBox) &&
            encode(&stv[0], buf0, nx, ny, kTX) && encode(&stv[1], buf1, nx, ny, kTX);
    return m->ok;
}

template <int ORDER>
static cudaError_t launch_tma_t(const StepArgs &a, const TmaMaps &m, int src_buf, cudaStream_t s) {
    constexpr int H = Stencil<ORDER>::H;
    const KParams<float> k = make_params<float>(a);
    const CUtensorMap *ld = reinterpret_cast<const CUtensorMap *>(m.load);
    const CUtensorMap *stv = reinterpret_cast<const CUtensorMap *>(m.store);
    const size_t smem = tma_smem<H>();
    dim3 grid(a.nx / kTX, (a.ny + a.strip_h - 1) / a.strip_h);
    const unsigned long long wait_ns = a.wait_ns < 0 ? kWaitNs : (unsigned long long)a.wait_ns;
    cudaError_t e;
    if (a.drho_out) {
        e = cudaFuncSetAttribute(step_kernel_tma<ORDER, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        step_kernel_tma<ORDER, true>
            <<<grid, kTX + 32, smem, s>>>(ld[src_buf], stv[src_buf ^ 1], k, wait_ns);
    } else {
        e = cudaFuncSetAttribute(step_kernel_tma<ORDER, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        step_kernel_tma<ORDER, false>
            <<<grid, kTX + 32, smem, s>>>(ld[src_buf], stv[src_buf ^ 1], k, wait_ns);
    }
    return cudaGetLastError();
}

cudaError_t launch_step_tma(int stencil, const StepArgs &a, const TmaMaps &m, int src_buf,
                            cudaStream_t s) {
    if (stencil == 4) return launch_tma_t<4>(a, m, src_buf, s);
    if (stencil == 6) return launch_tma_t<6>(a, m, src_buf, s);
    if (stencil == 8) return launch_tma_t<8>(a, m, src_buf, s);
    return cudaErrorInvalidValue;
}

}  // namespace lbsc
