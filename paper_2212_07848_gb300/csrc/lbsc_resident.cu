// Shared-memory-resident replicas of a batched ensemble.
//
// A replica of up to 4096 sites (64^2 FP32: 147 KB of populations) lives in
// one CTA's shared memory for a whole window of steps; a taller one (128^2)
// is split by rows over a cluster of C CTAs that read each other's boundary
// rows through distributed shared memory.  HBM is touched to load the state
// at the start of the window, to store it at the end and to write delta rho
// at a sampling step: a window of n steps moves 72 B per site once instead
// of n times.
//
// Layout of one CTA (rows [rank R, rank R + R) of its replica, R = ny / C):
// the nine population planes [9][Rtot][nx], Rtot = R + (nb + 1)(H + 1) --
// the R own rows, then nb + 1 blocks of H + 1 copied rows -- and nb rings of
// delta psi rows.  The CTA is nb bands of hb rows, one thread per column and
// band.  Each band sweeps its rows like a strip of the global kernel (pull
// one row ahead, delta psi into its ring, collide H rows behind) and writes
// the new populations in place.  All bands advance in lock step, one barrier
// per row, and in-place writes are safe because
//  * a band reads each of its own rows at least H rows before it writes it;
//  * a band pulls its lower halo (the last H + 1 rows of the band below)
//    at the start of its sweep, before that band writes them at the end;
//  * the first H + 1 rows of the band above are written at the start of the
//    sweep but pulled at the end, so they are copied before the sweep, each
//    step; so are the H + 1 rows below the CTA's lowest band, which belong
//    to the previous CTA of the cluster (to the CTA itself when C = 1).
// Copies from another CTA are distributed-shared-memory loads between two
// cluster barriers: one after the previous step's writes, one before this
// step's.  The arithmetic, summation order and Philox counters are those of
// the tile path, so a resident replica evolves bit-identically to a single
// lattice with the same seed and replica index.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbsc.h"
#include "lbsc_ens.cuh"

namespace lbsc {
namespace {

constexpr int kResMaxThreads = 512;

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The float at the offset of `p` in the shared memory of cluster CTA `rank`.
__device__ __forceinline__ float ld_cluster(const float *p, uint32_t rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra) : "memory");
    return v;
}
template <int C>
__device__ __forceinline__ void sync_all() {
    if constexpr (C > 1) cluster_sync();
    else __syncthreads();
}

template <int ORDER>
__host__ __device__ constexpr int res_ring() {
    return Stencil<ORDER>::H == 1 ? 4 : 8;   // >= 2H + 2 rows, power of two
}

// Pull of one site from shared memory, the streaming of the global pull:
// rows rm, rc, rp hold y - 1, y, y + 1 (shared-memory row indices).
__device__ __forceinline__ void pull_sm(const float *sm, uint32_t P, int nx, int xc, int xm,
                                        int xp, int rm, int rc, int rp, float g[9]) {
    const float *c = sm + rc * nx, *m = sm + rm * nx, *q = sm + rp * nx;
    g[0] = c[xc];
    g[1] = c[P + xm];
    g[2] = m[2u * P + xc];
    g[3] = c[3u * P + xp];
    g[4] = q[4u * P + xc];
    g[5] = m[5u * P + xm];
    g[6] = m[6u * P + xp];
    g[7] = q[7u * P + xp];
    g[8] = q[8u * P + xm];
}

// One step of one band: rows [y0, y0 + hb) of the CTA, in place.
template <int ORDER, bool UNIT>
__device__ __forceinline__ void res_sweep(const KParams<float> &p, const uint32_t *__restrict__ rk,
                                          float *sm, float *ring, uint32_t P, int nx, int rows,
                                          int band, int hb, int tx, int ybase) {
    using S = Stencil<ORDER>;
    constexpr int H = S::H;
    constexpr int RING = res_ring<ORDER>();
    const int y0 = band * hb, y1 = y0 + hb;
    const int xm = (tx - 1) & (nx - 1), xp = (tx + 1) & (nx - 1);
    // shared-memory row of local row ys as this band pulls it
    auto row_of = [&](int ys) {
        if (ys >= y1) return rows + (H + 1) * (1 + band) + (ys - y1);
        if (ys < 0) return rows + (ys + H + 1);
        return ys;
    };
    const float rho0 = p.rho0;
    constexpr int NQ = UNIT ? 4 : 9;
    float q[H + 1][NQ];
#pragma unroll
    for (int r = 0; r <= H; ++r)
#pragma unroll
        for (int i = 0; i < NQ; ++i) q[r][i] = 0.f;

    const int it_end = hb + 2 * H;
    float gn[9];
    pull_sm(sm, P, nx, tx, xm, xp, row_of(y0 - H - 1), row_of(y0 - H), row_of(y0 - H + 1), gn);
#pragma unroll 2
    for (int it = 0; it < it_end; ++it) {
        const int slot = it & (RING - 1);
        float g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = gn[i];
        if (it + 1 < it_end) {
            const int yc = y0 - H + it + 1;
            pull_sm(sm, P, nx, tx, xm, xp, row_of(yc - 1), row_of(yc), row_of(yc + 1), gn);
        }
        const float s9 = sum9(g);
        ring[slot * nx + tx] = delta_psi<float>(s9, p.psi_kind, rho0, p.psi_c, p.psi_b);
#pragma unroll
        for (int r = 0; r < H; ++r)
#pragma unroll
            for (int i = 0; i < NQ; ++i) q[r][i] = q[r + 1][i];
        if constexpr (UNIT) {
            q[H][0] = s9;
            unit_moments(g, q[H][1], q[H][2], q[H][3]);
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) q[H][i] = g[i];
        }
        __syncthreads();
        if (it < 2 * H) continue;

        const int yr = y0 - 2 * H + it;   // the row collided, local
        float sx = 0.f, sy = 0.f;
#pragma unroll
        for (int a = 0; a < S::N; ++a) {
            const HalfVec hv = S::v(a);
            const float dpl = ring[((it - H + hv.ey) & (RING - 1)) * nx + ((tx + hv.ex) & (nx - 1))];
            const float dmi = ring[((it - H - hv.ey) & (RING - 1)) * nx + ((tx - hv.ex) & (nx - 1))];
            const float d = float(hv.w) * (dpl - dmi);
            if (hv.ex != 0) sx += float(hv.ex) * d;
            if (hv.ey != 0) sy += float(hv.ey) * d;
        }
        const float psic = p.psi0 + ring[((it - H) & (RING - 1)) * nx + tx];
        const float Fx = p.force_pref * psic * sx;
        const float Fy = p.force_pref * psic * sy;

        float f[9];
        const int yg = ybase + yr;
        const uint32_t site = (uint32_t)tx + (uint32_t)nx * (uint32_t)yg;
        if constexpr (UNIT) collide_unit_m(q[0][1], q[0][2], q[0][3], Fx, Fy, p, rk, site, p.step, f);
        else collide<float, false>(q[0], Fx, Fy, p, rk, site, p.step, f);
        float *w = sm + yr * nx + tx;
#pragma unroll
        for (int i = 0; i < 9; ++i) w[i * P] = f[i];
        if (p.drho_out) {
            if constexpr (UNIT) p.drho_out[site] = q[0][0];
            else p.drho_out[site] = sum9(q[0]);
        }
        if (!isfinite(f[1] + f[5])) atomicOr(p.flag, LB_STEP_NONFINITE);
    }
}

// `nsteps` steps of every replica in `list` (one shape), C CTAs per replica.
template <int ORDER, int C>
__global__ void __launch_bounds__(kResMaxThreads)
ens_resident_kernel(const EnsRep *__restrict__ reps, const int *__restrict__ list,
                    const EnsClock *__restrict__ clk, int *flag, const EnsKeys keys, int nsteps,
                    int sample, int hb) {
    constexpr int H = Stencil<ORDER>::H;
    constexpr int RING = res_ring<ORDER>();
    extern __shared__ __align__(16) float sm[];
    __shared__ KParams<float> sp;
    __shared__ uint32_t s_t0;
    __shared__ int s_cur;
    const uint32_t rank = C > 1 ? cluster_rank() : 0u;
    const EnsRep &R = reps[list[blockIdx.x / C]];
    const int nx = R.nx, ny = R.ny;
    const int rows = ny / C, nb = rows / hb;
    const uint32_t P = (uint32_t)(rows + (nb + 1) * (H + 1)) * nx;   // plane stride
    const int tx = threadIdx.x & (nx - 1), band = threadIdx.x / nx;
    const int ybase = (int)rank * rows;
    float *ring = sm + 9 * P + band * RING * nx;
    if (threadIdx.x == 0) {
        s_t0 = __ldcg(&clk->t);
        s_cur = __ldcg(&clk->cur);
        const EnsTile whole = {0, 0, 0, hb};
        fill_tile_params(sp, R, whole, s_t0, s_cur, false, flag);
    }
    __syncthreads();
    const uint32_t t0 = s_t0;
    const int cur = s_cur;
    const bool unit = sp.gamma == 0.f;   // every rate 1: the unit path
    const uint32_t gplane = (uint32_t)nx * ny;
    const uint32_t n4 = (uint32_t)rows * nx / 4;   // float4 of a plane's own rows
    {
        const float4 *src = reinterpret_cast<const float4 *>(R.buf[cur]);
        for (uint32_t k = threadIdx.x; k < 9 * n4; k += blockDim.x) {
            const uint32_t i = k / n4, e = k - i * n4;
            reinterpret_cast<float4 *>(sm + i * P)[e] =
                __ldcg(src + (i * gplane + (uint32_t)ybase * nx) / 4 + e);
        }
    }
    const int ncopy = (nb + 1) * (H + 1);
    for (int s = 0; s < nsteps; ++s) {
        sync_all<C>();   // the previous step's writes (or the load) are done
        // the copied rows: the lower halo of band 0, then each band's upper halo
        for (int c = band; c < ncopy; c += nb) {
            int drow, from;
            uint32_t srank = rank;
            if (c <= H) {
                drow = rows + c;
                from = rows - (H + 1) + c;
                srank = (rank + C - 1) % C;
            } else {
                const int b = c / (H + 1) - 1, j = c - (b + 1) * (H + 1);
                drow = rows + (H + 1) * (1 + b) + j;
                if (b < nb - 1) {
                    from = (b + 1) * hb + j;
                } else {
                    from = j;
                    srank = (rank + 1) % C;
                }
            }
            const float *src = sm + from * nx + tx;
            float *dst = sm + drow * nx + tx;
#pragma unroll
            for (int i = 0; i < 9; ++i)
                dst[i * P] = (C > 1 && srank != rank) ? ld_cluster(src + i * P, srank) : src[i * P];
        }
        if (threadIdx.x == 0) {
            sp.step = t0 + (uint32_t)s;
            sp.drho_out = (sample && s == nsteps - 1) ? R.drho : nullptr;
        }
        sync_all<C>();   // the copies are done before any row is overwritten
        if (unit) res_sweep<ORDER, true>(sp, keys.rk, sm, ring, P, nx, rows, band, hb, tx, ybase);
        else res_sweep<ORDER, false>(sp, keys.rk, sm, ring, P, nx, rows, band, hb, tx, ybase);
    }
    __syncthreads();
    {
        float4 *dst = reinterpret_cast<float4 *>(R.buf[cur ^ (nsteps & 1)]);
        for (uint32_t k = threadIdx.x; k < 9 * n4; k += blockDim.x) {
            const uint32_t i = k / n4, e = k - i * n4;
            dst[(i * gplane + (uint32_t)ybase * nx) / 4 + e] =
                reinterpret_cast<const float4 *>(sm + i * P)[e];
        }
    }
}

template <int ORDER>
const void *res_fn_o(int C) {
    switch (C) {
    case 1: return (const void *)ens_resident_kernel<ORDER, 1>;
    case 2: return (const void *)ens_resident_kernel<ORDER, 2>;
    case 4: return (const void *)ens_resident_kernel<ORDER, 4>;
    case 8: return (const void *)ens_resident_kernel<ORDER, 8>;
    default: return nullptr;
    }
}
const void *res_fn(int stencil, int C) {
    return stencil == 4 ? res_fn_o<4>(C) : stencil == 6 ? res_fn_o<6>(C) : res_fn_o<8>(C);
}

}  // namespace

size_t resident_smem(int nx, int rows, int hb, int stencil) {
    const int H = stencil == 4 ? 1 : 2, ring = H == 1 ? 4 : 8;
    if ((nx != 32 && nx != 64 && nx != 128) || hb < 2 * H + 2 || rows % hb) return 0;
    const int nb = rows / hb;
    if (nb * nx > kResMaxThreads) return 0;
    return ((size_t)9 * (rows + (nb + 1) * (H + 1)) * nx + (size_t)nb * ring * nx) *
           sizeof(float);
}

cudaError_t resident_prepare(int stencil, int C, size_t smem) {
    const void *fn = res_fn(stencil, C);
    if (!fn) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int resident_max_clusters(int stencil, int C, int nx, int rows, int hb, size_t smem) {
    const void *fn = res_fn(stencil, C);
    if (!fn) return 0;
    const int threads = rows / hb * nx;
    if (C == 1) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess)
            return 0;
        return n;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = C;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_ens_resident(const ResLaunch &a, cudaStream_t s) {
    const void *fn = res_fn(a.stencil, a.C);
    if (!fn || a.nres < 1) return cudaErrorInvalidValue;
    const int rows = a.ny / a.C;
    const size_t smem = resident_smem(a.nx, rows, a.hb, a.stencil);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.nres * a.C);
    cfg.blockDim = dim3(rows / a.hb * a.nx);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = a.C;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = a.C > 1 ? 1 : 0;
    const EnsRep *reps = a.reps;
    const int *list = a.list;
    const EnsClock *clk = a.clk;
    int *flag = a.flag;
    const EnsKeys keys = a.keys;
    int nsteps = a.nsteps, sample = a.sample, hb = a.hb;
    void *args[] = {(void *)&reps, (void *)&list, (void *)&clk,    (void *)&flag,
                    (void *)&keys, (void *)&nsteps, (void *)&sample, (void *)&hb};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace lbsc
