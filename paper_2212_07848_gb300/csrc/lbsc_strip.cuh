// The fused D2Q9 step for one strip of a lattice (shared by the
// single-lattice kernel and the batched ensemble kernel).  See lbsc_step.cu
// for the design.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbsc_collide.cuh"
#include "lbsc_device.cuh"
#include "lbsc_internal.cuh"

namespace lbsc {

// One CTA's work: the strip of columns [x0, x0 + kStepTX) and rows [y0, y1)
// of the lattice described by p (the CTA has kStepTX + 32 threads).  Shared
// by the single-lattice kernel and the batched ensemble kernel.
// rk: the Philox round keys (kept apart from p so that callers can serve
// them from the constant bank).  CG: pull through L2 only (the source was
// written earlier in the same launch, as in the persistent ensemble kernel).
// UNIT: all relaxation rates are 1 (see collide).
template <typename T, int ORDER, bool SAMPLE, bool CG = false, bool UNIT = false>
__device__ __forceinline__ void step_strip(const KParams<T> &p, const uint32_t *__restrict__ rk,
                                           int x0, int y0, int y1) {
    using S = Stencil<ORDER>;
    constexpr int H = S::H;
    constexpr int RING = (H == 1) ? 4 : 8;   // >= 2H + 2 rows, power of two
    constexpr int W = kStepTX + 2 * H;
    __shared__ T s_dpsi[RING][W];

    const int nx = p.nx, ny = p.ny;
    const size_t plane = (size_t)nx * ny;
    const int tx = threadIdx.x;
    const int xe = min(x0 + kStepTX, nx);
    const int ncol = xe - x0;

    // Threads 0..kStepTX-1 own the strip's columns; the extra warp owns the
    // 2H halo columns (left, then right) and only computes their
    // pseudopotential, so every warp does the same pull-and-psi work per row.
    const bool interior = tx < kStepTX;
    const int hl = tx - kStepTX;
    const bool active = interior ? (tx < ncol) : (hl < 2 * H);
    int x, slot_col;
    if (interior) {
        x = active ? x0 + tx : x0;
        slot_col = tx + H;
    } else if (hl < H) {
        x = wrap_once(x0 - H + hl, nx);
        slot_col = hl;
    } else {
        x = wrap_once(xe + (min(hl, 2 * H - 1) - H), nx);
        slot_col = ncol + H + (min(hl, 2 * H - 1) - H);
    }
    const bool collides = interior && active;
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;

    const T rho0 = p.rho0;
    const uint32_t step = step_of(p);   // the noise counter of this step

    // what a row keeps for its collision H rows later: the nine pulled
    // populations, or on the unit-relaxation path only (sum for the sample,
    // mass, momentum x, momentum y), which that collision reads
    constexpr int NQ = UNIT ? 4 : 9;
    T q[H + 1][NQ];   // rows yy-H .. yy
#pragma unroll
    for (int r = 0; r <= H; ++r)
#pragma unroll
        for (int i = 0; i < NQ; ++i) q[r][i] = T(0);

    const int it_end = (y1 - y0) + 2 * H;
    // Register prefetch: the loads of row it+1 are issued before row it is
    // collided, so they are in flight during the collision arithmetic.
    T gn[9];
    {
        const int yc = wrap_once(y0 - H, ny);
        const int ym = yc == 0 ? ny - 1 : yc - 1;
        const int yp = yc == ny - 1 ? 0 : yc + 1;
        if (active) pull<CG>(p.src, plane, nx, x, xm, xp, yc, ym, yp, gn);
    }
#pragma unroll 2
    for (int it = 0; it < it_end; ++it) {
        const int slot = it & (RING - 1);
        T g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = gn[i];
        if (it + 1 < it_end && active) {
            const int yc = wrap_once(y0 - H + it + 1, ny);
            const int ym = yc == 0 ? ny - 1 : yc - 1;
            const int yp = yc == ny - 1 ? 0 : yc + 1;
            pull<CG>(p.src, plane, nx, x, xm, xp, yc, ym, yp, gn);
        }
        const int yy = y0 - H + it;
        const T s9 = sum9(g);
        if (active)
            s_dpsi[slot][slot_col] = delta_psi<T>(s9, p.psi_kind, rho0, p.psi_c, p.psi_b);
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
        if (it < 2 * H || !collides) continue;

        // ---- collide row yr = yy - H ------------------------------------
        const int yr = yy - H;
        const int cslot = (it - H) & (RING - 1);

        // Shan-Chen force, Eq. (1), as antisymmetric pairs so that a uniform
        // psi gives exactly zero: sum_a w_a psi(x+e_a) e_a over the full set
        // equals sum over half pairs of w_a [dpsi(x+e_a) - dpsi(x-e_a)] e_a.
        T sx = T(0), sy = T(0);
#pragma unroll
        for (int a = 0; a < S::N; ++a) {
            const HalfVec hv = S::v(a);
            const T dpl = s_dpsi[(it - H + hv.ey) & (RING - 1)][tx + H + hv.ex];
            const T dmi = s_dpsi[(it - H - hv.ey) & (RING - 1)][tx + H - hv.ex];
            const T d = T(hv.w) * (dpl - dmi);
            if (hv.ex != 0) sx += T(hv.ex) * d;
            if (hv.ey != 0) sy += T(hv.ey) * d;
        }
        const T psic = p.psi0 + s_dpsi[cslot][tx + H];
        const T Fx = p.force_pref * psic * sx;
        const T Fy = p.force_pref * psic * sy;

        T f[9];
        const uint32_t site = (uint32_t)x + (uint32_t)nx * (uint32_t)yr;
        if constexpr (UNIT) collide_unit_m(q[0][1], q[0][2], q[0][3], Fx, Fy, p, rk, site, step, f);
        else collide<T, false>(q[0], Fx, Fy, p, rk, site, step, f);

        const uint32_t o = (uint32_t)yr * nx + x, pl = (uint32_t)plane;
        p.dst[o] = f[0];
        p.dst[o + pl] = f[1];
        p.dst[o + 2u * pl] = f[2];
        p.dst[o + 3u * pl] = f[3];
        p.dst[o + 4u * pl] = f[4];
        p.dst[o + 5u * pl] = f[5];
        p.dst[o + 6u * pl] = f[6];
        p.dst[o + 7u * pl] = f[7];
        p.dst[o + 8u * pl] = f[8];
        if (SAMPLE) {
            if constexpr (UNIT) p.drho_out[o] = q[0][0];
            else p.drho_out[o] = sum9(q[0]);
        }
        if (!isfinite(f[1] + f[5])) atomicOr(p.flag, LB_STEP_NONFINITE);
    }
}

// Columns per CTA of the overlapped layout: a CTA of kStepTX threads owns
// kStepTX - 2H interior columns and recomputes the pseudopotential of the H
// halo columns on each side itself (each of its threads pulls one column),
// so no warp is set aside for the halo and every warp does the same work up
// to the row barrier.
template <int ORDER> __host__ __device__ constexpr int ov_cols() {
    return kStepTX - 2 * Stencil<ORDER>::H;
}

// One CTA's work in the overlapped layout: interior columns [xs, xs + ncol),
// ncol = min(ov_cols, nx - xs), rows [y0, y1).  Thread t handles column
// xs - H + t (periodic); threads H .. H + ncol - 1 collide.  Same arithmetic,
// same bits as step_strip.
template <typename T, int ORDER, bool SAMPLE, bool CG = false, bool UNIT = false>
__device__ __forceinline__ void step_strip_ov(const KParams<T> &p,
                                              const uint32_t *__restrict__ rk, int xs, int y0,
                                              int y1) {
    using S = Stencil<ORDER>;
    constexpr int H = S::H;
    constexpr int RING = (H == 1) ? 4 : 8;   // >= 2H + 2 rows, power of two
    __shared__ T s_dpsi[RING][kStepTX];

    const int nx = p.nx, ny = p.ny;
    const size_t plane = (size_t)nx * ny;
    const int tx = threadIdx.x;
    const int ncol = min(ov_cols<ORDER>(), nx - xs);
    const bool active = tx < ncol + 2 * H;
    const bool collides = tx >= H && tx < H + ncol;
    const int x = active ? wrap_once(xs - H + tx, nx) : 0;
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;

    const T rho0 = p.rho0;
    const uint32_t step = step_of(p);   // the noise counter of this step

    // what a row keeps for its collision H rows later: the nine pulled
    // populations, or on the unit-relaxation path only (sum for the sample,
    // mass, momentum x, momentum y), which that collision reads
    constexpr int NQ = UNIT ? 4 : 9;
    T q[H + 1][NQ];   // rows yy-H .. yy
#pragma unroll
    for (int r = 0; r <= H; ++r)
#pragma unroll
        for (int i = 0; i < NQ; ++i) q[r][i] = T(0);

    const int it_end = (y1 - y0) + 2 * H;
    T gn[9];
    {
        const int yc = wrap_once(y0 - H, ny);
        const int ym = yc == 0 ? ny - 1 : yc - 1;
        const int yp = yc == ny - 1 ? 0 : yc + 1;
        if (active) pull<CG>(p.src, plane, nx, x, xm, xp, yc, ym, yp, gn);
    }
#pragma unroll 2
    for (int it = 0; it < it_end; ++it) {
        const int slot = it & (RING - 1);
        T g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = gn[i];
        if (it + 1 < it_end && active) {
            const int yc = wrap_once(y0 - H + it + 1, ny);
            const int ym = yc == 0 ? ny - 1 : yc - 1;
            const int yp = yc == ny - 1 ? 0 : yc + 1;
            pull<CG>(p.src, plane, nx, x, xm, xp, yc, ym, yp, gn);
        }
        const int yy = y0 - H + it;
        const T s9 = sum9(g);
        if (active) s_dpsi[slot][tx] = delta_psi<T>(s9, p.psi_kind, rho0, p.psi_c, p.psi_b);
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
        if (it < 2 * H || !collides) continue;

        const int yr = yy - H;
        const int cslot = (it - H) & (RING - 1);
        T sx = T(0), sy = T(0);
#pragma unroll
        for (int a = 0; a < S::N; ++a) {
            const HalfVec hv = S::v(a);
            const T dpl = s_dpsi[(it - H + hv.ey) & (RING - 1)][tx + hv.ex];
            const T dmi = s_dpsi[(it - H - hv.ey) & (RING - 1)][tx - hv.ex];
            const T d = T(hv.w) * (dpl - dmi);
            if (hv.ex != 0) sx += T(hv.ex) * d;
            if (hv.ey != 0) sy += T(hv.ey) * d;
        }
        const T psic = p.psi0 + s_dpsi[cslot][tx];
        const T Fx = p.force_pref * psic * sx;
        const T Fy = p.force_pref * psic * sy;

        T f[9];
        const uint32_t site = (uint32_t)x + (uint32_t)nx * (uint32_t)yr;
        if constexpr (UNIT) collide_unit_m(q[0][1], q[0][2], q[0][3], Fx, Fy, p, rk, site, step, f);
        else collide<T, false>(q[0], Fx, Fy, p, rk, site, step, f);

        const uint32_t o = (uint32_t)yr * nx + x, pl = (uint32_t)plane;
        p.dst[o] = f[0];
        p.dst[o + pl] = f[1];
        p.dst[o + 2u * pl] = f[2];
        p.dst[o + 3u * pl] = f[3];
        p.dst[o + 4u * pl] = f[4];
        p.dst[o + 5u * pl] = f[5];
        p.dst[o + 6u * pl] = f[6];
        p.dst[o + 7u * pl] = f[7];
        p.dst[o + 8u * pl] = f[8];
        if (SAMPLE) {
            if constexpr (UNIT) p.drho_out[o] = q[0][0];
            else p.drho_out[o] = sum9(q[0]);
        }
        if (!isfinite(f[1] + f[5])) atomicOr(p.flag, LB_STEP_NONFINITE);
    }
}

}  // namespace lbsc
