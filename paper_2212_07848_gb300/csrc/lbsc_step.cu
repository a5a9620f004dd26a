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
// Work decomposition: a CTA owns a strip of kStepTX columns and sweeps
// strip_h rows downwards.  Each iteration pulls one new row (one thread per
// column, plus 2H threads for the halo columns), writes the pseudopotential
// deviation of that row into a shared-memory ring of rows, and collides the
// row H above it, whose 2H+1 pseudopotential rows are then complete.  The
// pulled populations of the last H+1 rows stay in registers, so every
// population is read from DRAM once per step (halo rows and columns are
// re-read from L2 only at strip boundaries).
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbsc_device.cuh"
#include "lbsc_internal.cuh"

namespace lbsc {

template <typename T> struct KParams {
    const T *__restrict__ src;
    T *__restrict__ dst;
    T *__restrict__ drho_out;
    int *__restrict__ flag;
    int nx, ny, strip_h, psi_kind, noise;
    uint32_t step, replica;
    T rho0, force_pref, psi_c, psi_b, psi0, gamma, src_scale;
    T amp[6];
    uint32_t rk[20];
};

__device__ __forceinline__ int wrap_once(int a, int n) {
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

// Pull streaming of one site: g_i(x) = f*_i(x - c_i).
template <typename T>
__device__ __forceinline__ void pull(const T *__restrict__ src, size_t plane, int nx, int xc,
                                     int xm, int xp, int yc, int ym, int yp, T g[9]) {
    const size_t rc = (size_t)yc * nx, rm = (size_t)ym * nx, rp = (size_t)yp * nx;
    g[0] = __ldg(src + 0 * plane + rc + xc);
    g[1] = __ldg(src + 1 * plane + rc + xm);   // c = ( 1, 0)
    g[2] = __ldg(src + 2 * plane + rm + xc);   // c = ( 0, 1)
    g[3] = __ldg(src + 3 * plane + rc + xp);   // c = (-1, 0)
    g[4] = __ldg(src + 4 * plane + rp + xc);   // c = ( 0,-1)
    g[5] = __ldg(src + 5 * plane + rm + xm);   // c = ( 1, 1)
    g[6] = __ldg(src + 6 * plane + rm + xp);   // c = (-1, 1)
    g[7] = __ldg(src + 7 * plane + rp + xp);   // c = (-1,-1)
    g[8] = __ldg(src + 8 * plane + rp + xm);   // c = ( 1,-1)
}

// 1/rho and sqrt(rho) from one reciprocal square root (FP32); FP64 keeps the
// correctly rounded operations.
__device__ __forceinline__ void inv_and_sqrt(float rho, float &inv, float &sr) {
    const float r = rsqrtf(rho);
    inv = r * r;
    sr = rho * r;
}
__device__ __forceinline__ void inv_and_sqrt(double rho, double &inv, double &sr) {
    inv = 1.0 / rho;
    sr = sqrt(rho);
}

template <typename T>
__device__ __forceinline__ T sum9(const T g[9]) {
    return ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
}

template <typename T, int ORDER, bool SAMPLE>
__global__ void __launch_bounds__(kStepTX) step_kernel(const KParams<T> p) {
    using S = Stencil<ORDER>;
    constexpr int H = S::H;
    constexpr int RING = (H == 1) ? 4 : 8;   // >= 2H + 2 rows, power of two
    constexpr int W = kStepTX + 2 * H;
    __shared__ T s_dpsi[RING][W];

    const int nx = p.nx, ny = p.ny;
    const size_t plane = (size_t)nx * ny;
    const int tx = threadIdx.x;
    const int x0 = blockIdx.x * kStepTX;
    const int xe = min(x0 + kStepTX, nx);
    const int ncol = xe - x0;
    const bool active = tx < ncol;
    const int x = active ? x0 + tx : x0;
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;

    // Threads 0..2H-1 also own one halo column each (left, then right).
    const bool halo = tx < 2 * H;
    int hcol = 0, hslot = 0;
    if (tx < H) {
        hcol = wrap_once(x0 - H + tx, nx);
        hslot = tx;
    } else {
        hcol = wrap_once(xe + (tx - H), nx);
        hslot = ncol + H + (tx - H);
    }
    const int hxm = hcol == 0 ? nx - 1 : hcol - 1;
    const int hxp = hcol == nx - 1 ? 0 : hcol + 1;

    const int y0 = blockIdx.y * p.strip_h;
    const int y1 = min(y0 + p.strip_h, ny);
    const T rho0 = p.rho0;

    T q[H + 1][9];   // pulled populations of rows yy-H .. yy
#pragma unroll
    for (int r = 0; r <= H; ++r)
#pragma unroll
        for (int i = 0; i < 9; ++i) q[r][i] = T(0);

    const int it_end = (y1 - y0) + 2 * H;
    // Register prefetch: the loads of row it+1 are issued before row it is
    // collided, so they are in flight during the collision arithmetic.
    T gn[9], ghn[9];
    {
        const int yc = wrap_once(y0 - H, ny);
        const int ym = yc == 0 ? ny - 1 : yc - 1;
        const int yp = yc == ny - 1 ? 0 : yc + 1;
        if (active) pull(p.src, plane, nx, x, xm, xp, yc, ym, yp, gn);
        if (halo) pull(p.src, plane, nx, hcol, hxm, hxp, yc, ym, yp, ghn);
    }
    for (int it = 0; it < it_end; ++it) {
        const int slot = it & (RING - 1);
        T g[9], gh[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            g[i] = gn[i];
            gh[i] = ghn[i];
        }
        if (it + 1 < it_end) {
            const int yc = wrap_once(y0 - H + it + 1, ny);
            const int ym = yc == 0 ? ny - 1 : yc - 1;
            const int yp = yc == ny - 1 ? 0 : yc + 1;
            if (active) pull(p.src, plane, nx, x, xm, xp, yc, ym, yp, gn);
            if (halo) pull(p.src, plane, nx, hcol, hxm, hxp, yc, ym, yp, ghn);
        }
        const int yy = y0 - H + it;
        if (active)
            s_dpsi[slot][tx + H] = delta_psi<T>(sum9(g), p.psi_kind, rho0, p.psi_c, p.psi_b);
        if (halo)
            s_dpsi[slot][hslot] = delta_psi<T>(sum9(gh), p.psi_kind, rho0, p.psi_c, p.psi_b);
#pragma unroll
        for (int r = 0; r < H; ++r)
#pragma unroll
            for (int i = 0; i < 9; ++i) q[r][i] = q[r + 1][i];
        if (active) {
#pragma unroll
            for (int i = 0; i < 9; ++i) q[H][i] = g[i];
        }
        __syncthreads();
        if (it < 2 * H || !active) continue;

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

        const T *gq = q[0];
        const T g0 = gq[0], g1 = gq[1], g2 = gq[2], g3 = gq[3], g4 = gq[4];
        const T g5 = gq[5], g6 = gq[6], g7 = gq[7], g8 = gq[8];

        // Hermite moments of the deviations (integer-coefficient transform).
        const T sa = (g1 + g3) + (g2 + g4);
        const T sd = (g5 + g7) + (g6 + g8);
        const T drho = g0 + sa + sd;
        const T m1 = (g1 - g3) + (g5 - g7) + (g8 - g6);
        const T m2 = (g2 - g4) + (g5 - g7) + (g6 - g8);
        const T m3 = T(-2) * g0 + sa + T(4) * sd;
        const T m4 = (g1 + g3) - (g2 + g4);
        const T m5 = (g5 + g7) - (g6 + g8);
        const T m6 = (g3 - g1) + T(2) * ((g5 - g7) + (g8 - g6));
        const T m7 = (g4 - g2) + T(2) * ((g5 - g7) + (g6 - g8));
        const T m8 = T(2) * g0 - T(4) * sa + T(8) * sd;

        // Guo forcing: u = (j + F/2) / rho; post-collision momentum j + F.
        const T rho = rho0 + drho;
        T inv_rho, sr;
        inv_and_sqrt(rho, inv_rho, sr);
        const T ux = (m1 + T(0.5) * Fx) * inv_rho;
        const T uy = (m2 + T(0.5) * Fy) * inv_rho;
        const T gam = p.gamma, hs = p.src_scale;
        const T eq3 = T(3) * rho * (ux * ux + uy * uy);
        const T eq4 = rho * (ux * ux - uy * uy);
        const T eq5 = rho * ux * uy;
        const T S3 = T(6) * (ux * Fx + uy * Fy);
        const T S4 = T(2) * (ux * Fx - uy * Fy);
        const T S5 = ux * Fy + uy * Fx;
        T m3s = eq3 + gam * (m3 - eq3) + hs * S3;
        T m4s = eq4 + gam * (m4 - eq4) + hs * S4;
        T m5s = eq5 + gam * (m5 - eq5) + hs * S5;
        T m6s = gam * m6, m7s = gam * m7, m8s = gam * m8;

        if (p.noise) {
            const uint32_t site = (uint32_t)x + (uint32_t)nx * (uint32_t)yr;
            const uint4 r0 = philox4x32_10(make_uint4(site, p.step, p.replica, 0u), p.rk);
            const uint4 r1 = philox4x32_10(make_uint4(site, p.step, p.replica, 1u), p.rk);
            T z3, z4, z5, z6, z7, z8;
            box_muller(uniform01<T>(r0.x), uniform01<T>(r0.y), z3, z4);
            box_muller(uniform01<T>(r0.z), uniform01<T>(r0.w), z5, z6);
            box_muller(uniform01<T>(r1.x), uniform01<T>(r1.y), z7, z8);
            m3s += p.amp[0] * sr * z3;
            m4s += p.amp[1] * sr * z4;
            m5s += p.amp[2] * sr * z5;
            m6s += p.amp[3] * sr * z6;
            m7s += p.amp[4] * sr * z7;
            m8s += p.amp[5] * sr * z8;
        }

        // Inverse transform: delta f_i = w_i sum_k e_ki m_k / b_k.
        const T a0 = drho, a1 = T(3) * (m1 + Fx), a2 = T(3) * (m2 + Fy);
        const T a3 = T(0.25) * m3s, a4 = T(2.25) * m4s, a5 = T(9) * m5s;
        const T a6 = T(1.5) * m6s, a7 = T(1.5) * m7s, a8 = T(0.0625) * m8s;
        const T b0 = a0 + a3 - T(4) * a8;
        const T d0 = a0 + T(4) * a3 + T(8) * a8;
        const T w0 = T(4.0 / 9.0), w1 = T(1.0 / 9.0), w2 = T(1.0 / 36.0);
        const T f0 = w0 * (a0 - T(2) * a3 + T(2) * a8);
        const T f1 = w1 * (b0 + a1 + a4 - a6);
        const T f2 = w1 * (b0 + a2 - a4 - a7);
        const T f3 = w1 * (b0 - a1 + a4 + a6);
        const T f4 = w1 * (b0 - a2 - a4 + a7);
        const T f5 = w2 * (d0 + a1 + a2 + a5 + T(2) * (a6 + a7));
        const T f6 = w2 * (d0 - a1 + a2 - a5 + T(2) * (a7 - a6));
        const T f7 = w2 * (d0 - a1 - a2 + a5 - T(2) * (a6 + a7));
        const T f8 = w2 * (d0 + a1 - a2 - a5 + T(2) * (a6 - a7));

        T *__restrict__ o = p.dst + (size_t)yr * nx + x;
        o[0 * plane] = f0;
        o[1 * plane] = f1;
        o[2 * plane] = f2;
        o[3 * plane] = f3;
        o[4 * plane] = f4;
        o[5 * plane] = f5;
        o[6 * plane] = f6;
        o[7 * plane] = f7;
        o[8 * plane] = f8;
        if (SAMPLE) p.drho_out[(size_t)yr * nx + x] = drho;
        if (!isfinite(f1 + f5)) *p.flag = 1;
    }
}

template <typename T>
static KParams<T> make_params(const StepArgs &a) {
    KParams<T> k;
    k.src = (const T *)a.src;
    k.dst = (T *)a.dst;
    k.drho_out = (T *)a.drho_out;
    k.flag = a.flag;
    k.nx = a.nx;
    k.ny = a.ny;
    k.strip_h = a.strip_h;
    k.psi_kind = (int)a.psi_kind;
    k.noise = a.noise;
    k.step = a.step;
    k.replica = a.replica;
    k.rho0 = (T)a.rho0;
    k.force_pref = (T)a.force_pref;
    k.psi_c = (T)a.psi_c;
    k.psi_b = (T)a.psi_b;
    k.psi0 = (T)a.psi0;
    k.gamma = (T)a.gamma;
    k.src_scale = (T)a.src_scale;
    for (int i = 0; i < 6; ++i) k.amp[i] = (T)a.noise_amp[i];
    for (int i = 0; i < 20; ++i) k.rk[i] = a.round_keys[i];
    return k;
}

template <typename T, int ORDER>
static cudaError_t launch_t(const StepArgs &a, cudaStream_t s) {
    KParams<T> k = make_params<T>(a);
    dim3 grid((a.nx + kStepTX - 1) / kStepTX, (a.ny + a.strip_h - 1) / a.strip_h);
    if (a.drho_out)
        step_kernel<T, ORDER, true><<<grid, kStepTX, 0, s>>>(k);
    else
        step_kernel<T, ORDER, false><<<grid, kStepTX, 0, s>>>(k);
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
