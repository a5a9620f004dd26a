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
// column, plus one extra warp for the 2H halo columns), writes the pseudopotential
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
    T rho0, force_pref, psi_c, psi_b, psi0, gamma;
    T c3a, c3b, c4a, c4b, c5a, c5b;   // folded relaxation/source constants
    T amp[6];
    uint32_t rk[20];
};

__device__ __forceinline__ int wrap_once(int a, int n) {
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

// Pull streaming of one site: g_i(x) = f*_i(x - c_i).  32-bit element
// indices (the context requires 9 nx ny < 2^32).
template <typename T>
__device__ __forceinline__ void pull(const T *__restrict__ src, size_t plane_, int nx, int xc,
                                     int xm, int xp, int yc, int ym, int yp, T g[9]) {
    const uint32_t plane = (uint32_t)plane_;
    const uint32_t rc = (uint32_t)yc * nx, rm = (uint32_t)ym * nx, rp = (uint32_t)yp * nx;
    g[0] = __ldg(src + (0u * plane + rc + xc));
    g[1] = __ldg(src + (1u * plane + rc + xm));
    g[2] = __ldg(src + (2u * plane + rm + xc));
    g[3] = __ldg(src + (3u * plane + rc + xp));
    g[4] = __ldg(src + (4u * plane + rp + xc));
    g[5] = __ldg(src + (5u * plane + rm + xm));
    g[6] = __ldg(src + (6u * plane + rm + xp));
    g[7] = __ldg(src + (7u * plane + rp + xp));
    g[8] = __ldg(src + (8u * plane + rp + xm));
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

// Collision of one site in the Hermite moment basis, Eq. (12):
// moments of the pulled deviations g -> Guo velocity u = (j + F/2)/rho ->
// BGK relaxation of the stress modes towards rho u u with the Guo source
// (1 - 1/2tau)(u F + F u), ghost modes relaxed towards zero, momentum j + F
// -> noise sqrt(mu rho b_k (1 - gamma^2)) z_k on modes 3..8 -> inverse
// transform delta f_i = w_i sum_k e_ki m_k / b_k.  The inverse is factored
// into symmetric sums and differences with the weights folded in.
template <typename T>
__device__ __forceinline__ void collide(const T g[9], T Fx, T Fy, const KParams<T> &p,
                                        uint32_t site, T f[9]) {
    // forward transform (integer coefficients, shared subexpressions)
    const T e13 = g[1] - g[3], e24 = g[2] - g[4];
    const T s13 = g[1] + g[3], s24 = g[2] + g[4];
    const T d57 = g[5] - g[7], d86 = g[8] - g[6];
    const T s57 = g[5] + g[7], s68 = g[6] + g[8];
    const T sa = s13 + s24, sd = s57 + s68;
    const T drho = g[0] + (sa + sd);
    const T t1 = d57 + d86, t2 = d57 - d86;
    const T m1 = e13 + t1;                                   // j_x
    const T m2 = e24 + t2;                                   // j_y
    const T m3 = fma(T(4), sd, fma(T(-2), g[0], sa));        // 3c^2 - 2
    const T m4 = s13 - s24;                                  // cx^2 - cy^2
    const T m5 = s57 - s68;                                  // cx cy
    const T m6 = fma(T(2), t1, -e13);                        // (3c^2 - 4) cx
    const T m7 = fma(T(2), t2, -e24);                        // (3c^2 - 4) cy
    const T m8 = fma(T(8), sd, fma(T(-4), sa, g[0] + g[0])); // 9c^4 - 15c^2 + 2

    T inv_rho, sr;
    inv_and_sqrt(p.rho0 + drho, inv_rho, sr);
    const T jxh = fma(T(0.5), Fx, m1), jyh = fma(T(0.5), Fy, m2);   // rho u
    const T ux = jxh * inv_rho, uy = jyh * inv_rho;
    const T qxx = jxh * ux, qyy = jyh * uy, qxy = jxh * uy;          // rho u u
    const T pxx = ux * Fx, pyy = uy * Fy, pxy = fma(ux, Fy, uy * Fx);
    const T gam = p.gamma;
    T m3s = fma(gam, m3, fma(p.c3a, qxx + qyy, p.c3b * (pxx + pyy)));
    T m4s = fma(gam, m4, fma(p.c4a, qxx - qyy, p.c4b * (pxx - pyy)));
    T m5s = fma(gam, m5, fma(p.c5a, qxy, p.c5b * pxy));
    T m6s = gam * m6, m7s = gam * m7, m8s = gam * m8;
    const T jxs = m1 + Fx, jys = m2 + Fy;

    if (p.noise) {
        const uint4 r0 = philox4x32_10(make_uint4(site, p.step, p.replica, 0u), p.rk);
        const uint4 r1 = philox4x32_10(make_uint4(site, p.step, p.replica, 1u), p.rk);
        T c, sn, rad;
        box_muller_polar(uniform01<T>(r0.x), uniform01<T>(r0.y), rad, c, sn);
        rad *= sr;
        m3s = fma(p.amp[0] * rad, c, m3s);
        m4s = fma(p.amp[1] * rad, sn, m4s);
        box_muller_polar(uniform01<T>(r0.z), uniform01<T>(r0.w), rad, c, sn);
        rad *= sr;
        m5s = fma(p.amp[2] * rad, c, m5s);
        m6s = fma(p.amp[3] * rad, sn, m6s);
        box_muller_polar(uniform01<T>(r1.x), uniform01<T>(r1.y), rad, c, sn);
        rad *= sr;
        m7s = fma(p.amp[4] * rad, c, m7s);
        m8s = fma(p.amp[5] * rad, sn, m8s);
    }

    // inverse transform
    f[0] = fma(T(1.0 / 18.0), m8s, fma(T(-2.0 / 9.0), m3s, T(4.0 / 9.0) * drho));
    const T B = fma(T(1.0 / 36.0), m3s - m8s, T(1.0 / 9.0) * drho);
    const T P = fma(T(0.25), m4s, B), R = fma(T(-0.25), m4s, B);
    const T Q = fma(T(-1.0 / 6.0), m6s, T(1.0 / 3.0) * jxs);
    const T Sq = fma(T(-1.0 / 6.0), m7s, T(1.0 / 3.0) * jys);
    f[1] = P + Q;
    f[3] = P - Q;
    f[2] = R + Sq;
    f[4] = R - Sq;
    const T D = fma(T(1.0 / 72.0), m8s, T(1.0 / 36.0) * (drho + m3s));
    const T U = fma(T(0.25), m5s, D), V = fma(T(-0.25), m5s, D);
    const T A = T(1.0 / 12.0) * (jxs + m6s), Bd = T(1.0 / 12.0) * (jys + m7s);
    const T X = A + Bd, Y = A - Bd;
    f[5] = U + X;
    f[7] = U - X;
    f[6] = V - Y;
    f[8] = V + Y;
}

template <typename T, int ORDER, bool SAMPLE>
__global__ void __launch_bounds__(kStepTX + 32) step_kernel(const KParams<T> p) {
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
    T gn[9];
    {
        const int yc = wrap_once(y0 - H, ny);
        const int ym = yc == 0 ? ny - 1 : yc - 1;
        const int yp = yc == ny - 1 ? 0 : yc + 1;
        if (active) pull(p.src, plane, nx, x, xm, xp, yc, ym, yp, gn);
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
            pull(p.src, plane, nx, x, xm, xp, yc, ym, yp, gn);
        }
        const int yy = y0 - H + it;
        if (active)
            s_dpsi[slot][slot_col] = delta_psi<T>(sum9(g), p.psi_kind, rho0, p.psi_c, p.psi_b);
#pragma unroll
        for (int r = 0; r < H; ++r)
#pragma unroll
            for (int i = 0; i < 9; ++i) q[r][i] = q[r + 1][i];
#pragma unroll
        for (int i = 0; i < 9; ++i) q[H][i] = g[i];
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
        collide(q[0], Fx, Fy, p, (uint32_t)x + (uint32_t)nx * (uint32_t)yr, f);

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
        if (SAMPLE) p.drho_out[o] = sum9(q[0]);
        if (!isfinite(f[1] + f[5])) *p.flag = 1;
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
    // m3: (1-gamma) * 3 rho u^2 + hs * 6 u.F ; m4: (1-gamma) rho (ux^2-uy^2) + hs * 2 (uxFx-uyFy)
    // m5: (1-gamma) rho ux uy + hs (ux Fy + uy Fx), hs = 1 - 1/(2 tau)
    k.c3a = (T)(3.0 * (1.0 - a.gamma));
    k.c3b = (T)(6.0 * a.src_scale);
    k.c4a = (T)(1.0 - a.gamma);
    k.c4b = (T)(2.0 * a.src_scale);
    k.c5a = (T)(1.0 - a.gamma);
    k.c5b = (T)a.src_scale;
    for (int i = 0; i < 6; ++i) k.amp[i] = (T)a.noise_amp[i];
    for (int i = 0; i < 20; ++i) k.rk[i] = a.round_keys[i];
    return k;
}

template <typename T, int ORDER>
static cudaError_t launch_t(const StepArgs &a, cudaStream_t s) {
    KParams<T> k = make_params<T>(a);
    dim3 grid((a.nx + kStepTX - 1) / kStepTX, (a.ny + a.strip_h - 1) / a.strip_h);
    if (a.drho_out)
        step_kernel<T, ORDER, true><<<grid, kStepTX + 32, 0, s>>>(k);
    else
        step_kernel<T, ORDER, false><<<grid, kStepTX + 32, 0, s>>>(k);
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
