// Per-site arithmetic of the fused D2Q9 step shared by the step kernels:
// kernel parameters, pull streaming from global memory, and the
// moment-space collision with Guo forcing and Philox noise (Eq. (12)).
#pragma once

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
    T rho0, force_pref, psi_c, psi_b, psi0;
    T gamma_b, gamma, gamma_g;        // 1 - 1/tau of the bulk, shear and ghost modes
    T c3a, c3b, c4a, c4b, c5a, c5b;   // folded relaxation/source constants
    T amp[6];
    uint32_t rk[20];
    // when not null, the step counter of the noise is *clock + step (a
    // captured window of steps replays for any starting step)
    const uint32_t *__restrict__ clock;
};

__device__ __forceinline__ int wrap_once(int a, int n) {
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

// Pull streaming of one site: g_i(x) = f*_i(x - c_i).  32-bit element
// indices (the context requires 9 nx ny < 2^32).  CG: load through L2 only
// (ld.global.cg) instead of the read-only path, for kernels in which the
// source buffer was written earlier in the same launch.
template <bool CG = false, typename T>
__device__ __forceinline__ T ldsrc(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return __ldg(p);
}
template <bool CG = false, typename T>
__device__ __forceinline__ void pull(const T *__restrict__ src, size_t plane_, int nx, int xc,
                                     int xm, int xp, int yc, int ym, int yp, T g[9]) {
    const uint32_t plane = (uint32_t)plane_;
    const uint32_t rc = (uint32_t)yc * nx, rm = (uint32_t)ym * nx, rp = (uint32_t)yp * nx;
    g[0] = ldsrc<CG>(src + (0u * plane + rc + xc));
    g[1] = ldsrc<CG>(src + (1u * plane + rc + xm));
    g[2] = ldsrc<CG>(src + (2u * plane + rm + xc));
    g[3] = ldsrc<CG>(src + (3u * plane + rc + xp));
    g[4] = ldsrc<CG>(src + (4u * plane + rp + xc));
    g[5] = ldsrc<CG>(src + (5u * plane + rm + xm));
    g[6] = ldsrc<CG>(src + (6u * plane + rm + xp));
    g[7] = ldsrc<CG>(src + (7u * plane + rp + xp));
    g[8] = ldsrc<CG>(src + (8u * plane + rp + xm));
}

// 1/rho: FP32 from the reciprocal square root squared; FP64 correctly rounded.
__device__ __forceinline__ float inv_rho_of(float rho) {
    const float r = rsqrtf(rho);
    return r * r;
}
__device__ __forceinline__ double inv_rho_of(double rho) { return 1.0 / rho; }

template <typename T>
__device__ __forceinline__ T sum9(const T g[9]) {
    return ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
}

// Collision of one site in the Hermite moment basis, Eq. (12):
// moments of the pulled deviations g -> Guo velocity u = (j + F/2)/rho ->
// relaxation of the stress modes towards rho u u with the Guo source
// (1 - 1/2tau_k)(u F + F u) (BGK when every rate is 1/tau; bulk mode 3,
// shear modes 4-5 and ghosts 6-8 may relax at their own rates), ghost modes
// relaxed towards zero, momentum j + F
// -> noise sqrt(mu rho b_k (1 - gamma^2)) z_k on modes 3..8 (one Philox
// call, Box-Muller on a ring of 1024 angles) -> inverse
// transform delta f_i = w_i sum_k e_ki m_k / b_k.  The inverse is factored
// into symmetric sums and differences with the weights folded in.
// UNIT: every relaxation rate is 1 (tau = tau_bulk = tau_ghost = 1, gamma = 0):
// the non-conserved moments are replaced by their equilibrium, source and
// noise, so m3..m8 of the pulled populations are not needed; the result is
// bit-identical to the general path with gamma = 0.
template <typename T>
__device__ __forceinline__ void collide_tail(T drho, T m1, T m2, T m3, T m4, T m5, T m6, T m7,
                                             T m8, T Fx, T Fy, const KParams<T> &p,
                                             const uint32_t *__restrict__ rk, uint32_t site,
                                             uint32_t step, T f[9], bool unit);

// The step counter of the noise for a kernel launched with params p.
template <typename T>
__device__ __forceinline__ uint32_t step_of(const KParams<T> &p) {
    return p.clock ? p.step + __ldg(p.clock) : p.step;
}

// Mass and momentum deviations of the pulled populations, with exactly the
// arithmetic of the forward transform in collide (so that a kernel may keep
// them instead of the nine populations on the unit-relaxation path).
template <typename T>
__device__ __forceinline__ void unit_moments(const T g[9], T &drho, T &m1, T &m2) {
    const T e13 = g[1] - g[3], e24 = g[2] - g[4];
    const T s13 = g[1] + g[3], s24 = g[2] + g[4];
    const T d57 = g[5] - g[7], d86 = g[8] - g[6];
    const T s57 = g[5] + g[7], s68 = g[6] + g[8];
    const T sa = s13 + s24, sd = s57 + s68;
    drho = g[0] + (sa + sd);
    const T t1 = d57 + d86, t2 = d57 - d86;
    m1 = e13 + t1;
    m2 = e24 + t2;
}

// The unit-relaxation collision from the mass and momentum deviations alone.
template <typename T>
__device__ __forceinline__ void collide_unit_m(T drho, T m1, T m2, T Fx, T Fy, const KParams<T> &p,
                                               const uint32_t *__restrict__ rk, uint32_t site,
                                               uint32_t step, T f[9]) {
    collide_tail<T>(drho, m1, m2, T(0), T(0), T(0), T(0), T(0), T(0), Fx, Fy, p, rk, site, step, f,
                    true);
}

template <typename T, bool UNIT = false>
__device__ __forceinline__ void collide(const T g[9], T Fx, T Fy, const KParams<T> &p,
                                        const uint32_t *__restrict__ rk, uint32_t site,
                                        uint32_t step, T f[9]) {
    if constexpr (UNIT) {
        T drho, m1, m2;
        unit_moments(g, drho, m1, m2);
        collide_unit_m(drho, m1, m2, Fx, Fy, p, rk, site, step, f);
        return;
    }
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
    collide_tail<T>(drho, m1, m2, m3, m4, m5, m6, m7, m8, Fx, Fy, p, rk, site, step, f, false);
}

// Everything after the forward transform: Guo velocity, relaxation with the
// source, noise, inverse transform.  unit: every rate is 1 (m3 .. m8 unused).
template <typename T>
__device__ __forceinline__ void collide_tail(T drho, T m1, T m2, T m3, T m4, T m5, T m6, T m7,
                                             T m8, T Fx, T Fy, const KParams<T> &p,
                                             const uint32_t *__restrict__ rk, uint32_t site,
                                             uint32_t step, T f[9], bool unit) {
    const T rho = p.rho0 + drho;
    const T inv_rho = inv_rho_of(rho);
    const T jxh = fma(T(0.5), Fx, m1), jyh = fma(T(0.5), Fy, m2);   // rho u
    const T ux = jxh * inv_rho, uy = jyh * inv_rho;
    const T qxx = jxh * ux, qyy = jyh * uy, qxy = jxh * uy;          // rho u u
    const T pxx = ux * Fx, pyy = uy * Fy, pxy = fma(ux, Fy, uy * Fx);
    T m3s, m4s, m5s, m6s, m7s, m8s;
    if (unit) {
        m3s = fma(p.c3a, qxx + qyy, p.c3b * (pxx + pyy));
        m4s = fma(p.c4a, qxx - qyy, p.c4b * (pxx - pyy));
        m5s = fma(p.c5a, qxy, p.c5b * pxy);
        m6s = m7s = m8s = T(0);
    } else {
        const T gs = p.gamma, gg = p.gamma_g;
        m3s = fma(p.gamma_b, m3, fma(p.c3a, qxx + qyy, p.c3b * (pxx + pyy)));
        m4s = fma(gs, m4, fma(p.c4a, qxx - qyy, p.c4b * (pxx - pyy)));
        m5s = fma(gs, m5, fma(p.c5a, qxy, p.c5b * pxy));
        m6s = gg * m6;
        m7s = gg * m7;
        m8s = gg * m8;
    }
    const T jxs = m1 + Fx, jys = m2 + Fy;

    if (p.noise) {
        // one Philox call per site and step: radius words r.x, r.y, r.z and
        // three 10-bit angle indices of r.w (bits 0-9, 10-19, 20-29)
        const uint4 r = philox4x32_10(make_uint4(site, step, p.replica, 0u), rk);
        T c, sn, rad;
        box_ring_polar(uniform01<T>(r.x), r.w & 1023u, rho, rad, c, sn);
        m3s = fma(p.amp[0] * rad, c, m3s);
        m4s = fma(p.amp[1] * rad, sn, m4s);
        box_ring_polar(uniform01<T>(r.y), (r.w >> 10) & 1023u, rho, rad, c, sn);
        m5s = fma(p.amp[2] * rad, c, m5s);
        m6s = fma(p.amp[3] * rad, sn, m6s);
        box_ring_polar(uniform01<T>(r.z), (r.w >> 20) & 1023u, rho, rad, c, sn);
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

template <typename T>
inline KParams<T> make_params(const StepArgs &a) {
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
    k.clock = a.clock;
    k.replica = a.replica;
    k.rho0 = (T)a.rho0;
    k.force_pref = (T)a.force_pref;
    k.psi_c = (T)a.psi_c;
    k.psi_b = (T)a.psi_b;
    k.psi0 = (T)a.psi0;
    k.gamma = (T)a.gamma;
    k.gamma_b = (T)a.gamma_b;
    k.gamma_g = (T)a.gamma_g;
    // m3: (1-gb) 3 rho u^2 + hb 6 u.F ; m4: (1-gs) rho (ux^2-uy^2) + hs 2 (uxFx-uyFy)
    // m5: (1-gs) rho ux uy + hs (ux Fy + uy Fx), h = (1 + gamma)/2 = 1 - 1/(2 tau)
    k.c3a = (T)(3.0 * (1.0 - a.gamma_b));
    k.c3b = (T)(3.0 * (1.0 + a.gamma_b));
    k.c4a = (T)(1.0 - a.gamma);
    k.c4b = (T)(1.0 + a.gamma);
    k.c5a = (T)(1.0 - a.gamma);
    k.c5b = (T)(0.5 * (1.0 + a.gamma));
    for (int i = 0; i < 6; ++i) k.amp[i] = (T)a.noise_amp[i];
    for (int i = 0; i < 20; ++i) k.rk[i] = a.round_keys[i];
    return k;
}

}  // namespace lbsc
