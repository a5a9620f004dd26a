// Device helpers of the fused D2Q9 step: counter-based random numbers, the
// pseudopotential deviation, and the force-stencil tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbsc {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11).  The ten round keys
// are precomputed on the host (they depend only on the seed), so a round is
// two 32x32->64 multiplies (one wide multiply each gives both halves) and
// two three-input XORs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint32_t *__restrict__ rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1], (uint32_t)p0);
    }
    return c;
}

// Uniform deviates in (0, 1]: (r + 1/2) 2^-32.  FP64 is exact; FP32 rounds r
// to 24 significant bits first (relative error < 2^-24).
template <typename T> __device__ __forceinline__ T uniform01(uint32_t r);
template <> __device__ __forceinline__ float uniform01<float>(uint32_t r) {
    return __fmaf_rn(__uint2float_rn(r), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}
template <> __device__ __forceinline__ double uniform01<double>(uint32_t r) {
    return ((double)r + 0.5) * 2.3283064365386963e-10;
}

// Box-Muller: (u1, u2) -> (sqrt(-2 ln u1) cos 2 pi u2, sqrt(-2 ln u1) sin 2 pi u2).
// FP32 uses the hardware approximations: ln u1 = ln 2 log2 u1, the square root
// as x rsqrt(x), and the angle shifted to 2 pi u2 - pi in [-pi, pi) where the
// fast sine/cosine are accurate (cos(a - pi) = -cos a, sin(a - pi) = -sin a).
// Against the FP64 evaluation of the same two 32-bit words the deviates agree
// to about 1e-6 typically; the worst case (a few 1e-4) is u1 within 2^-24 of
// 1, where the FP32 uniform itself rounds (probability below 1e-7 per pair).
__device__ __forceinline__ void box_muller(float u1, float u2, float &z0, float &z1) {
    const float x = -1.3862943611198906f * __log2f(u1);      // -2 ln u1 >= 0
    const float r = x * rsqrtf(fmaxf(x, 1e-30f));
    float s, c;
    __sincosf(fmaf(6.2831853071795865f, u2, -3.1415926535897932f), &s, &c);
    z0 = -r * c;
    z1 = -r * s;
}
__device__ __forceinline__ void box_muller(double u1, double u2, double &z0, double &z1) {
    double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// Box-Muller on a ring of 1024 angles, the noise draw of the step kernels:
// a radius word gives u1 = (r + 1/2) 2^-32 and a 10-bit index a gives the
// angle th = 2 pi (a + 1/2) / 1024, so that one Philox4x32 call (three radius
// words and three 10-bit fields of the fourth word) yields the six normals of
// a site.  Because the 1024 angles are equally spaced, every moment of
// (cos th, sin th) below order 1024 equals its continuous average, so the pair
// rad (cos th, sin th) has the exact moments of two independent standard
// normals up to that order.  Returned in polar form with the local density
// folded into the radius: rad = sqrt(-2 rho ln u1), (z0, z1) = rad (c, s).
// FP32 uses the same hardware forms as box_muller (angle shifted by -pi, the
// sign folded into rad).
__device__ __forceinline__ void box_ring_polar(float u1, uint32_t a, float rho, float &rad,
                                               float &c, float &s) {
    const float x = (-1.3862943611198906f * rho) * __log2f(u1);   // -2 rho ln u1 >= 0
    rad = -x * rsqrtf(fmaxf(x, 1e-30f));
    __sincosf(fmaf((float)a, 6.1359231515425647e-3f, -3.1385246920140220f), &s, &c);
}
__device__ __forceinline__ void box_ring_polar(double u1, uint32_t a, double rho, double &rad,
                                               double &c, double &s) {
    rad = sqrt(-2.0 * rho * log(u1));
    sincospi(((double)a + 0.5) * (1.0 / 512.0), &s, &c);
}

// e^x - 1.  FP32: the Taylor series through x^7 for |x| <= 1/4 (truncation
// below 2e-9 relative), else the hardware exponential minus one (relative
// error about 1e-6 there, where |e^x - 1| > 0.22).  FP64: the library expm1.
__device__ __forceinline__ float dev_expm1(float x) {
    if (fabsf(x) <= 0.25f) {
        float q = fmaf(x, 1.0f / 5040.0f, 1.0f / 720.0f);
        q = fmaf(x, q, 1.0f / 120.0f);
        q = fmaf(x, q, 1.0f / 24.0f);
        q = fmaf(x, q, 1.0f / 6.0f);
        q = fmaf(x, q, 0.5f);
        q = fmaf(x, q, 1.0f);
        return x * q;
    }
    return __expf(x) - 1.0f;
}
__device__ __forceinline__ double dev_expm1(double x) { return expm1(x); }

// delta psi = psi(rho0 + drho) - psi(rho0), written so that a small drho keeps
// its relative precision:
//   kind 0 (1 - e^-rho):          -e^{-rho0} expm1(-drho)
//   kinds 1, 2 (c e^{-b/rho}):     psi0 expm1(b drho / (rho0 rho))
template <typename T>
__device__ __forceinline__ T delta_psi(T drho, int kind, T rho0, T psi_c, T psi_b) {
    if (kind == 0) return -psi_c * dev_expm1(-drho);
    return psi_c * dev_expm1(psi_b * drho / (rho0 * (rho0 + drho)));
}

// ---------------------------------------------------------------------------
// Half stencils of the isotropic force sets (one vector of each +/- pair),
// weights normalised to sum over the full set of w e_x^2 = 1.
//   E4: |e|^2 = 1 : 1/3,  2 : 1/12
//   E6: |e|^2 = 1 : 4/15, 2 : 1/10, 4 : 1/120
//   E8: |e|^2 = 1 : 4/21, 2 : 4/45, 4 : 1/60, 5 : 2/315, 8 : 1/5040
// ---------------------------------------------------------------------------
struct HalfVec {
    int ex, ey;
    double w;
};

template <int ORDER> struct Stencil;
template <> struct Stencil<4> {
    static constexpr int H = 1;   // reach
    static constexpr int N = 4;
    __device__ static constexpr HalfVec v(int a) {
        return a == 0 ? HalfVec{1, 0, 1.0 / 3.0}
             : a == 1 ? HalfVec{0, 1, 1.0 / 3.0}
             : a == 2 ? HalfVec{1, 1, 1.0 / 12.0}
                      : HalfVec{-1, 1, 1.0 / 12.0};
    }
};
template <> struct Stencil<6> {
    static constexpr int H = 2;
    static constexpr int N = 6;
    __device__ static constexpr HalfVec v(int a) {
        return a == 0 ? HalfVec{1, 0, 4.0 / 15.0}
             : a == 1 ? HalfVec{0, 1, 4.0 / 15.0}
             : a == 2 ? HalfVec{1, 1, 1.0 / 10.0}
             : a == 3 ? HalfVec{-1, 1, 1.0 / 10.0}
             : a == 4 ? HalfVec{2, 0, 1.0 / 120.0}
                      : HalfVec{0, 2, 1.0 / 120.0};
    }
};
template <> struct Stencil<8> {
    static constexpr int H = 2;
    static constexpr int N = 12;
    __device__ static constexpr HalfVec v(int a) {
        return a == 0  ? HalfVec{1, 0, 4.0 / 21.0}
             : a == 1  ? HalfVec{0, 1, 4.0 / 21.0}
             : a == 2  ? HalfVec{1, 1, 4.0 / 45.0}
             : a == 3  ? HalfVec{-1, 1, 4.0 / 45.0}
             : a == 4  ? HalfVec{2, 0, 1.0 / 60.0}
             : a == 5  ? HalfVec{0, 2, 1.0 / 60.0}
             : a == 6  ? HalfVec{2, 1, 2.0 / 315.0}
             : a == 7  ? HalfVec{1, 2, 2.0 / 315.0}
             : a == 8  ? HalfVec{-1, 2, 2.0 / 315.0}
             : a == 9  ? HalfVec{-2, 1, 2.0 / 315.0}
             : a == 10 ? HalfVec{2, 2, 1.0 / 5040.0}
                       : HalfVec{-2, 2, 1.0 / 5040.0};
    }
};

}  // namespace lbsc
