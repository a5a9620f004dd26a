// Fluctuating Shan-Chen step in three dimensions (D3Q19): the paper's own
// setting, Eq. (12) with the force of Eq. (1) and noise on the moments
// a > 3 (the noise paragraph after Eq. (16)).  Deviations delta f_i = f_i -
// w_i rho0 are stored structure-of-arrays [19][nz][ny][nx], two buffers.
//
// Work decomposition: a CTA owns a 32 x 4 tile of (x, y) columns and marches
// a strip of z planes.  Its 34 x 6 threads cover the tile and its one-column
// halo ring: every thread pulls its column's populations for plane z + 1 and
// writes that plane's pseudopotential deviation into a shared-memory ring of
// four planes; after the barrier the 32 x 4 interior threads pull plane z
// again (L1 hits: they pulled it one iteration earlier) and collide it.
// The force is Eq. (1) over the 18 D3Q19 neighbours with the fourth-order
// isotropic weights 1/6 (axes) and 1/12 (face diagonals), summed as
// antisymmetric pairs.  The collision runs in the 19-moment basis:
// mass and momentum conserved (momentum + F), the six stress modes relaxed
// to rho u u with the Guo source, the nine ghost modes relaxed to zero, and
// noise sqrt(mu rho b_k (1 - gamma^2)) z_k on the fifteen modes 4..18 from
// two Philox4x32-10 calls (ring Box-Muller, one pair per word).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include <type_traits>

#include "lbsc.h"
#include "lbsc_device.cuh"
#include "lbsc_fft.cuh"
#include "lbsc_internal.cuh"

namespace lbsc {
namespace {

// D3Q19 velocities: rest; +x, -x, +y, -y, +z, -z; xy, xz, yz face diagonals
// as (+,+), (-,-), (+,-), (-,+).  Opposite velocities are adjacent (1-2, ...).
__host__ __device__ constexpr int cx3(int i) {
    return i == 1 || i == 7 || i == 9 || i == 11 || i == 13 ? 1
         : i == 2 || i == 8 || i == 10 || i == 12 || i == 14 ? -1 : 0;
}
__host__ __device__ constexpr int cy3(int i) {
    return i == 3 || i == 7 || i == 10 || i == 15 || i == 17 ? 1
         : i == 4 || i == 8 || i == 9 || i == 16 || i == 18 ? -1 : 0;
}
__host__ __device__ constexpr int cz3(int i) {
    return i == 5 || i == 11 || i == 14 || i == 15 || i == 18 ? 1
         : i == 6 || i == 12 || i == 13 || i == 16 || i == 17 ? -1 : 0;
}
__host__ __device__ constexpr double wq3(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}
// Moment polynomial k at velocity i (integer values).
__host__ __device__ constexpr int mom3(int k, int i) {
    const int x = cx3(i), y = cy3(i), z = cz3(i), c2 = x * x + y * y + z * z;
    return k == 0 ? 1
         : k == 1 ? x : k == 2 ? y : k == 3 ? z
         : k == 4 ? c2 - 1
         : k == 5 ? 3 * x * x - c2
         : k == 6 ? y * y - z * z
         : k == 7 ? x * y : k == 8 ? y * z : k == 9 ? z * x
         : k == 10 ? (3 * c2 - 5) * x : k == 11 ? (3 * c2 - 5) * y : k == 12 ? (3 * c2 - 5) * z
         : k == 13 ? (y * y - z * z) * x : k == 14 ? (z * z - x * x) * y
         : k == 15 ? (x * x - y * y) * z
         : k == 16 ? 3 * c2 * c2 - 6 * c2 + 1
         : k == 17 ? (2 * c2 - 3) * (3 * x * x - c2)
                   : (2 * c2 - 3) * (y * y - z * z);
}
// b_k = sum_i w_i e_ki^2, and the same values written out (checked against
// each other at compile time) for the device code
__host__ __device__ constexpr double norm3(int k) {
    double b = 0.0;
    for (int i = 0; i < 19; ++i) b += wq3(i) * mom3(k, i) * mom3(k, i);
    return b;
}
__host__ __device__ constexpr double norm3_lit(int k) {
    return k == 0 ? 1.0 : k <= 3 ? 1.0 / 3.0 : k == 4 ? 2.0 / 3.0 : k == 5 ? 4.0 / 3.0
         : k == 6 ? 4.0 / 9.0 : k <= 9 ? 1.0 / 9.0 : k <= 12 ? 2.0 / 3.0 : k <= 15 ? 2.0 / 9.0
         : k == 16 ? 2.0 : k == 17 ? 4.0 / 3.0 : 4.0 / 9.0;
}
constexpr bool norms_agree() {
    for (int k = 0; k < 19; ++k) {
        const double d = norm3(k) - norm3_lit(k);
        if (d > 1e-15 || d < -1e-15) return false;
    }
    return true;
}
static_assert(norms_agree(), "moment norms");

// A CTA owns a 32 x TY tile of (x, y) columns plus their one-column halo ring
// (34 x (TY + 2) threads).  Each interior row is one warp, so the collision
// runs on full warps; the ring rows and columns take the remaining threads.
// FP32 uses 32 x 8 tiles (340 threads, 80 registers, two CTAs per SM) when
// ny is a multiple of 8, else 32 x 4 (204 threads, four per SM); FP64 always
// 32 x 4 (two per SM).  Measured at 256^3 FP32 on GB300: 32 x 8 30.1 GLUPS,
// 32 x 4 28.9, 32 x 8 at three CTAs per SM (56 registers, spilling) 26.0,
// 32 x 16 (612 threads, 96 registers, one CTA per SM: a sixth fewer ring
// pulls, but nothing issues while the CTA waits at its plane barrier) 27.8;
// with the rows split across warps (the linear thread order) 32 x 4 ran at
// 24.5.  Prefetching the next plane (into registers at three CTAs per SM, or
// by cp.async into shared memory) measured slower: the step is bound by issue
// and resident warps, not by the loads' latency.
constexpr int kTX3 = 32;
constexpr int kTYMin3 = 4;   // ny must be a multiple of this
static_assert(kTX3 == 32, "one warp per interior row");
template <int TY> constexpr int threads3() { return (kTX3 + 2) * (TY + 2); }

// Thread -> (tx, ty) of the 34 x (TY + 2) block: warps 0 .. TY - 1 are the
// interior rows (ty = 1 .. TY, tx = 1 .. 32); then the two ring rows
// (ty = 0, TY + 1) and the 2 (TY + 2) ring columns (tx = 0, 33).
template <int TY>
__device__ __forceinline__ void ring_xy3(int t, int &tx, int &ty) {
    constexpr int BY = TY + 2;
    if (t < kTX3 * TY) {
        tx = 1 + (t & 31);
        ty = 1 + (t >> 5);
    } else if (t < kTX3 * BY) {
        t -= kTX3 * TY;
        tx = 1 + (t & 31);
        ty = t < kTX3 ? 0 : BY - 1;
    } else {
        t -= kTX3 * BY;
        tx = t < BY ? 0 : kTX3 + 1;
        ty = t < BY ? t : t - BY;
    }
}

template <typename T> struct K3 {
    const T *__restrict__ src;
    T *__restrict__ dst;
    T *__restrict__ drho_out;
    int *__restrict__ flag;
    int nx, ny, nz, strip_z, noise, psi_kind;
    uint32_t step, replica;
    T rho0, force_pref, psi_c, psi_b, psi0, gamma, hsrc;
    T amp[19];     // modes 4..18 used
    uint32_t rk[20];
    const float2 *ring;   // (cos, sin) of the 1024 ring angles 2 pi (a + 1/2) / 1024
};

constexpr int kRing3 = 1024;

// Uniform in (0, 1) from the high 22 bits of a word: ((w >> 10) + 1/2) 2^-22
// (exact in FP32 and FP64).
template <typename T> __device__ __forceinline__ T uniform22(uint32_t w);
template <> __device__ __forceinline__ float uniform22<float>(uint32_t w) {
    return __fmaf_rn(__uint2float_rn(w >> 10), 2.384185791015625e-07f, 1.1920928955078125e-07f);
}
template <> __device__ __forceinline__ double uniform22<double>(uint32_t w) {
    return ((double)(w >> 10) + 0.5) * 2.384185791015625e-07;
}

// One ring Box-Muller pair folded with sqrt(rho): rad = sqrt(-2 rho ln u1),
// (c, s) = (cos, sin) of angle a.  FP32 reads the angle's cosine and sine from
// the table (correctly rounded from FP64) instead of evaluating them; FP64
// evaluates them.
__device__ __forceinline__ void ring_pair3(float u1, uint32_t a, float rho,
                                           const float2 *__restrict__ ring, float &rad, float &c,
                                           float &s) {
    const float x = (-1.3862943611198906f * rho) * __log2f(u1);   // -2 rho ln u1 > 0
    rad = x * rsqrtf(fmaxf(x, 1e-30f));
    const float2 cs = ring[a];
    c = cs.x;
    s = cs.y;
}
__device__ __forceinline__ void ring_pair3(double u1, uint32_t a, double rho, const float2 *,
                                           double &rad, double &c, double &s) {
    box_ring_polar(u1, a, rho, rad, c, s);
}

// Pull of one site from precomputed wrapped offsets: xo[1 + d] = x + d,
// yo[1 + d] = (y + d) nx and zo[1 + d] = (z + d) nx ny for d = -1, 0, 1.
template <typename T>
__device__ __forceinline__ void pull3(const T *__restrict__ src, uint32_t plane,
                                      const uint32_t xo[3], const uint32_t yo[3],
                                      const uint32_t zo[3], T g[19]) {
#pragma unroll
    for (int i = 0; i < 19; ++i)
        g[i] = __ldg(src + ((uint32_t)i * plane + zo[1 - cz3(i)] + yo[1 - cy3(i)] + xo[1 - cx3(i)]));
}

template <typename T>
__device__ __forceinline__ T sum19(const T g[19]) {
    T s = g[0];
#pragma unroll
    for (int p = 0; p < 9; ++p) s += g[2 * p + 1] + g[2 * p + 2];
    return s;
}

// 1/rho: FP32 from the reciprocal square root squared (a few ulp); FP64
// correctly rounded.
__device__ __forceinline__ float inv3(float rho) {
    const float r = rsqrtf(rho);
    return r * r;
}
__device__ __forceinline__ double inv3(double rho) { return 1.0 / rho; }

// Collision of one site (moment space), Eq. (12) in 3D.
// UNIT: every relaxation rate is 1 (gamma = 0): the non-conserved moments of
// the pulled populations are not needed (stress modes become their
// equilibrium plus source, ghosts zero, before the noise); the result is
// that of the general path with gamma = 0.
// Moments m_k = sum_i e_ki g_i of the pulled populations, k < NK (NK = 4:
// mass and momentum only), from pair sums and differences: pair q =
// velocities 2q+1 (c) and 2q+2 (-c); even polynomials use the sums, odd the
// differences.
template <typename T, int NK>
__device__ __forceinline__ void moments3(const T g[19], T *m) {
    T s[10], d[10];
    s[0] = g[0];
    d[0] = T(0);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        s[q + 1] = g[2 * q + 1] + g[2 * q + 2];
        d[q + 1] = g[2 * q + 1] - g[2 * q + 2];
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const bool odd = (k >= 1 && k <= 3) || (k >= 10 && k <= 15);
        T acc = odd ? T(0) : T(mom3(k, 0)) * s[0];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int e = mom3(k, 2 * q + 1);
            if (e != 0) acc = fma(T(e), odd ? d[q + 1] : s[q + 1], acc);
        }
        m[k] = acc;
    }
}

template <typename T, bool UNIT = false>
__device__ __forceinline__ void collide3_m(const T m[19], T Fx, T Fy, T Fz, const K3<T> &p,
                                           uint32_t site, const float2 *ring, T f[19]);

template <typename T, bool UNIT = false>
__device__ __forceinline__ void collide3(const T g[19], T Fx, T Fy, T Fz, const K3<T> &p,
                                         uint32_t site, const float2 *ring, T f[19]) {
    T m[19];
    moments3<T, UNIT ? 4 : 19>(g, m);
    collide3_m<T, UNIT>(m, Fx, Fy, Fz, p, site, ring, f);
}

// The collision from the moments of the pulled populations (UNIT: only
// m_0 .. m_3 are read).
template <typename T, bool UNIT>
__device__ __forceinline__ void collide3_m(const T m[19], T Fx, T Fy, T Fz, const K3<T> &p,
                                           uint32_t site, const float2 *ring, T f[19]) {
    const T rho = p.rho0 + m[0];
    const T inv = inv3(rho);
    const T jx = fma(T(0.5), Fx, m[1]), jy = fma(T(0.5), Fy, m[2]), jz = fma(T(0.5), Fz, m[3]);
    const T ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const T qxx = jx * ux, qyy = jy * uy, qzz = jz * uz;
    const T qxy = jx * uy, qyz = jy * uz, qzx = jz * ux;
    const T q2 = qxx + qyy + qzz;
    const T pxx = ux * Fx, pyy = uy * Fy, pzz = uz * Fz;
    const T p2 = pxx + pyy + pzz;
    const T g_ = p.gamma, a = T(1) - p.gamma, h = p.hsrc;   // h = (1 + gamma) / 2
    T ms[19];
    ms[0] = m[0];
    ms[1] = m[1] + Fx;
    ms[2] = m[2] + Fy;
    ms[3] = m[3] + Fz;
    ms[4] = fma(a, q2, h * (T(2) * p2));
    ms[5] = fma(a, T(3) * qxx - q2, h * (T(6) * pxx - T(2) * p2));
    ms[6] = fma(a, qyy - qzz, h * (T(2) * (pyy - pzz)));
    ms[7] = fma(a, qxy, h * fma(ux, Fy, uy * Fx));
    ms[8] = fma(a, qyz, h * fma(uy, Fz, uz * Fy));
    ms[9] = fma(a, qzx, h * fma(uz, Fx, ux * Fz));
    if constexpr (UNIT) {
#pragma unroll
        for (int k = 10; k < 19; ++k) ms[k] = T(0);
    } else {
#pragma unroll
        for (int k = 4; k < 10; ++k) ms[k] = fma(g_, m[k], ms[k]);
#pragma unroll
        for (int k = 10; k < 19; ++k) ms[k] = g_ * m[k];
    }
    if (p.noise) {
        // two Philox calls, one ring pair per word (radius from the high 22
        // bits, angle index from the low 10): block 0 -> modes 4..11, block 1
        // -> modes 12..17 and 18 (the cosine of its last pair)
        const uint4 r0 = philox4x32_10(make_uint4(site, p.step, p.replica, 0u), p.rk);
        const uint4 r1 = philox4x32_10(make_uint4(site, p.step, p.replica, 1u), p.rk);
        T c, sn, rad;
#define NOISE_PAIR(W, KA, KB)                                                \
    ring_pair3(uniform22<T>(W), (W) & 1023u, rho, ring, rad, c, sn);      \
    ms[KA] = fma(p.amp[KA] * rad, c, ms[KA]);                              \
    ms[KB] = fma(p.amp[KB] * rad, sn, ms[KB]);
        NOISE_PAIR(r0.x, 4, 5)
        NOISE_PAIR(r0.y, 6, 7)
        NOISE_PAIR(r0.z, 8, 9)
        NOISE_PAIR(r0.w, 10, 11)
        NOISE_PAIR(r1.x, 12, 13)
        NOISE_PAIR(r1.y, 14, 15)
        NOISE_PAIR(r1.z, 16, 17)
#undef NOISE_PAIR
        ring_pair3(uniform22<T>(r1.w), r1.w & 1023u, rho, ring, rad, c, sn);
        ms[18] = fma(p.amp[18] * rad, c, ms[18]);
    }
    // inverse: delta f_i = w_i sum_k e_ki m*_k / b_k, assembled per pair as
    // (even part) +- (odd part).  Each part is split so that velocities of the
    // same family share work: the even part is a sum over the modes whose
    // polynomial depends on the squares c_a^2 only (the same for every
    // velocity of a family) plus the cross modes c_a c_b; the odd part is
    // sum_a c_a P_a with P_a over the modes odd in c_a, whose coefficients
    // again depend on the squares only.
    constexpr int kEvenSq[7] = {0, 4, 16, 5, 6, 17, 18};
    constexpr int kCross[3] = {7, 8, 9};
    constexpr int kOddAxis[3][3] = {{1, 10, 13}, {2, 11, 14}, {3, 12, 15}};
    T ev[10], od[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        const int i = q == 0 ? 0 : 2 * q - 1;
        const int ci[3] = {cx3(i), cy3(i), cz3(i)};
        T e_sq = T(0), e_x = T(0);
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const int k = kEvenSq[j], e = mom3(k, i);
            if (e != 0) e_sq = fma(T(wq3(i) * e / norm3_lit(k)), ms[k], e_sq);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int k = kCross[j], e = mom3(k, i);
            if (e != 0) e_x = fma(T(wq3(i) * e / norm3_lit(k)), ms[k], e_x);
        }
        T o = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (ci[a] == 0) continue;
            T pa = T(0);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int k = kOddAxis[a][j], h = mom3(k, i) * ci[a];   // e_k / c_a
                if (h != 0) pa = fma(T(wq3(i) * h / norm3_lit(k)), ms[k], pa);
            }
            o = ci[a] > 0 ? o + pa : o - pa;
        }
        ev[q] = e_sq + e_x;
        od[q] = o;
    }
    f[0] = ev[0];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        f[2 * q + 1] = ev[q + 1] + od[q + 1];
        f[2 * q + 2] = ev[q + 1] - od[q + 1];
    }
}


template <typename T, bool SAMPLE, bool UNIT, int TY>
__global__ void __launch_bounds__(threads3<TY>(), (sizeof(T) == 4 && TY == 4) ? 4 : 2)
step3_kernel(const K3<T> p) {
    constexpr int kBX3 = kTX3 + 2, kBY3 = TY + 2;
    __shared__ T s_psi[4][kBY3][kBX3];   // ring of planes: one barrier per plane suffices
    __shared__ float2 s_ring[kRing3];    // noise angles (FP32 path; read after the first barrier)
    if (std::is_same<T, float>::value && p.noise)
        for (int i = threadIdx.x; i < kRing3; i += blockDim.x) s_ring[i] = p.ring[i];
    int tx, ty;
    ring_xy3<TY>(threadIdx.x, tx, ty);
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const uint32_t plane = (uint32_t)nx * ny * nz;
    int x = blockIdx.x * kTX3 - 1 + tx, y = blockIdx.y * TY - 1 + ty;
    x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    const bool interior = tx >= 1 && tx <= kTX3 && ty >= 1 && ty <= TY;
    const int z0 = blockIdx.z * p.strip_z, z1 = min(z0 + p.strip_z, nz);
    const int it_end = (z1 - z0) + 2;

    // wrapped neighbour offsets of this column (constant along z)
    const uint32_t xo[3] = {(uint32_t)(x == 0 ? nx - 1 : x - 1), (uint32_t)x,
                            (uint32_t)(x == nx - 1 ? 0 : x + 1)};
    const uint32_t yo[3] = {(uint32_t)(y == 0 ? ny - 1 : y - 1) * nx, (uint32_t)y * nx,
                            (uint32_t)(y == ny - 1 ? 0 : y + 1) * nx};
    const uint32_t nxy = (uint32_t)nx * ny;

    uint32_t zprev[3] = {0u, 0u, 0u};   // offsets of the plane pulled one iteration ago
    // UNIT: the collision needs only the mass and momentum of the pulled
    // populations, so they are kept from the pull of the previous iteration
    // (and the density deviation for a sample) instead of pulling again
    T mprev[4] = {T(0), T(0), T(0), T(0)};
    T dprev = T(0);
    for (int it = 0; it < it_end; ++it) {
        int zz = z0 - 1 + it;
        zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
        const uint32_t zo[3] = {(uint32_t)(zz == 0 ? nz - 1 : zz - 1) * nxy, (uint32_t)zz * nxy,
                                (uint32_t)(zz == nz - 1 ? 0 : zz + 1) * nxy};
        T mnew[4] = {T(0), T(0), T(0), T(0)}, dnew = T(0);
        {
            T g[19];
            pull3(p.src, plane, xo, yo, zo, g);
            dnew = sum19(g);
            s_psi[it & 3][ty][tx] = delta_psi<T>(dnew, p.psi_kind, p.rho0, p.psi_c, p.psi_b);
            if (UNIT) moments3<T, 4>(g, mnew);
        }
        __syncthreads();
        if (it >= 2 && interior) {
            // collide plane zc = zz - 1: its populations are pulled again (they
            // were pulled in the previous iteration and come from L1), which
            // keeps 19 values per thread out of the registers
            const int zc = z0 - 2 + it;
            const int sm = (it - 2) & 3, sc = (it - 1) & 3, sp = it & 3;
            // Eq. (1): sum over the 18 neighbours as antisymmetric pairs
            const T w1 = T(1.0 / 6.0), w2 = T(1.0 / 12.0);
            T Sx = w1 * (s_psi[sc][ty][tx + 1] - s_psi[sc][ty][tx - 1]);
            T Sy = w1 * (s_psi[sc][ty + 1][tx] - s_psi[sc][ty - 1][tx]);
            T Sz = w1 * (s_psi[sp][ty][tx] - s_psi[sm][ty][tx]);
            const T dxy1 = s_psi[sc][ty + 1][tx + 1] - s_psi[sc][ty - 1][tx - 1];   // (1,1,0)
            const T dxy2 = s_psi[sc][ty - 1][tx + 1] - s_psi[sc][ty + 1][tx - 1];   // (1,-1,0)
            const T dxz1 = s_psi[sp][ty][tx + 1] - s_psi[sm][ty][tx - 1];           // (1,0,1)
            const T dxz2 = s_psi[sm][ty][tx + 1] - s_psi[sp][ty][tx - 1];           // (1,0,-1)
            const T dyz1 = s_psi[sp][ty + 1][tx] - s_psi[sm][ty - 1][tx];           // (0,1,1)
            const T dyz2 = s_psi[sm][ty + 1][tx] - s_psi[sp][ty - 1][tx];           // (0,1,-1)
            Sx = fma(w2, (dxy1 + dxy2) + (dxz1 + dxz2), Sx);
            Sy = fma(w2, (dxy1 - dxy2) + (dyz1 + dyz2), Sy);
            Sz = fma(w2, (dxz1 - dxz2) + (dyz1 - dyz2), Sz);
            const T psic = p.psi0 + s_psi[sc][ty][tx];
            const T Fx = p.force_pref * psic * Sx, Fy = p.force_pref * psic * Sy,
                    Fz = p.force_pref * psic * Sz;
            const uint32_t site = ((uint32_t)zc * ny + y) * nx + x;
            T f[19];
            if constexpr (UNIT) {
                T m[19];
#pragma unroll
                for (int k = 0; k < 4; ++k) m[k] = mprev[k];
                collide3_m<T, true>(m, Fx, Fy, Fz, p, site, s_ring, f);
                if (SAMPLE) p.drho_out[site] = dprev;
            } else {
                T g[19];
                pull3(p.src, plane, xo, yo, zprev, g);
                collide3<T, false>(g, Fx, Fy, Fz, p, site, s_ring, f);
                if (SAMPLE) p.drho_out[site] = sum19(g);
            }
#pragma unroll
            for (int i = 0; i < 19; ++i) p.dst[(uint32_t)i * plane + site] = f[i];
            if (!isfinite(f[1] + f[7])) atomicOr(p.flag, LB_STEP_NONFINITE);
        }
        zprev[0] = zo[0];
        zprev[1] = zo[1];
        zprev[2] = zo[2];
        if (UNIT) {
#pragma unroll
            for (int k = 0; k < 4; ++k) mprev[k] = mnew[k];
            dprev = dnew;
        }
        // slot (it + 1) & 3, written next, was last read in iteration it - 1,
        // before this iteration's barrier
    }
}

// ---------------------------------------------------------------------------
// Axis structure factor: per z plane the partial x and y profiles of delta
// rho and the plane total; then the profiles are summed over planes in a
// fixed order and Fourier transformed on the x, y and z axes.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void profile3_kernel(const T *__restrict__ drho, int nx, int ny, double *__restrict__ px,
                                double *__restrict__ py, double *__restrict__ pz) {
    // block = one z plane
    const int z = blockIdx.x;
    const T *pl = drho + (size_t)z * nx * ny;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        double s = 0.0;
        for (int y = 0; y < ny; ++y) s += (double)pl[(size_t)y * nx + x];
        px[(size_t)z * nx + x] = s;
    }
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
        double s = 0.0;
        for (int x = 0; x < nx; ++x) s += (double)pl[(size_t)y * nx + x];
        py[(size_t)z * ny + y] = s;
    }
    __shared__ double red[256];
    double s = 0.0;
    for (size_t i = threadIdx.x; i < (size_t)nx * ny; i += blockDim.x) s += (double)pl[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) pz[z] = red[0];
}

// one block: the profiles are summed over planes in a fixed order into
// shared memory, then a thread per axis mode accumulates
// |sum_c p(c) e^{-2 pi i m c / n}|^2 / N.
__global__ void axis_dft3_kernel(const double *__restrict__ px, const double *__restrict__ py,
                                 const double *__restrict__ pz, int nx, int ny, int nz,
                                 double *__restrict__ acc) {
    extern __shared__ double tot[];   // [nx] + [ny] + [nz]
    for (int c = threadIdx.x; c < nx; c += blockDim.x) {
        double v = 0.0;
        for (int z = 0; z < nz; ++z) v += px[(size_t)z * nx + c];
        tot[c] = v;
    }
    for (int c = threadIdx.x; c < ny; c += blockDim.x) {
        double v = 0.0;
        for (int z = 0; z < nz; ++z) v += py[(size_t)z * ny + c];
        tot[nx + c] = v;
    }
    for (int c = threadIdx.x; c < nz; c += blockDim.x) tot[nx + ny + c] = pz[c];
    __syncthreads();
    const int nmodes = nx / 2 + ny / 2 + nz / 2;
    const double N = (double)nx * ny * nz;
    for (int t = threadIdx.x; t < nmodes; t += blockDim.x) {
        int m, n, off;
        if (t < nx / 2) { m = t + 1; n = nx; off = 0; }
        else if (t < nx / 2 + ny / 2) { m = t - nx / 2 + 1; n = ny; off = nx; }
        else { m = t - nx / 2 - ny / 2 + 1; n = nz; off = nx + ny; }
        double re = 0.0, im = 0.0;
        for (int c = 0; c < n; ++c) {
            double sn, cs;
            sincospi(2.0 * (double)(((long long)m * c) % n) / n, &sn, &cs);
            re += tot[off + c] * cs;
            im -= tot[off + c] * sn;
        }
        acc[t] += (re * re + im * im) / N;
    }
}

template <typename T>
__global__ void drho3_kernel(const T *__restrict__ df, T *__restrict__ out, size_t n) {
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n;
         s += (size_t)gridDim.x * blockDim.x) {
        T g = df[s];
#pragma unroll
        for (int i = 1; i < 19; ++i) g += df[(size_t)i * n + s];
        out[s] = g;
    }
}

// FP64 conserved sums (mass deviation, jx, jy, jz): fixed two-pass order.
template <typename T>
__global__ void conserved3_kernel(const T *__restrict__ df, size_t n, double *__restrict__ part) {
    __shared__ double red[4][256];
    double m = 0, jx = 0, jy = 0, jz = 0;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n;
         s += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const double v = (double)df[(size_t)i * n + s];
            m += v;
            jx += cx3(i) * v;
            jy += cy3(i) * v;
            jz += cz3(i) * v;
        }
    }
    red[0][threadIdx.x] = m;
    red[1][threadIdx.x] = jx;
    red[2][threadIdx.x] = jy;
    red[3][threadIdx.x] = jz;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) part[4 * blockIdx.x + c] = red[c][0];
}

struct InitKeys3 {
    uint32_t rk[20];
};

// delta f_i = w_i amp z(site), z from Philox block 3 of step 0 (amp = 0: rest).
template <typename T>
__global__ void init3_kernel(T *__restrict__ df, size_t n, T amp, InitKeys3 keys,
                             uint32_t replica) {
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n;
         s += (size_t)gridDim.x * blockDim.x) {
        T d = T(0);
        if (amp != T(0)) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)s, 0u, replica, 3u), keys.rk);
            T z0, z1;
            box_muller(uniform01<T>(r.x), uniform01<T>(r.y), z0, z1);
            d = amp * z0;
        }
#pragma unroll
        for (int i = 0; i < 19; ++i) df[(size_t)i * n + s] = T(wq3(i)) * d;
    }
}

template <typename T>
__global__ void widen3_kernel(const T *__restrict__ df, double rho0, double *__restrict__ out,
                              size_t n, int mode) {
    // mode 0: density rho0 + sum_i delta f_i; mode 1: full populations
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n;
         s += (size_t)gridDim.x * blockDim.x) {
        if (mode == 0) {
            double v = 0.0;
            for (int i = 0; i < 19; ++i) v += (double)df[(size_t)i * n + s];
            out[s] = rho0 + v;
        } else {
            for (int i = 0; i < 19; ++i)
                out[(size_t)i * n + s] = (double)df[(size_t)i * n + s] + wq3(i) * rho0;
        }
    }
}
template <typename T>
__global__ void narrow3_kernel(const double *__restrict__ f, double rho0, T *__restrict__ df,
                               size_t n) {
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n;
         s += (size_t)gridDim.x * blockDim.x)
        for (int i = 0; i < 19; ++i)
            df[(size_t)i * n + s] = (T)(f[(size_t)i * n + s] - wq3(i) * rho0);
}

int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

// ---------------------------------------------------------------------------
// Full 3D structure factor: the density sample [nz][ny][nx] is transformed
// along x (two real rows per complex transform, half spectrum [nz][ny][ldx]),
// then along y and z in place by fft_lines_kernel, whose last pass adds
// |X(k)|^2 / N to the FP64 sums.  Power-of-two sizes.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void sk3_rows_kernel(const T *__restrict__ drho, typename C2<T>::t *__restrict__ spec,
                                const typename C2<T>::t *__restrict__ tw, int nx, int log2nx,
                                int ldx) {
    sk_rows_block<T>(drho, spec, tw, nx, log2nx, ldx, blockIdx.x);
}

// Length-n transforms of `cpb` neighbouring lines of plane blockIdx.y (line c
// holds data[c + j stride], j < n; lines c0 .. c0 + cpb - 1 of the nlines of
// the plane).  Without acc the result is written back; with acc, |X|^2 inv_n
// is added at the same index for the lines of a real half spectrum
// (c % ldx < hx).
template <typename T>
__global__ void fft_lines_kernel(typename C2<T>::t *__restrict__ data, int n, int log2n,
                                 size_t stride, size_t nlines, size_t plane, int cpb,
                                 const typename C2<T>::t *__restrict__ tw,
                                 double *__restrict__ acc, double inv_n, int ldx, int hx) {
    using CT = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *s = reinterpret_cast<CT *>(smem_raw);
    data += (size_t)blockIdx.y * plane;
    const size_t c0 = (size_t)blockIdx.x * cpb;
    const int total = cpb * n;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int c = e % cpb, j = e / cpb;
        CT v;
        if (c0 + c < nlines) {
            v = data[c0 + c + (size_t)j * stride];
        } else {
            v.x = T(0);
            v.y = T(0);
        }
        s[c * n + (__brev((unsigned)j) >> (32 - log2n))] = v;
    }
    __syncthreads();
    fft_smem<CT>(s, n, log2n, cpb, tw);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int c = e % cpb, k = e / cpb;
        if (c0 + c >= nlines) continue;
        const size_t idx = c0 + c + (size_t)k * stride;
        const CT v = s[c * n + k];
        if (acc) {
            if ((int)((c0 + c) % ldx) < hx) {
                const double re = (double)v.x, im = (double)v.y;
                acc[(size_t)blockIdx.y * plane + idx] += (re * re + im * im) * inv_n;
            }
        } else {
            data[idx] = v;
        }
    }
}

// Radial bins over the full k cube from the half spectrum: b = round(|q|),
// q_a = (wave number index on axis a) x max(n) / n_a; a kx column with
// 0 < kx < nx/2 stands for two modes (k and -k).  k = 0 excluded.
__global__ void sk3_bins_kernel(const double *__restrict__ acc, double inv_count,
                                double *__restrict__ bins, double *__restrict__ counts, int nbins,
                                int nx, int ny, int nz, int ldx) {
    const int hx = nx / 2 + 1;
    const size_t total = (size_t)hx * ny * nz;
    const double L = (double)max(nx, max(ny, nz));
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(e % hx);
        const size_t r = e / hx;
        const int ky = (int)(r % ny), kz = (int)(r / ny);
        if (kx == 0 && ky == 0 && kz == 0) continue;
        const int my = ky <= ny / 2 ? ky : ky - ny, mz = kz <= nz / 2 ? kz : kz - nz;
        const double qx = (double)kx * (L / nx), qy = (double)my * (L / ny),
                     qz = (double)mz * (L / nz);
        const int b = (int)rint(sqrt(qx * qx + qy * qy + qz * qz));
        if (b >= nbins) continue;
        const double w = (kx == 0 || 2 * kx == nx) ? 1.0 : 2.0;
        atomicAdd(&bins[b], w * acc[((size_t)kz * ny + ky) * ldx + kx] * inv_count);
        atomicAdd(&counts[b], w);
    }
}

// (sum_k S(k), sum_k |k| S(k)) over the full k cube, k = 0 excluded, |k| =
// 2 pi sqrt((kx/nx)^2 + (ky/ny)^2 + (kz/nz)^2) with folded indices.  One
// block, fixed summation order.
__global__ void __launch_bounds__(256)
sk3_moments_kernel(const double *__restrict__ acc, double inv_count, int nx, int ny, int nz,
                   int ldx, double *__restrict__ out) {
    const int hx = nx / 2 + 1;
    const size_t total = (size_t)hx * ny * nz;
    double s0 = 0.0, s1 = 0.0;
    for (size_t e = threadIdx.x; e < total; e += blockDim.x) {
        const int kx = (int)(e % hx);
        const size_t r = e / hx;
        const int ky = (int)(r % ny), kz = (int)(r / ny);
        if (kx == 0 && ky == 0 && kz == 0) continue;
        const int my = ky <= ny / 2 ? ky : ky - ny, mz = kz <= nz / 2 ? kz : kz - nz;
        const double w = (kx == 0 || 2 * kx == nx) ? 1.0 : 2.0;
        const double S = acc[((size_t)kz * ny + ky) * ldx + kx] * inv_count;
        const double qx = (double)kx / nx, qy = (double)my / ny, qz = (double)mz / nz;
        s0 += w * S;
        s1 += w * S * 6.283185307179586 * sqrt(qx * qx + qy * qy + qz * qz);
    }
    __shared__ double sh0[256], sh1[256];
    sh0[threadIdx.x] = s0;
    sh1[threadIdx.x] = s1;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh0[threadIdx.x] += sh0[threadIdx.x + o];
            sh1[threadIdx.x] += sh1[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh0[0];
        out[1] = sh1[0];
    }
}

}  // namespace
}  // namespace lbsc

using namespace lbsc;

struct lb3_ctx {
    int nx = 0, ny = 0, nz = 0, precision = 0, dev = 0;
    double G = 0, tau = 1, kT = 0, rho0 = 0;
    int psi_kind = LB_PSI_EXP;
    double psi_p1 = 0, psi_p2 = 0;
    size_t n = 0, esize = 4;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *df[2] = {nullptr, nullptr};
    int cur = 0;
    int *d_flag = nullptr;
    double *d_part = nullptr;      // conserved partials
    int nred = 0;
    void *drho = nullptr;          // delta rho of a sampling step
    double *d_prof = nullptr;      // [nz][nx] + [nz][ny] + [nz] plane profiles
    double *d_acc = nullptr;       // axis S(k) sums [nx/2 + ny/2 + nz/2]
    double *d_io = nullptr;        // n doubles for read-outs
    float2 *d_ring = nullptr;      // [1024] (cos, sin) of the noise ring angles
    bool sk_full = false;          // full 3D S(k) on sampling steps
    int ldx3 = 0;                  // padded half-spectrum row (nx / 2 + 1 -> multiple of 4)
    void *d_spec = nullptr;        // complex [nz][ny][ldx3] (storage precision)
    double *d_acc3 = nullptr;      // FP64 sums of |X|^2 / N, [nz][ny][ldx3]
    void *d_tw = nullptr;          // twiddles for nx, ny, nz (nx/2 + ny/2 + nz/2 complex)
    double *d_bins = nullptr;      // read-out scratch: bins, counts (2 nbins_cap) + 2 moments
    int nbins_cap = 0;
    int sk_every = 0;
    long long sk_start = 0, sk_count = 0, t = 0;
    uint64_t seed = 0;
    uint32_t replica = 0;
    int strip_z = 32;
    bool inited = false;
};

namespace {

#define L3_CHECK(call)                                                         \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess)                                                 \
            return e_ == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA; \
    } while (0)

template <typename T>
K3<T> params3(const lb3_ctx *h, bool sample) {
    K3<T> k;
    memset(&k, 0, sizeof(k));
    k.src = (const T *)h->df[h->cur];
    k.dst = (T *)h->df[h->cur ^ 1];
    k.drho_out = sample ? (T *)h->drho : nullptr;
    k.flag = h->d_flag;
    k.nx = h->nx;
    k.ny = h->ny;
    k.nz = h->nz;
    k.strip_z = h->strip_z;
    k.noise = h->kT > 0.0 ? 1 : 0;
    k.step = (uint32_t)h->t;
    k.replica = h->replica;
    k.rho0 = (T)h->rho0;
    k.force_pref = (T)(-h->G / 3.0);
    k.psi_kind = h->psi_kind;
    double psi0;
    switch (h->psi_kind) {
    case LB_PSI_CRITICAL: psi0 = sqrt(h->psi_p1 * h->psi_p2) * exp(1.0 - h->psi_p2 / h->rho0); break;
    case LB_PSI_AEXP: psi0 = h->psi_p1 * exp(-h->psi_p2 / h->rho0); break;
    default: psi0 = -expm1(-h->rho0);
    }
    k.psi0 = (T)psi0;
    k.psi_c = (T)(h->psi_kind == LB_PSI_EXP ? exp(-h->rho0) : psi0);
    k.psi_b = (T)(h->psi_kind == LB_PSI_EXP ? 0.0 : h->psi_p2);
    const double gam = 1.0 - 1.0 / h->tau;
    k.gamma = (T)gam;
    k.hsrc = (T)(0.5 * (1.0 + gam));
    const double mu = h->kT * 3.0;
    for (int kk = 4; kk < 19; ++kk) k.amp[kk] = (T)sqrt(mu * norm3(kk) * (1.0 - gam * gam));
    philox_round_keys(h->seed, k.rk);
    k.ring = h->d_ring;
    return k;
}

template <typename T, int TY>
int step3_launch(lb3_ctx *h, const K3<T> &k, bool sample) {
    const dim3 grid(h->nx / kTX3, h->ny / TY, (h->nz + h->strip_z - 1) / h->strip_z);
    const int nt = threads3<TY>();
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
        if (h->tau == 1.0) {   // gamma = 0: the unit-relaxation path
            if (sample) step3_kernel<T, true, true, TY><<<grid, nt, 0, h->stream>>>(k);
            else step3_kernel<T, false, true, TY><<<grid, nt, 0, h->stream>>>(k);
            done = true;
        }
    }
    if (!done && sample) step3_kernel<T, true, false, TY><<<grid, nt, 0, h->stream>>>(k);
    else if (!done) step3_kernel<T, false, false, TY><<<grid, nt, 0, h->stream>>>(k);
    L3_CHECK(cudaGetLastError());
    return LB_OK;
}

template <typename T>
int step3_once(lb3_ctx *h, bool sample) {
    const K3<T> k = params3<T>(h, sample);
    if constexpr (std::is_same<T, float>::value) {
        if (h->ny % 8 == 0) return step3_launch<T, 8>(h, k, sample);
    }
    return step3_launch<T, 4>(h, k, sample);
}

// Lines per block of a length-n transform: as many as fit 128 KB (at most 64).
int lines_per_block(int n, size_t csize) {
    int cpb = 64;
    while (cpb > 1 && (size_t)cpb * n * csize > 128 * 1024) cpb >>= 1;
    return cpb;
}

template <typename T>
int sample_full3(lb3_ctx *h) {
    using CT = typename C2<T>::t;
    const int nx = h->nx, ny = h->ny, nz = h->nz, ldx = h->ldx3, hx = nx / 2 + 1;
    const CT *twx = (const CT *)h->d_tw, *twy = twx + nx / 2, *twz = twy + ny / 2;
    CT *spec = (CT *)h->d_spec;
    // x: two real rows per block over the nz ny rows
    const size_t row_smem = (size_t)nx * sizeof(CT);
    L3_CHECK(cudaFuncSetAttribute(sk3_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)row_smem));
    const int rthreads = nx / 2 < 512 ? (nx / 2 < 32 ? 32 : nx / 2) : 512;
    sk3_rows_kernel<T><<<nz * ny / 2, rthreads, row_smem, h->stream>>>(
        (const T *)h->drho, spec, twx, nx, ilog2(nx), ldx);
    L3_CHECK(cudaGetLastError());
    L3_CHECK(cudaFuncSetAttribute(fft_lines_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  128 * 1024));
    // y: in place, the hx columns of each z plane
    int cpb = lines_per_block(ny, sizeof(CT));
    dim3 gy((hx + cpb - 1) / cpb, nz);
    fft_lines_kernel<T><<<gy, 512, (size_t)cpb * ny * sizeof(CT), h->stream>>>(
        spec, ny, ilog2(ny), (size_t)ldx, (size_t)hx, (size_t)ny * ldx, cpb, twy, nullptr, 0.0,
        ldx, hx);
    L3_CHECK(cudaGetLastError());
    // z: over all (y, kx) lines, adding |X|^2 / N
    cpb = lines_per_block(nz, sizeof(CT));
    const size_t nl = (size_t)ny * ldx;
    dim3 gz((unsigned)((nl + cpb - 1) / cpb), 1);
    fft_lines_kernel<T><<<gz, 512, (size_t)cpb * nz * sizeof(CT), h->stream>>>(
        spec, nz, ilog2(nz), nl, nl, 0, cpb, twz, h->d_acc3, 1.0 / ((double)nx * ny * nz), ldx,
        hx);
    L3_CHECK(cudaGetLastError());
    return LB_OK;
}

int sample3(lb3_ctx *h) {
    double *px = h->d_prof, *py = px + (size_t)h->nz * h->nx, *pz = py + (size_t)h->nz * h->ny;
    if (h->precision == LB_FP32)
        profile3_kernel<float><<<h->nz, 256, 0, h->stream>>>((const float *)h->drho, h->nx, h->ny,
                                                             px, py, pz);
    else
        profile3_kernel<double><<<h->nz, 256, 0, h->stream>>>((const double *)h->drho, h->nx,
                                                              h->ny, px, py, pz);
    L3_CHECK(cudaGetLastError());
    axis_dft3_kernel<<<1, 512, (size_t)(h->nx + h->ny + h->nz) * sizeof(double), h->stream>>>(
        px, py, pz, h->nx, h->ny, h->nz, h->d_acc);
    L3_CHECK(cudaGetLastError());
    if (h->sk_full) {
        const int rc = h->precision == LB_FP32 ? sample_full3<float>(h) : sample_full3<double>(h);
        if (rc) return rc;
    }
    h->sk_count += 1;
    return LB_OK;
}

int sync3(lb3_ctx *h) {
    L3_CHECK(cudaStreamSynchronize(h->stream));
    int flag = 0;
    L3_CHECK(cudaMemcpy(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        L3_CHECK(cudaMemset(h->d_flag, 0, sizeof(int)));
        return LB_ERR_NONFINITE;
    }
    return LB_OK;
}

void free3(lb3_ctx *h) {
    cudaFree(h->df[0]);
    cudaFree(h->df[1]);
    cudaFree(h->d_flag);
    cudaFree(h->d_part);
    cudaFree(h->drho);
    cudaFree(h->d_prof);
    cudaFree(h->d_acc);
    cudaFree(h->d_io);
    cudaFree(h->d_ring);
    cudaFree(h->d_spec);
    cudaFree(h->d_acc3);
    cudaFree(h->d_tw);
    cudaFree(h->d_bins);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

}  // namespace

extern "C" {

int lb3_create(lb3_ctx **out, int nx, int ny, int nz, double G, double tau, double kT,
               int precision, void *stream) {
    if (!out) return LB_ERR_ARG;
    *out = nullptr;
    if (nx < kTX3 || ny < kTYMin3 || nz < 3 || nx % kTX3 || ny % kTYMin3) return LB_ERR_ARG;
    if (19.0 * (double)nx * ny * nz >= 4294967296.0) return LB_ERR_ARG;
    if (!(tau > 0.5) || !(kT >= 0.0) || !isfinite(G)) return LB_ERR_ARG;
    if (precision != LB_FP32 && precision != LB_FP64) return LB_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return LB_ERR_CUDA;
    lb3_ctx *h = new (std::nothrow) lb3_ctx();
    if (!h) return LB_ERR_NOMEM;
    cudaGetDevice(&h->dev);
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->G = G;
    h->tau = tau;
    h->kT = kT;
    h->precision = precision;
    h->esize = precision == LB_FP32 ? 4 : 8;
    h->n = (size_t)nx * ny * nz;
    h->strip_z = nz < 32 ? nz : 32;
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) == cudaSuccess) {
        h->own_stream = true;
    } else {
        delete h;
        return LB_ERR_CUDA;
    }
    h->nred = 152 * 4;
    const size_t nb = 19 * h->n * h->esize;
    cudaError_t e = cudaMalloc(&h->df[0], nb);
    if (e == cudaSuccess) e = cudaMalloc(&h->df[1], nb);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_flag, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_part, 4 * h->nred * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_ring, kRing3 * sizeof(float2));
    if (e == cudaSuccess) {
        float2 tab[kRing3];
        for (int a = 0; a < kRing3; ++a) {
            const double th = M_PI * (2.0 * a + 1.0) / kRing3;   // 2 pi (a + 1/2) / 1024
            tab[a] = make_float2((float)cos(th), (float)sin(th));
        }
        e = cudaMemcpy(h->d_ring, tab, sizeof(tab), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        free3(h);
        delete h;
        return e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA;
    }
    *out = h;
    return LB_OK;
}

void lb3_destroy(lb3_ctx *h) {
    if (!h) return;
    cudaSetDevice(h->dev);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free3(h);
    delete h;
}

int lb3_init(lb3_ctx *h, double rho0, uint64_t seed, double init_amp) {
    if (!h || !(rho0 > 0.0) || !isfinite(init_amp)) return LB_ERR_ARG;
    L3_CHECK(cudaSetDevice(h->dev));
    h->rho0 = rho0;
    h->seed = seed;
    h->t = 0;
    h->cur = 0;
    InitKeys3 k;
    philox_round_keys(seed, k.rk);
    if (h->precision == LB_FP32)
        init3_kernel<float><<<grid_for(h->n), 256, 0, h->stream>>>((float *)h->df[0], h->n,
                                                                    (float)init_amp, k, h->replica);
    else
        init3_kernel<double><<<grid_for(h->n), 256, 0, h->stream>>>((double *)h->df[0], h->n,
                                                                     init_amp, k, h->replica);
    L3_CHECK(cudaGetLastError());
    if (h->d_acc) {
        L3_CHECK(cudaMemsetAsync(h->d_acc, 0, (h->nx / 2 + h->ny / 2 + h->nz / 2) * sizeof(double),
                                 h->stream));
        h->sk_count = 0;
    }
    if (h->d_acc3)
        L3_CHECK(cudaMemsetAsync(h->d_acc3, 0, (size_t)h->nz * h->ny * h->ldx3 * sizeof(double),
                                 h->stream));
    h->inited = true;
    return LB_OK;
}

int lb3_set_psi(lb3_ctx *h, int psi_kind, double p1, double p2) {
    if (!h || psi_kind < LB_PSI_EXP || psi_kind > LB_PSI_AEXP) return LB_ERR_ARG;
    if (psi_kind != LB_PSI_EXP && !(p1 > 0.0 && p2 > 0.0)) return LB_ERR_ARG;
    h->psi_kind = psi_kind;
    h->psi_p1 = p1;
    h->psi_p2 = p2;
    return LB_OK;
}

int lb3_set_replica(lb3_ctx *h, uint32_t replica) {
    if (!h) return LB_ERR_ARG;
    h->replica = replica;
    return LB_OK;
}

int lb3_set_strip(lb3_ctx *h, int planes) {
    if (!h || planes < 1 || planes > h->nz) return LB_ERR_ARG;
    h->strip_z = planes;
    return LB_OK;
}

int lb3_step(lb3_ctx *h, int n) {
    if (!h || n < 0) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    L3_CHECK(cudaSetDevice(h->dev));
    for (int s = 0; s < n; ++s) {
        const long long tn = h->t + 1;
        const bool sample = h->sk_every > 0 && h->d_acc && tn >= h->sk_start &&
                            (tn - h->sk_start) % h->sk_every == 0;
        const int rc = h->precision == LB_FP32 ? step3_once<float>(h, sample)
                                               : step3_once<double>(h, sample);
        if (rc) return rc;
        h->cur ^= 1;
        h->t = tn;
        if (sample) {
            const int r2 = sample3(h);
            if (r2) return r2;
        }
    }
    return LB_OK;
}

int lb3_sync(lb3_ctx *h) {
    if (!h) return LB_ERR_ARG;
    L3_CHECK(cudaSetDevice(h->dev));
    return sync3(h);
}

long long lb3_get_step(const lb3_ctx *h) { return h ? h->t : -1; }

static int ensure_io3(lb3_ctx *h) {
    if (h->d_io) return LB_OK;
    L3_CHECK(cudaMalloc(&h->d_io, 19 * h->n * sizeof(double)));
    return LB_OK;
}

int lb3_density(lb3_ctx *h, double *host_out) {
    if (!h || !host_out) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    L3_CHECK(cudaSetDevice(h->dev));
    int rc = ensure_io3(h);
    if (rc) return rc;
    if (h->precision == LB_FP32)
        widen3_kernel<float><<<grid_for(h->n), 256, 0, h->stream>>>(
            (const float *)h->df[h->cur], h->rho0, h->d_io, h->n, 0);
    else
        widen3_kernel<double><<<grid_for(h->n), 256, 0, h->stream>>>(
            (const double *)h->df[h->cur], h->rho0, h->d_io, h->n, 0);
    L3_CHECK(cudaGetLastError());
    L3_CHECK(cudaMemcpyAsync(host_out, h->d_io, h->n * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    return sync3(h);
}

int lb3_populations(lb3_ctx *h, double *host_out) {
    if (!h || !host_out) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    L3_CHECK(cudaSetDevice(h->dev));
    int rc = ensure_io3(h);
    if (rc) return rc;
    if (h->precision == LB_FP32)
        widen3_kernel<float><<<grid_for(h->n), 256, 0, h->stream>>>(
            (const float *)h->df[h->cur], h->rho0, h->d_io, h->n, 1);
    else
        widen3_kernel<double><<<grid_for(h->n), 256, 0, h->stream>>>(
            (const double *)h->df[h->cur], h->rho0, h->d_io, h->n, 1);
    L3_CHECK(cudaGetLastError());
    L3_CHECK(cudaMemcpyAsync(host_out, h->d_io, 19 * h->n * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
    return sync3(h);
}

int lb3_set_populations(lb3_ctx *h, const double *host_f) {
    if (!h || !host_f) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    L3_CHECK(cudaSetDevice(h->dev));
    int rc = ensure_io3(h);
    if (rc) return rc;
    L3_CHECK(cudaMemcpyAsync(h->d_io, host_f, 19 * h->n * sizeof(double), cudaMemcpyHostToDevice,
                             h->stream));
    if (h->precision == LB_FP32)
        narrow3_kernel<float><<<grid_for(h->n), 256, 0, h->stream>>>(h->d_io, h->rho0,
                                                                      (float *)h->df[h->cur], h->n);
    else
        narrow3_kernel<double><<<grid_for(h->n), 256, 0, h->stream>>>(
            h->d_io, h->rho0, (double *)h->df[h->cur], h->n);
    L3_CHECK(cudaGetLastError());
    return sync3(h);
}

int lb3_conserved(lb3_ctx *h, double out[4]) {
    if (!h || !out) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    L3_CHECK(cudaSetDevice(h->dev));
    if (h->precision == LB_FP32)
        conserved3_kernel<float><<<h->nred, 256, 0, h->stream>>>((const float *)h->df[h->cur],
                                                                  h->n, h->d_part);
    else
        conserved3_kernel<double><<<h->nred, 256, 0, h->stream>>>((const double *)h->df[h->cur],
                                                                   h->n, h->d_part);
    L3_CHECK(cudaGetLastError());
    double *part = new (std::nothrow) double[4 * h->nred];
    if (!part) return LB_ERR_NOMEM;
    cudaError_t e = cudaMemcpyAsync(part, h->d_part, 4 * h->nred * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->stream);
    int rc = e == cudaSuccess ? sync3(h) : LB_ERR_CUDA;
    if (rc == LB_OK) {
        double s[4] = {0, 0, 0, 0};
        for (int b = 0; b < h->nred; ++b)
            for (int c = 0; c < 4; ++c) s[c] += part[4 * b + c];
        out[0] = (double)h->n * h->rho0 + s[0];
        out[1] = s[1];
        out[2] = s[2];
        out[3] = s[3];
    }
    delete[] part;
    return rc;
}

int lb3_sk_config(lb3_ctx *h, int every, long long start) {
    if (!h || every < 0 || start < 0) return LB_ERR_ARG;
    L3_CHECK(cudaSetDevice(h->dev));
    if (every > 0 && !h->d_acc) {
        const int nm = h->nx / 2 + h->ny / 2 + h->nz / 2;
        L3_CHECK(cudaMalloc(&h->drho, h->n * h->esize));
        L3_CHECK(cudaMalloc(&h->d_prof, ((size_t)h->nz * (h->nx + h->ny + 1)) * sizeof(double)));
        L3_CHECK(cudaMalloc(&h->d_acc, nm * sizeof(double)));
        L3_CHECK(cudaMemsetAsync(h->d_acc, 0, nm * sizeof(double), h->stream));
        h->sk_count = 0;
    }
    h->sk_every = every;
    h->sk_start = start;
    return LB_OK;
}

int lb3_sk_reset(lb3_ctx *h) {
    if (!h) return LB_ERR_ARG;
    if (h->d_acc) {
        L3_CHECK(cudaSetDevice(h->dev));
        L3_CHECK(cudaMemsetAsync(h->d_acc, 0, (h->nx / 2 + h->ny / 2 + h->nz / 2) * sizeof(double),
                                 h->stream));
    }
    if (h->d_acc3)
        L3_CHECK(cudaMemsetAsync(h->d_acc3, 0, (size_t)h->nz * h->ny * h->ldx3 * sizeof(double),
                                 h->stream));
    h->sk_count = 0;
    return LB_OK;
}

static bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int lb3_sk_full(lb3_ctx *h, int enable) {
    if (!h) return LB_ERR_ARG;
    if (!enable) {
        h->sk_full = false;
        return LB_OK;
    }
    if (!pow2(h->nx) || !pow2(h->ny) || !pow2(h->nz) || h->nx > 16384 || h->ny > 16384 ||
        h->nz > 16384)
        return LB_ERR_UNSUPPORTED;
    if (!h->d_acc) return LB_ERR_STATE;      // lb3_sk_config first
    L3_CHECK(cudaSetDevice(h->dev));
    if (!h->d_acc3) {
        const size_t cs = h->precision == LB_FP32 ? sizeof(float2) : sizeof(double2);
        h->ldx3 = ((h->nx / 2 + 1) + 3) / 4 * 4;
        const size_t ne = (size_t)h->nz * h->ny * h->ldx3;
        cudaError_t e = cudaMalloc(&h->d_spec, ne * cs);
        if (e == cudaSuccess) e = cudaMalloc(&h->d_acc3, ne * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&h->d_tw, (size_t)(h->nx + h->ny + h->nz) / 2 * cs);
        if (e != cudaSuccess) {
            cudaFree(h->d_spec);
            cudaFree(h->d_acc3);
            cudaFree(h->d_tw);
            h->d_spec = h->d_tw = nullptr;
            h->d_acc3 = nullptr;
            return e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA;
        }
        L3_CHECK(cudaMemsetAsync(h->d_spec, 0, ne * cs, h->stream));
        L3_CHECK(cudaMemsetAsync(h->d_acc3, 0, ne * sizeof(double), h->stream));
        const int prec = h->precision == LB_FP32 ? 0 : 1;
        char *tw = (char *)h->d_tw;
        L3_CHECK(launch_twiddles(prec, tw, h->nx, h->stream));
        L3_CHECK(launch_twiddles(prec, tw + (size_t)h->nx / 2 * cs, h->ny, h->stream));
        L3_CHECK(launch_twiddles(prec, tw + (size_t)(h->nx + h->ny) / 2 * cs, h->nz, h->stream));
    }
    h->sk_full = true;
    return LB_OK;
}

static int bins_scratch3(lb3_ctx *h, int nbins) {
    if (h->d_bins && h->nbins_cap >= nbins) return LB_OK;
    cudaFree(h->d_bins);
    h->d_bins = nullptr;
    h->nbins_cap = 0;
    if (cudaMalloc(&h->d_bins, (2 * (size_t)nbins + 2) * sizeof(double)) != cudaSuccess)
        return LB_ERR_NOMEM;
    h->nbins_cap = nbins;
    return LB_OK;
}

int lb3_structure_factor(lb3_ctx *h, double *host_bins, int nbins, long long *nsamples_out) {
    if (!h || !host_bins || nbins < 1) return LB_ERR_ARG;
    if (!h->d_acc3) return LB_ERR_STATE;
    L3_CHECK(cudaSetDevice(h->dev));
    int rc = bins_scratch3(h, nbins);
    if (rc) return rc;
    double *bins = h->d_bins, *counts = bins + nbins;
    L3_CHECK(cudaMemsetAsync(bins, 0, 2 * (size_t)nbins * sizeof(double), h->stream));
    const double inv = h->sk_count ? 1.0 / (double)h->sk_count : 0.0;
    const size_t total = (size_t)(h->nx / 2 + 1) * h->ny * h->nz;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    sk3_bins_kernel<<<blocks, 256, 0, h->stream>>>(h->d_acc3, inv, bins, counts, nbins, h->nx,
                                                   h->ny, h->nz, h->ldx3);
    L3_CHECK(cudaGetLastError());
    double *tmp = new (std::nothrow) double[2 * (size_t)nbins];
    if (!tmp) return LB_ERR_NOMEM;
    cudaError_t e = cudaMemcpyAsync(tmp, bins, 2 * (size_t)nbins * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->stream);
    rc = e == cudaSuccess ? sync3(h) : LB_ERR_CUDA;
    if (rc == LB_OK)
        for (int b = 0; b < nbins; ++b)
            host_bins[b] = tmp[nbins + b] > 0.0 ? tmp[b] / tmp[nbins + b] : 0.0;
    delete[] tmp;
    if (rc) return rc;
    if (nsamples_out) *nsamples_out = h->sk_count;
    return LB_OK;
}

int lb3_sk_moments(lb3_ctx *h, double *host_out2) {
    if (!h || !host_out2) return LB_ERR_ARG;
    if (!h->d_acc3) return LB_ERR_STATE;
    L3_CHECK(cudaSetDevice(h->dev));
    int rc = bins_scratch3(h, 1);
    if (rc) return rc;
    double *m = h->d_bins + 2 * (size_t)h->nbins_cap;
    const double inv = h->sk_count ? 1.0 / (double)h->sk_count : 0.0;
    sk3_moments_kernel<<<1, 256, 0, h->stream>>>(h->d_acc3, inv, h->nx, h->ny, h->nz, h->ldx3, m);
    L3_CHECK(cudaGetLastError());
    L3_CHECK(cudaMemcpyAsync(host_out2, m, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return sync3(h);
}

int lb3_structure_factor_axes(lb3_ctx *h, double *host_out, long long *nsamples_out) {
    if (!h || !host_out) return LB_ERR_ARG;
    const int nm = h->nx / 2 + h->ny / 2 + h->nz / 2;
    if (!h->d_acc) return LB_ERR_STATE;
    L3_CHECK(cudaSetDevice(h->dev));
    L3_CHECK(cudaMemcpyAsync(host_out, h->d_acc, nm * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    const int rc = sync3(h);
    if (rc) return rc;
    for (int m = 0; m < nm; ++m) host_out[m] = h->sk_count ? host_out[m] / (double)h->sk_count : 0.0;
    if (nsamples_out) *nsamples_out = h->sk_count;
    return LB_OK;
}

}  // extern "C"
