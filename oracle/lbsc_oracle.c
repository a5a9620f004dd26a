/*
 * lbsc_oracle.c -- plain, slow FP64 CPU oracle for the fluctuating Shan-Chen
 * D2Q9 lattice Boltzmann step of Lulli, Biferale, Falcucci, Sbragaglia, Yang
 * and Shan, "Metastable and Unstable Dynamics in multi-phase lattice
 * Boltzmann" (arXiv:2212.07848).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the package smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it computes, in the paper's order:
 *   - the lattice Boltzmann equation with collision, forcing and noise,
 *     Eq. (12): f_i(x + xi_i, t + 1) - f_i(x, t) = Omega_i + F_i + eta_i;
 *   - Omega_i: single-relaxation-time BGK towards the second-order Hermite
 *     equilibrium (the text after Eq. (12) names "the usual BGK");
 *   - F_i: the forcing of Guo, Zheng and Shi (2002), which the text after
 *     Eq. (12) names, driven by the Shan-Chen force of Eq. (1);
 *   - eta_i: Gaussian noise with a covariance diagonal in moment space, zero
 *     on the conserved moments (mass and momentum), following the noise
 *     paragraph after Eq. (16) in two dimensions;
 *   - the density structure factor S(k) = <|delta n(k)|^2> defined after
 *     Eq. (12), by a direct (separable) discrete Fourier sum.
 *
 * Storage is the FULL population f_i in FP64 (not a deviation from
 * equilibrium), the collision is written in POPULATION space and the
 * noise is projected explicitly from moment space.  The GPU path uses
 * deviation storage and a moment-space collision; for a single relaxation
 * time the two are algebraically identical, so agreement is a real check.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - sign convention: F = -G c_s^2 psi(x) sum_a w_a psi(x+e_a) e_a with the
 *     force-stencil weights normalised so that sum_a w_a e_ax^2 = 1; G < 0 is
 *     attractive.  This gives p = rho c_s^2 + (G c_s^2 / 2) psi^2, i.e. the
 *     paper's Eq. (2) with T = c_s^2 and psi_paper^2 = -G c_s^2 psi^2;
 *   - noise amplitude (the paper defers it to its supplement): fluctuation-
 *     dissipation amplitude sqrt(mu rho b_k (1 - gamma^2)) on each
 *     non-conserved Hermite moment k, mu = k_B theta / c_s^2, gamma = 1-1/tau,
 *     rho the local pre-collision density;
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11,
 *     "Parallel random numbers: as easy as 1, 2, 3"), key = 64-bit seed,
 *     counter = (site, step, replica, block), uniforms (r + 1/2) 2^-32.  One
 *     call (block 0) per site and step: Box-Muller on a ring of 1024 angles,
 *     radius word r0 with angle index bits 0-9 of r3 -> modes 3,4; r1 with
 *     bits 10-19 -> modes 5,6; r2 with bits 20-29 -> modes 7,8.  Block 2 of
 *     step 0 drives the optional initial density kick (a plain Box-Muller
 *     pair (r0, r1)).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* D2Q9 velocity set and weights (standard lattice, c_s^2 = 1/3).            */
/* ------------------------------------------------------------------------ */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WQ[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

/* Hermite moment basis, written as polynomials of the velocity c:
 *   0: 1            1: cx            2: cy
 *   3: 3c^2 - 2     4: cx^2 - cy^2   5: cx cy
 *   6: (3c^2-4) cx  7: (3c^2-4) cy   8: 9c^4 - 15c^2 + 2
 * Modes 0..2 are conserved (mass, momentum); 3..8 carry noise. */
static double basis(int k, int i) {
    double cx = CX[i], cy = CY[i], c2 = cx * cx + cy * cy;
    switch (k) {
    case 0: return 1.0;
    case 1: return cx;
    case 2: return cy;
    case 3: return 3.0 * c2 - 2.0;
    case 4: return cx * cx - cy * cy;
    case 5: return cx * cy;
    case 6: return (3.0 * c2 - 4.0) * cx;
    case 7: return (3.0 * c2 - 4.0) * cy;
    case 8: return 9.0 * c2 * c2 - 15.0 * c2 + 2.0;
    }
    return 0.0;
}

/* b_k = sum_i w_i e_ki^2, computed rather than tabulated. */
static double basis_norm_sum(int k) {
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += WQ[i] * basis(k, i) * basis(k, i);
    return s;
}

/* Values e_ki and norms b_k, evaluated once from the definitions above. */
static double E_KI[9][9], B_K[9];
static int basis_ready = 0;
static void basis_setup(void) {
    if (basis_ready) return;
    for (int k = 0; k < 9; ++k) {
        for (int i = 0; i < 9; ++i) E_KI[k][i] = basis(k, i);
        B_K[k] = basis_norm_sum(k);
    }
    basis_ready = 1;
}
static double basis_norm(int k) { basis_setup(); return B_K[k]; }

/* ------------------------------------------------------------------------ */
/* Isotropic force stencils E4 / E6 / E8 (Eq. (1): the weights w(|e_a|^2)).  */
/* The paper does not print them; these are the standard isotropic sets,    */
/* normalised to sum_a w_a e_ax^2 = 1 (the test suite re-derives them from   */
/* the isotropy equations).                                                  */
/* ------------------------------------------------------------------------ */
static double stencil_weight(int order, int e2) {
    if (order == 4) {
        if (e2 == 1) return 1.0 / 3.0;
        if (e2 == 2) return 1.0 / 12.0;
    } else if (order == 6) {
        if (e2 == 1) return 4.0 / 15.0;
        if (e2 == 2) return 1.0 / 10.0;
        if (e2 == 4) return 1.0 / 120.0;
    } else if (order == 8) {
        if (e2 == 1) return 4.0 / 21.0;
        if (e2 == 2) return 4.0 / 45.0;
        if (e2 == 4) return 1.0 / 60.0;
        if (e2 == 5) return 2.0 / 315.0;
        if (e2 == 8) return 1.0 / 5040.0;
    }
    return 0.0;
}

/* Enumerate the neighbour vectors with a nonzero weight: every (ex, ey)
 * with |ex|, |ey| <= 2, (ex, ey) != 0. Returns the count. */
static int stencil_vectors(int order, int *ex, int *ey, double *w) {
    int n = 0;
    for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
            int e2 = dx * dx + dy * dy;
            if (e2 == 0) continue;
            double ww = stencil_weight(order, e2);
            if (ww == 0.0) continue;
            if (ex) { ex[n] = dx; ey[n] = dy; w[n] = ww; }
            ++n;
        }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Philox4xW-10 (Salmon et al., SC'11).  One macro defines the round        */
/* structure for both word widths so that the 64-bit instance, which numpy  */
/* also provides, pins the structure shared with the 32-bit instance.       */
/* Round: (c0,c1,c2,c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),                  */
/*                          hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));                 */
/* key schedule: (k0,k1) += (W0,W1) before every round but the first.       */
/* ------------------------------------------------------------------------ */
static inline uint32_t mulhilo32(uint32_t a, uint32_t b, uint32_t *lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *lo = (uint32_t)p;
    return (uint32_t)(p >> 32);
}
static inline uint64_t mulhilo64(uint64_t a, uint64_t b, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *lo = (uint64_t)p;
    return (uint64_t)(p >> 64);
}

#define DEFINE_PHILOX4(NAME, T, MULHILO, M0, M1, W0, W1)                     \
    void NAME(const T *ctr, const T *key, T *out) {                          \
        T c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];                \
        T k0 = key[0], k1 = key[1];                                          \
        for (int r = 0; r < 10; ++r) {                                       \
            if (r > 0) { k0 = (T)(k0 + (W0)); k1 = (T)(k1 + (W1)); }         \
            T lo0, lo1;                                                      \
            T hi0 = MULHILO((T)(M0), c0, &lo0);                              \
            T hi1 = MULHILO((T)(M1), c2, &lo1);                              \
            T n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;                        \
            c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;                            \
        }                                                                    \
        out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;                  \
    }

DEFINE_PHILOX4(or_philox4x32_10, uint32_t, mulhilo32, 0xD2511F53u,
               0xCD9E8D57u, 0x9E3779B9u, 0xBB67AE85u)
DEFINE_PHILOX4(or_philox4x64_10, uint64_t, mulhilo64, 0xD2E7470EE14C6C93ull,
               0xCA5A826395121157ull, 0x9E3779B97F4A7C15ull,
               0xBB67AE8584CAA73Bull)

/* Uniform in (0,1): (r + 1/2) * 2^-32, exact in FP64. */
static double uniform01(uint32_t r) {
    return ((double)r + 0.5) * (1.0 / 4294967296.0);
}

/* Box-Muller: two uniforms -> two independent standard normals. */
static void box_muller(uint32_t ra, uint32_t rb, double *z0, double *z1) {
    double rad = sqrt(-2.0 * log(uniform01(ra)));
    double th = 2.0 * M_PI * uniform01(rb);
    *z0 = rad * cos(th);
    *z1 = rad * sin(th);
}

/* Box-Muller with the angle taken from 1024 equally spaced values: radius
 * from the uniform of word ra, angle th = 2 pi (a + 1/2) / 1024 for a 10-bit
 * index a.  All moments of (cos th, sin th) below order 1024 equal those of a
 * uniform angle, so (z0, z1) has the moments of two independent standard
 * normals up to that order. */
static void box_muller_ring(uint32_t ra, uint32_t a, double *z0, double *z1) {
    double rad = sqrt(-2.0 * log(uniform01(ra)));
    double th = 2.0 * M_PI * ((double)(a & 1023u) + 0.5) / 1024.0;
    *z0 = rad * cos(th);
    *z1 = rad * sin(th);
}

/* The six thermal normals of a site: one Philox draw (block 0). */
static void site_normals(const uint32_t r[4], double z[6]) {
    box_muller_ring(r[0], r[3], &z[0], &z[1]);
    box_muller_ring(r[1], r[3] >> 10, &z[2], &z[3]);
    box_muller_ring(r[2], r[3] >> 20, &z[4], &z[5]);
}

/* ------------------------------------------------------------------------ */
/* Model parameters (mirrors the product's create arguments).               */
/* ------------------------------------------------------------------------ */
typedef struct or_params {
    int nx, ny;
    double G, tau, kT;
    int psi_kind;            /* 0: 1-exp(-rho); 1: sqrt(Tc nc) exp(1-nc/rho);
                                2: a exp(-b/rho) */
    double psi_p1, psi_p2;   /* kind 1: (Tc, nc); kind 2: (a, b) */
    int stencil;             /* 4, 6 or 8 */
    double rho0;             /* reference density of the homogeneous state */
    uint64_t seed;
    uint32_t replica;
    double tau_bulk;         /* relaxation time of mode 3 (0: tau)          */
    double tau_ghost;        /* relaxation time of modes 6, 7, 8 (0: tau)   */
    int force_mrt;           /* 1: use the moment-space path even for one tau */
} or_params;

/* Pseudopotential psi(n), Eq. (5) (kind 1), the a exp(-b/n) form preceding
 * Eq. (3) (kind 2), and the classic 1 - exp(-rho) (kind 0). */
double or_psi(const or_params *p, double rho) {
    switch (p->psi_kind) {
    case 0: return 1.0 - exp(-rho);
    case 1: return sqrt(p->psi_p1 * p->psi_p2) * exp(1.0 - p->psi_p2 / rho);
    case 2: return p->psi_p1 * exp(-p->psi_p2 / rho);
    }
    return NAN;
}

/* Four Philox words for (site, step, block). */
static void draw(const or_params *p, uint32_t site, uint32_t step,
                 uint32_t block, uint32_t out[4]) {
    uint32_t ctr[4] = {site, step, p->replica, block};
    uint32_t key[2] = {(uint32_t)(p->seed & 0xffffffffu),
                       (uint32_t)(p->seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

static inline int wrap(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

#define IDX(i, x, y, nx, ny) (((size_t)(i) * (size_t)(ny) + (size_t)(y)) * (size_t)(nx) + (size_t)(x))

/* Post-collision populations of one site, given its streamed populations g,
 * its Shan-Chen force F, and the step counter t (number of completed steps).
 * Eq. (12) with BGK Omega, Guo forcing and moment-space noise. */
static void collide_site(const or_params *p, uint32_t site, uint32_t t,
                         const double g[9], double Fx, double Fy,
                         double out[9]) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho += g[i];
        jx += CX[i] * g[i];
        jy += CY[i] * g[i];
    }
    /* Guo et al. (2002): the equilibrium and source use u = (j + F/2)/rho. */
    double ux = (jx + 0.5 * Fx) / rho;
    double uy = (jy + 0.5 * Fy) / rho;
    double usq = ux * ux + uy * uy;
    double tau = p->tau;

    /* Thermal noise: N_k = sqrt(mu rho b_k (1-gamma^2)) z_k on k = 3..8. */
    double z[9] = {0};
    if (p->kT > 0.0) {
        uint32_t r[4];
        draw(p, site, t, 0, r);
        site_normals(r, &z[3]);
    }
    double gam = 1.0 - 1.0 / tau;
    double mu = p->kT / CS2;
    basis_setup();
    double N[9] = {0};
    for (int k = 3; k < 9; ++k)
        N[k] = sqrt(mu * rho * basis_norm(k) * (1.0 - gam * gam)) * z[k];

    double tb = p->tau_bulk > 0.0 ? p->tau_bulk : tau;
    double tg = p->tau_ghost > 0.0 ? p->tau_ghost : tau;
    if (p->force_mrt || tb != tau || tg != tau) {
        /* Multiple relaxation times (the NEXT variant of the BGK collision):
         * in the Hermite basis, m*_k = m_k + l_k (m_eq_k - m_k)
         * + (1 - l_k/2) S_k + N_k with l_k = 1/tau_k per mode (mode 3: bulk,
         * modes 4, 5: shear, modes 6, 7, 8: ghosts), S_k the moments of the
         * Guo source, N_k = sqrt(mu rho b_k (1 - (1 - l_k)^2)) z_k. */
        double feq[9], sg[9];
        for (int i = 0; i < 9; ++i) {
            double cu = CX[i] * ux + CY[i] * uy;
            feq[i] = WQ[i] * rho *
                     (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - usq / (2.0 * CS2));
            double sx = (CX[i] - ux) / CS2 + cu * CX[i] / (CS2 * CS2);
            double sy = (CY[i] - uy) / CS2 + cu * CY[i] / (CS2 * CS2);
            sg[i] = WQ[i] * (sx * Fx + sy * Fy);
        }
        double mstar[9];
        for (int k = 0; k < 9; ++k) {
            double m = 0.0, meq = 0.0, sm = 0.0;
            for (int i = 0; i < 9; ++i) {
                m += E_KI[k][i] * g[i];
                meq += E_KI[k][i] * feq[i];
                sm += E_KI[k][i] * sg[i];
            }
            double tk = (k == 3) ? tb : (k >= 6 ? tg : tau);
            double lk = 1.0 / tk;
            double nk = 0.0;
            if (k >= 3) {
                double gk = 1.0 - lk;
                nk = sqrt(mu * rho * B_K[k] * (1.0 - gk * gk)) * z[k];
            }
            mstar[k] = m + lk * (meq - m) + (1.0 - 0.5 * lk) * sm + nk;
        }
        for (int i = 0; i < 9; ++i) {
            double v = 0.0;
            for (int k = 0; k < 9; ++k) v += E_KI[k][i] * mstar[k] / B_K[k];
            out[i] = WQ[i] * v;
        }
        return;
    }

    for (int i = 0; i < 9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        double feq = WQ[i] * rho *
                     (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) -
                      usq / (2.0 * CS2));
        /* Guo source: w_i [ (c_i - u)/c_s^2 + (c_i.u) c_i / c_s^4 ] . F */
        double sx = (CX[i] - ux) / CS2 + cu * CX[i] / (CS2 * CS2);
        double sy = (CY[i] - uy) / CS2 + cu * CY[i] / (CS2 * CS2);
        double src = (1.0 - 1.0 / (2.0 * tau)) * WQ[i] * (sx * Fx + sy * Fy);
        double eta = 0.0;
        for (int k = 3; k < 9; ++k)
            eta += E_KI[k][i] * N[k] / B_K[k];
        eta *= WQ[i];
        out[i] = g[i] - (g[i] - feq) / tau + src + eta;
    }
}

/* ------------------------------------------------------------------------ */
/* Lattice state.                                                            */
/* ------------------------------------------------------------------------ */
typedef struct or_lattice {
    or_params p;
    long long t;        /* completed steps */
    double *f;          /* [9][ny][nx], full populations, post-collision */
    double *g;          /* streamed populations (work) */
    double *rho, *psi;  /* [ny][nx] (work) */
    int sk_every;
    long long sk_start, sk_count;
    double *sk_acc;     /* [ny][nx/2+1], sum over samples of |X(k)|^2 / N */
} or_lattice;

or_lattice *or_create(const or_params *p) {
    if (p->nx < 1 || p->ny < 1) return NULL;
    if (p->stencil != 4 && p->stencil != 6 && p->stencil != 8) return NULL;
    or_lattice *h = (or_lattice *)calloc(1, sizeof(or_lattice));
    if (!h) return NULL;
    h->p = *p;
    size_t n = (size_t)p->nx * (size_t)p->ny;
    h->f = (double *)calloc(9 * n, sizeof(double));
    h->g = (double *)calloc(9 * n, sizeof(double));
    h->rho = (double *)calloc(n, sizeof(double));
    h->psi = (double *)calloc(n, sizeof(double));
    h->sk_acc = (double *)calloc((size_t)(p->nx / 2 + 1) * p->ny, sizeof(double));
    h->sk_every = 0;
    if (!h->f || !h->g || !h->rho || !h->psi || !h->sk_acc) {
        free(h->f); free(h->g); free(h->rho); free(h->psi); free(h->sk_acc);
        free(h);
        return NULL;
    }
    return h;
}

void or_destroy(or_lattice *h) {
    if (!h) return;
    free(h->f); free(h->g); free(h->rho); free(h->psi); free(h->sk_acc);
    free(h);
}

/* Homogeneous density rho0 at rest (f = f^eq(rho0, 0) = w_i rho0), plus an
 * optional density kick rho0 + amp * z(site), z from Philox block 2. */
void or_init(or_lattice *h, double rho0, uint64_t seed, double init_amp) {
    h->p.rho0 = rho0;
    h->p.seed = seed;
    h->t = 0;
    int nx = h->p.nx, ny = h->p.ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double rho = rho0;
            if (init_amp != 0.0) {
                uint32_t r[4];
                double z0, z1;
                draw(&h->p, (uint32_t)(x + nx * y), 0, 2, r);
                box_muller(r[0], r[1], &z0, &z1);
                rho = rho0 + init_amp * z0;
            }
            for (int i = 0; i < 9; ++i) h->f[IDX(i, x, y, nx, ny)] = WQ[i] * rho;
        }
}

void or_set_replica(or_lattice *h, uint32_t replica) { h->p.replica = replica; }
void or_set_step(or_lattice *h, long long t) { h->t = t; }
long long or_get_step(const or_lattice *h) { return h->t; }

/* f = f^eq(rho(x), u = 0) = w_i rho(x). */
void or_set_density(or_lattice *h, const double *rho) {
    int nx = h->p.nx, ny = h->p.ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int i = 0; i < 9; ++i)
                h->f[IDX(i, x, y, nx, ny)] = WQ[i] * rho[x + (size_t)nx * y];
}

void or_set_populations(or_lattice *h, const double *f) {
    memcpy(h->f, f, sizeof(double) * 9 * (size_t)h->p.nx * h->p.ny);
}
void or_get_populations(const or_lattice *h, double *f) {
    memcpy(f, h->f, sizeof(double) * 9 * (size_t)h->p.nx * h->p.ny);
}

/* Density of the stored (post-collision) state: rho(x) = sum_i f_i(x). */
void or_density(const or_lattice *h, double *rho) {
    int nx = h->p.nx, ny = h->p.ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double s = 0.0;
            for (int i = 0; i < 9; ++i) s += h->f[IDX(i, x, y, nx, ny)];
            rho[x + (size_t)nx * y] = s;
        }
}

/* Total mass and momentum of the stored state. */
void or_conserved(const or_lattice *h, double out[3]) {
    int nx = h->p.nx, ny = h->p.ny;
    double m = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double v = h->f[IDX(i, x, y, nx, ny)];
                m += v;
                jx += CX[i] * v;
                jy += CY[i] * v;
            }
    out[0] = m; out[1] = jx; out[2] = jy;
}

/* Shan-Chen force of Eq. (1) at (x, y) from a full psi field. */
typedef struct stencil_t { int n; int ex[32], ey[32]; double w[32]; } stencil_t;

static void sc_force(const or_params *p, const stencil_t *st, const double *psi,
                     int x, int y, double *Fx, double *Fy) {
    int na = st->n;
    const int *ex = st->ex, *ey = st->ey;
    const double *w = st->w;
    int nx = p->nx, ny = p->ny;
    double sx = 0.0, sy = 0.0;
    for (int a = 0; a < na; ++a) {
        double pn = psi[wrap(x + ex[a], nx) + (size_t)nx * wrap(y + ey[a], ny)];
        sx += w[a] * pn * ex[a];
        sy += w[a] * pn * ey[a];
    }
    double pc = psi[x + (size_t)nx * y];
    *Fx = -p->G * CS2 * pc * sx;
    *Fy = -p->G * CS2 * pc * sy;
}

/* Force field of the stored state's density (diagnostic). */
void or_force_field(const or_lattice *h, double *Fx, double *Fy) {
    int nx = h->p.nx, ny = h->p.ny;
    double *rho = (double *)malloc(sizeof(double) * nx * (size_t)ny);
    double *psi = (double *)malloc(sizeof(double) * nx * (size_t)ny);
    stencil_t st;
    st.n = stencil_vectors(h->p.stencil, st.ex, st.ey, st.w);
    or_density(h, rho);
    for (size_t s = 0; s < (size_t)nx * ny; ++s) psi[s] = or_psi(&h->p, rho[s]);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            sc_force(&h->p, &st, psi, x, y, &Fx[x + (size_t)nx * y], &Fy[x + (size_t)nx * y]);
    free(rho);
    free(psi);
}

/* ------------------------------------------------------------------------ */
/* Structure factor: S(k) = |sum_x drho(x) e^{-i k.x}|^2 / N, drho = rho -   */
/* mean(rho), on the half plane kx = 0..nx/2, ky = 0..ny-1; k = 0 excluded.  */
/* Separable direct DFT (rows, then columns) with a table of e^{-2 pi i m/n}.*/
/* ------------------------------------------------------------------------ */
static void sk_sample(or_lattice *h) {
    int nx = h->p.nx, ny = h->p.ny, hx = nx / 2 + 1;
    size_t N = (size_t)nx * ny;
    double *rho = (double *)malloc(sizeof(double) * N);
    double *rr = (double *)malloc(sizeof(double) * (size_t)hx * ny);
    double *ri = (double *)malloc(sizeof(double) * (size_t)hx * ny);
    double *cx = (double *)malloc(sizeof(double) * nx), *sx = (double *)malloc(sizeof(double) * nx);
    double *cy = (double *)malloc(sizeof(double) * ny), *sy = (double *)malloc(sizeof(double) * ny);
    for (int m = 0; m < nx; ++m) { cx[m] = cos(2.0 * M_PI * m / nx); sx[m] = sin(2.0 * M_PI * m / nx); }
    for (int m = 0; m < ny; ++m) { cy[m] = cos(2.0 * M_PI * m / ny); sy[m] = sin(2.0 * M_PI * m / ny); }
    or_density(h, rho);
    double mean = 0.0;
    for (size_t s = 0; s < N; ++s) mean += rho[s];
    mean /= (double)N;
    for (size_t s = 0; s < N; ++s) rho[s] -= mean;
    /* rows: R(kx, y) = sum_x drho(x, y) e^{-2 pi i kx x / nx} */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int kx = 0; kx < hx; ++kx) {
            double re = 0.0, im = 0.0;
            for (int x = 0; x < nx; ++x) {
                int m = (int)(((long long)kx * x) % nx);
                re += rho[x + (size_t)nx * y] * cx[m];
                im -= rho[x + (size_t)nx * y] * sx[m];
            }
            rr[kx + (size_t)hx * y] = re;
            ri[kx + (size_t)hx * y] = im;
        }
    /* columns: X(kx, ky) = sum_y R(kx, y) e^{-2 pi i ky y / ny} */
#pragma omp parallel for schedule(static)
    for (int ky = 0; ky < ny; ++ky)
        for (int kx = 0; kx < hx; ++kx) {
            double re = 0.0, im = 0.0;
            for (int y = 0; y < ny; ++y) {
                int m = (int)(((long long)ky * y) % ny);
                double a = rr[kx + (size_t)hx * y], b = ri[kx + (size_t)hx * y];
                /* (a + i b)(cos - i sin) */
                re += a * cy[m] + b * sy[m];
                im += b * cy[m] - a * sy[m];
            }
            if (kx == 0 && ky == 0) continue;
            h->sk_acc[kx + (size_t)hx * ky] += (re * re + im * im) / (double)N;
        }
    h->sk_count += 1;
    free(rho); free(rr); free(ri); free(cx); free(sx); free(cy); free(sy);
}

/* Sample after completed step n when n >= start and (n - start) % every == 0. */
void or_sk_config(or_lattice *h, int every, long long start) {
    h->sk_every = every;
    h->sk_start = start;
}
void or_sk_reset(or_lattice *h) {
    memset(h->sk_acc, 0, sizeof(double) * (size_t)(h->p.nx / 2 + 1) * h->p.ny);
    h->sk_count = 0;
}
void or_sk_sample_now(or_lattice *h) { sk_sample(h); }
/* Mean S(k) over the samples, [ny][nx/2+1]; returns the sample count. */
long long or_sk_get(const or_lattice *h, double *out) {
    size_t n = (size_t)(h->p.nx / 2 + 1) * h->p.ny;
    for (size_t s = 0; s < n; ++s)
        out[s] = h->sk_count ? h->sk_acc[s] / (double)h->sk_count : 0.0;
    return h->sk_count;
}

/* ------------------------------------------------------------------------ */
/* One time step over the whole lattice.                                     */
/* ------------------------------------------------------------------------ */
static void step_once(or_lattice *h) {
    const or_params *p = &h->p;
    int nx = p->nx, ny = p->ny;
    stencil_t st;
    st.n = stencil_vectors(p->stencil, st.ex, st.ey, st.w);
    basis_setup();
    /* 1. pull streaming: g_i(x) = f_i(x - c_i), periodic */
    for (int i = 0; i < 9; ++i)
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                h->g[IDX(i, x, y, nx, ny)] =
                    h->f[IDX(i, wrap(x - CX[i], nx), wrap(y - CY[i], ny), nx, ny)];
    /* 2. density and pseudopotential on every site */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double s = 0.0;
            for (int i = 0; i < 9; ++i) s += h->g[IDX(i, x, y, nx, ny)];
            h->rho[x + (size_t)nx * y] = s;
            h->psi[x + (size_t)nx * y] = or_psi(p, s);
        }
    /* 3. force, collision, forcing and noise per site */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double g[9], out[9], Fx, Fy;
            for (int i = 0; i < 9; ++i) g[i] = h->g[IDX(i, x, y, nx, ny)];
            sc_force(p, &st, h->psi, x, y, &Fx, &Fy);
            collide_site(p, (uint32_t)(x + nx * y), (uint32_t)h->t, g, Fx, Fy, out);
            for (int i = 0; i < 9; ++i) h->f[IDX(i, x, y, nx, ny)] = out[i];
        }
    h->t += 1;
    if (h->sk_every > 0 && h->t >= h->sk_start &&
        (h->t - h->sk_start) % h->sk_every == 0)
        sk_sample(h);
}

int or_step(or_lattice *h, int n) {
    for (int s = 0; s < n; ++s) step_once(h);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One step evaluated only at the listed sites, from a full-lattice input    */
/* state f_in ([9][ny][nx], full populations) at step counter t.  Used to    */
/* check lattices too large for a whole oracle step: same arithmetic, with  */
/* rho and psi evaluated on demand for the sites the force needs.           */
/* ------------------------------------------------------------------------ */
static double density_after_streaming(const or_params *p, const double *f_in,
                                      int x, int y) {
    double s = 0.0;
    for (int i = 0; i < 9; ++i)
        s += f_in[IDX(i, wrap(x - CX[i], p->nx), wrap(y - CY[i], p->ny), p->nx, p->ny)];
    return s;
}

int or_step_sites(const or_params *p, long long t, const double *f_in,
                  int nsites, const int *xs, const int *ys, double *out) {
    int ex[32], ey[32];
    double w[32];
    int na = stencil_vectors(p->stencil, ex, ey, w);
    int nx = p->nx, ny = p->ny;
    for (int s = 0; s < nsites; ++s) {
        int x = xs[s], y = ys[s];
        if (x < 0 || x >= nx || y < 0 || y >= ny) return -1;
        double g[9];
        for (int i = 0; i < 9; ++i)
            g[i] = f_in[IDX(i, wrap(x - CX[i], nx), wrap(y - CY[i], ny), nx, ny)];
        double sxx = 0.0, syy = 0.0;
        for (int a = 0; a < na; ++a) {
            double pn = or_psi(p, density_after_streaming(p, f_in, wrap(x + ex[a], nx),
                                                          wrap(y + ey[a], ny)));
            sxx += w[a] * pn * ex[a];
            syy += w[a] * pn * ey[a];
        }
        double pc = or_psi(p, density_after_streaming(p, f_in, x, y));
        double Fx = -p->G * CS2 * pc * sxx, Fy = -p->G * CS2 * pc * syy;
        collide_site(p, (uint32_t)(x + nx * y), (uint32_t)t, g, Fx, Fy, out + 9 * (size_t)s);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Constants exported for the lattice-isotropy and stencil tests.            */
/* ------------------------------------------------------------------------ */
void or_lattice_constants(int cx[9], int cy[9], double w[9], double *cs2) {
    for (int i = 0; i < 9; ++i) { cx[i] = CX[i]; cy[i] = CY[i]; w[i] = WQ[i]; }
    *cs2 = CS2;
}
void or_moment_basis(double m[81], double b[9]) {
    for (int k = 0; k < 9; ++k) {
        b[k] = basis_norm(k);
        for (int i = 0; i < 9; ++i) m[9 * k + i] = basis(k, i);
    }
}
int or_stencil(int order, int *ex, int *ey, double *w) {
    return stencil_vectors(order, ex, ey, w);
}
void or_normals(const or_params *p, uint32_t site, uint32_t t, double z[6]) {
    uint32_t r[4];
    draw(p, site, t, 0, r);
    site_normals(r, z);
}
/* One ring Box-Muller pair from a radius word and an angle index. */
void or_box_muller_ring(uint32_t ra, uint32_t a, double z[2]) {
    box_muller_ring(ra, a, &z[0], &z[1]);
}

/* Threads the site loops run on (1 without OpenMP). */
int or_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
/* Set the threads of the site loops (timing on one core or all; ignored
 * without OpenMP). */
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
