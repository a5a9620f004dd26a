/*
 * Plain FP64 CPU oracle of the fluctuating Shan-Chen lattice Boltzmann step
 * in three dimensions (D3Q19): the paper's own setting (its Eq. (12) is
 * written for 3D, with the noise on the moments a > 3 of the noise
 * paragraph after Eq. (16)).  TEST INFRASTRUCTURE ONLY: the test suite and
 * the benchmark's CPU legs use it to check the CUDA path; the product never
 * loads it, and it shares no code with the CUDA sources.
 *
 * Written for clarity, not speed: full populations f_i, a separate streamed
 * copy, density and pseudopotential fields, then per site the force, the
 * population-space BGK collision with Guo forcing, and the noise projected
 * from moment space explicitly.
 *
 * Readings (the paper names no 3D lattice; listed in the design notes):
 *   - lattice D3Q19, c_s^2 = 1/3, weights 1/3, 1/18 (axes), 1/36 (face
 *     diagonals), velocity order: rest; +x, -x, +y, -y, +z, -z; then the
 *     diagonals of the xy, xz and yz planes as (+,+), (-,-), (+,-), (-,+);
 *   - moment basis: the 19 polynomials 1, cx, cy, cz, c^2-1, 3cx^2-c^2,
 *     cy^2-cz^2, cxcy, cycz, czcx, (3c^2-5)cx, (3c^2-5)cy, (3c^2-5)cz,
 *     (cy^2-cz^2)cx, (cz^2-cx^2)cy, (cx^2-cy^2)cz, 3c^4-6c^2+1,
 *     (2c^2-3)(3cx^2-c^2), (2c^2-3)(cy^2-cz^2), orthogonal under the weights;
 *     modes 0..3 conserved, 4..18 carry noise of variance mu rho b_k (1-gamma^2);
 *   - pseudopotential: the three forms of the 2D oracle, 1 - exp(-rho) (kind 0),
 *     Eq. (5) sqrt(Tc nc) exp(1 - nc/rho) (kind 1) and a exp(-b/rho) (kind 2);
 *   - force stencil (Eq. (1)): the 18 D3Q19 neighbours with w = 1/6 (axes) and
 *     1/12 (diagonals), normalised to sum_a w_a e_ax^2 = 1 (fourth-order
 *     isotropic), so p = rho c_s^2 + (G c_s^2 / 2) psi^2 as in 2D;
 *   - random numbers: Philox4x32-10, counter (site, step, replica, block),
 *     site = x + nx (y + ny z); blocks 0 and 1 give the 15 normals by the ring
 *     Box-Muller, one pair per 32-bit word (radius from the high 22 bits, angle
 *     index from the low 10): block 0 -> modes 4..11, block 1 -> modes 12..17
 *     and 18 (cosine of its last pair); block 3 of step 0 drives the optional
 *     initial density kick (plain Box-Muller pair (r0, r1));
 *   - S(k) on the three lattice axes: S(k e_a) = |sum_x drho(x) e^{-i k x_a}|^2 / N
 *     with drho = rho - mean(rho), k = 2 pi m / n_a, m = 1 .. n_a/2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Philox4x32-10 of the 2D oracle file (same library). */
void or_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out);

static const int C3[19][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double CS2 = 1.0 / 3.0;

static double w3(int i) {
    int c2 = C3[i][0] * C3[i][0] + C3[i][1] * C3[i][1] + C3[i][2] * C3[i][2];
    return c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

/* The moment polynomials of the reading above, evaluated at velocity i. */
static double basis3(int k, int i) {
    double x = C3[i][0], y = C3[i][1], z = C3[i][2];
    double c2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return c2 - 1.0;
    case 5: return 3.0 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return z * x;
    case 10: return (3.0 * c2 - 5.0) * x;
    case 11: return (3.0 * c2 - 5.0) * y;
    case 12: return (3.0 * c2 - 5.0) * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
    case 17: return (2.0 * c2 - 3.0) * (3.0 * x * x - c2);
    case 18: return (2.0 * c2 - 3.0) * (y * y - z * z);
    }
    return 0.0;
}

static double E3[19][19], B3[19], W3[19];
static int ready3 = 0;
static void setup3(void) {
    if (ready3) return;
    for (int i = 0; i < 19; ++i) W3[i] = w3(i);
    for (int k = 0; k < 19; ++k) {
        double b = 0.0;
        for (int i = 0; i < 19; ++i) {
            E3[k][i] = basis3(k, i);
            b += W3[i] * E3[k][i] * E3[k][i];
        }
        B3[k] = b;
    }
    ready3 = 1;
}

typedef struct or3_params {
    int nx, ny, nz;
    double G, tau, kT;
    double rho0;
    uint64_t seed;
    uint32_t replica;
    int psi_kind;            /* 0: 1-exp(-rho); 1: sqrt(Tc nc) exp(1-nc/rho) (Eq. (5));
                                2: a exp(-b/rho) */
    double psi_p1, psi_p2;   /* kind 1: (Tc, nc); kind 2: (a, b) */
} or3_params;

/* The pseudopotential of the chosen kind (the same three forms as in 2D). */
static double psi3(const or3_params *p, double rho) {
    switch (p->psi_kind) {
    case 1: return sqrt(p->psi_p1 * p->psi_p2) * exp(1.0 - p->psi_p2 / rho);
    case 2: return p->psi_p1 * exp(-p->psi_p2 / rho);
    default: return 1.0 - exp(-rho);
    }
}

static void draw3(const or3_params *p, uint32_t site, uint32_t step, uint32_t block,
                  uint32_t out[4]) {
    uint32_t ctr[4] = {site, step, p->replica, block};
    uint32_t key[2] = {(uint32_t)(p->seed & 0xffffffffu), (uint32_t)(p->seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

static double unif(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

/* One ring pair from a single word: the radius from its high 22 bits,
 * u = ((w >> 10) + 1/2) 2^-22, the angle index from its low 10 bits. */
static void ring_pair22(uint32_t w, double *z0, double *z1) {
    double u = ((double)(w >> 10) + 0.5) * (1.0 / 4194304.0);
    double rad = sqrt(-2.0 * log(u));
    double th = 2.0 * M_PI * ((double)(w & 1023u) + 0.5) / 1024.0;
    *z0 = rad * cos(th);
    *z1 = rad * sin(th);
}

/* The 15 thermal normals of a site and step: z[k - 4] for modes k = 4..18,
 * one ring pair per Philox word: block 0 words 0..3 -> modes (4,5), (6,7),
 * (8,9), (10,11); block 1 words 0..2 -> (12,13), (14,15), (16,17), word 3 ->
 * mode 18 (the cosine of its pair). */
static void site_normals3(const or3_params *p, uint32_t site, uint32_t t, double z[15]) {
    uint32_t r[4];
    double s;
    draw3(p, site, t, 0, r);
    for (int j = 0; j < 4; ++j) ring_pair22(r[j], &z[2 * j], &z[2 * j + 1]);
    draw3(p, site, t, 1, r);
    for (int j = 0; j < 3; ++j) ring_pair22(r[j], &z[8 + 2 * j], &z[9 + 2 * j]);
    ring_pair22(r[3], &z[14], &s);
}

static inline int wrap3(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}
#define IDX3(i, x, y, z, p) \
    ((((size_t)(i) * (size_t)(p)->nz + (size_t)(z)) * (size_t)(p)->ny + (size_t)(y)) * (size_t)(p)->nx + (size_t)(x))
#define SITE3(x, y, z, p) (((size_t)(z) * (size_t)(p)->ny + (size_t)(y)) * (size_t)(p)->nx + (size_t)(x))

/* Post-collision populations of one site (population-space BGK with Guo
 * forcing, noise projected from the moments 4..18). */
static void collide3(const or3_params *p, uint32_t site, uint32_t t, const double g[19],
                     const double F[3], double out[19]) {
    setup3();
    double rho = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < 19; ++i) {
        rho += g[i];
        for (int a = 0; a < 3; ++a) j[a] += C3[i][a] * g[i];
    }
    double u[3], usq = 0.0;
    for (int a = 0; a < 3; ++a) {
        u[a] = (j[a] + 0.5 * F[a]) / rho;
        usq += u[a] * u[a];
    }
    double tau = p->tau, gam = 1.0 - 1.0 / tau, mu = p->kT / CS2;
    double N[19] = {0};
    if (p->kT > 0.0) {
        double z[15];
        site_normals3(p, site, t, z);
        for (int k = 4; k < 19; ++k) N[k] = sqrt(mu * rho * B3[k] * (1.0 - gam * gam)) * z[k - 4];
    }
    for (int i = 0; i < 19; ++i) {
        double cu = 0.0, sF = 0.0;
        for (int a = 0; a < 3; ++a) cu += C3[i][a] * u[a];
        double feq = W3[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - usq / (2.0 * CS2));
        for (int a = 0; a < 3; ++a)
            sF += ((C3[i][a] - u[a]) / CS2 + cu * C3[i][a] / (CS2 * CS2)) * F[a];
        double src = (1.0 - 1.0 / (2.0 * tau)) * W3[i] * sF;
        double eta = 0.0;
        for (int k = 4; k < 19; ++k) eta += E3[k][i] * N[k] / B3[k];
        out[i] = g[i] - (g[i] - feq) / tau + src + W3[i] * eta;
    }
}

typedef struct or3_lattice {
    or3_params p;
    long long t;
    double *f, *g, *psi;
    int sk_every;
    long long sk_start, sk_count;
    double *sk_acc;   /* [nx/2 + ny/2 + nz/2]: x-axis modes, then y, then z */
    double *sk_full;  /* NULL, or [nz][ny][nx] sums of |delta rho(k)|^2 / N over every k */
} or3_lattice;

or3_lattice *or3_create(const or3_params *p) {
    if (p->nx < 2 || p->ny < 2 || p->nz < 2) return NULL;
    or3_lattice *h = (or3_lattice *)calloc(1, sizeof(or3_lattice));
    if (!h) return NULL;
    h->p = *p;
    size_t n = (size_t)p->nx * p->ny * p->nz;
    h->f = (double *)calloc(19 * n, sizeof(double));
    h->g = (double *)calloc(19 * n, sizeof(double));
    h->psi = (double *)calloc(n, sizeof(double));
    h->sk_acc = (double *)calloc((size_t)(p->nx / 2 + p->ny / 2 + p->nz / 2), sizeof(double));
    if (!h->f || !h->g || !h->psi || !h->sk_acc) {
        free(h->f); free(h->g); free(h->psi); free(h->sk_acc); free(h);
        return NULL;
    }
    return h;
}

void or3_destroy(or3_lattice *h) {
    if (!h) return;
    free(h->f); free(h->g); free(h->psi); free(h->sk_acc); free(h->sk_full); free(h);
}

void or3_init(or3_lattice *h, double rho0, uint64_t seed, double amp) {
    setup3();
    h->p.rho0 = rho0;
    h->p.seed = seed;
    h->t = 0;
    const or3_params *p = &h->p;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double rho = rho0;
                if (amp != 0.0) {
                    uint32_t r[4];
                    draw3(p, (uint32_t)SITE3(x, y, z, p), 0, 3, r);
                    double rad = sqrt(-2.0 * log(unif(r[0])));
                    rho = rho0 + amp * rad * cos(2.0 * M_PI * unif(r[1]));
                }
                for (int i = 0; i < 19; ++i) h->f[IDX3(i, x, y, z, p)] = W3[i] * rho;
            }
}

void or3_set_replica(or3_lattice *h, uint32_t r) { h->p.replica = r; }
long long or3_get_step(const or3_lattice *h) { return h->t; }
void or3_set_populations(or3_lattice *h, const double *f) {
    memcpy(h->f, f, sizeof(double) * 19 * (size_t)h->p.nx * h->p.ny * h->p.nz);
}
void or3_get_populations(const or3_lattice *h, double *f) {
    memcpy(f, h->f, sizeof(double) * 19 * (size_t)h->p.nx * h->p.ny * h->p.nz);
}

void or3_density(const or3_lattice *h, double *rho) {
    const or3_params *p = &h->p;
    size_t n = (size_t)p->nx * p->ny * p->nz;
    for (size_t s = 0; s < n; ++s) {
        double v = 0.0;
        for (int i = 0; i < 19; ++i) v += h->f[(size_t)i * n + s];
        rho[s] = v;
    }
}

void or3_conserved(const or3_lattice *h, double out[4]) {
    const or3_params *p = &h->p;
    size_t n = (size_t)p->nx * p->ny * p->nz;
    double m = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < 19; ++i)
        for (size_t s = 0; s < n; ++s) {
            double v = h->f[(size_t)i * n + s];
            m += v;
            for (int a = 0; a < 3; ++a) j[a] += C3[i][a] * v;
        }
    out[0] = m; out[1] = j[0]; out[2] = j[1]; out[3] = j[2];
}

/* Axis modes of S(k): direct sums over the whole lattice. */
static void sk_sample3(or3_lattice *h) {
    const or3_params *p = &h->p;
    size_t n = (size_t)p->nx * p->ny * p->nz;
    double *rho = (double *)malloc(sizeof(double) * n);
    or3_density(h, rho);
    double mean = 0.0;
    for (size_t s = 0; s < n; ++s) mean += rho[s];
    mean /= (double)n;
    int dims[3] = {p->nx, p->ny, p->nz}, off = 0;
    for (int a = 0; a < 3; ++a) {
        int L = dims[a];
        for (int m = 1; m <= L / 2; ++m) {
            double re = 0.0, im = 0.0;
            for (int z = 0; z < p->nz; ++z)
                for (int y = 0; y < p->ny; ++y)
                    for (int x = 0; x < p->nx; ++x) {
                        int c = a == 0 ? x : (a == 1 ? y : z);
                        double ph = 2.0 * M_PI * (double)(((long long)m * c) % L) / L;
                        double d = rho[SITE3(x, y, z, p)] - mean;
                        re += d * cos(ph);
                        im -= d * sin(ph);
                    }
            h->sk_acc[off + m - 1] += (re * re + im * im) / (double)n;
        }
        off += L / 2;
    }
    if (h->sk_full) {
        /* every wave vector: the 3D DFT of delta rho by three separable passes
         * (x, then y, then z), each the plain sum of its definition */
        int nx = p->nx, ny = p->ny, nz = p->nz;
        double *ar = (double *)calloc(n, sizeof(double)), *ai = (double *)calloc(n, sizeof(double));
        double *br = (double *)calloc(n, sizeof(double)), *bi = (double *)calloc(n, sizeof(double));
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int k = 0; k < nx; ++k) {
                    double re = 0.0, im = 0.0;
                    for (int x = 0; x < nx; ++x) {
                        double ph = 2.0 * M_PI * (double)(((long long)k * x) % nx) / nx;
                        double d = rho[SITE3(x, y, z, p)] - mean;
                        re += d * cos(ph);
                        im -= d * sin(ph);
                    }
                    ar[SITE3(k, y, z, p)] = re;
                    ai[SITE3(k, y, z, p)] = im;
                }
        for (int z = 0; z < nz; ++z)
            for (int k = 0; k < ny; ++k)
                for (int x = 0; x < nx; ++x) {
                    double re = 0.0, im = 0.0;
                    for (int y = 0; y < ny; ++y) {
                        double ph = 2.0 * M_PI * (double)(((long long)k * y) % ny) / ny;
                        double c = cos(ph), sn = sin(ph);
                        double vr = ar[SITE3(x, y, z, p)], vi = ai[SITE3(x, y, z, p)];
                        re += vr * c + vi * sn;
                        im += vi * c - vr * sn;
                    }
                    br[SITE3(x, k, z, p)] = re;
                    bi[SITE3(x, k, z, p)] = im;
                }
        for (int k = 0; k < nz; ++k)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    double re = 0.0, im = 0.0;
                    for (int z = 0; z < nz; ++z) {
                        double ph = 2.0 * M_PI * (double)(((long long)k * z) % nz) / nz;
                        double c = cos(ph), sn = sin(ph);
                        double vr = br[SITE3(x, y, z, p)], vi = bi[SITE3(x, y, z, p)];
                        re += vr * c + vi * sn;
                        im += vi * c - vr * sn;
                    }
                    h->sk_full[SITE3(x, y, k, p)] += (re * re + im * im) / (double)n;
                }
        free(ar); free(ai); free(br); free(bi);
    }
    h->sk_count += 1;
    free(rho);
}

/* Full 3D S(k) on the sampling steps (every wave vector; cleared here). */
int or3_sk_full(or3_lattice *h, int enable) {
    const or3_params *p = &h->p;
    free(h->sk_full);
    h->sk_full = NULL;
    if (enable) {
        h->sk_full = (double *)calloc((size_t)p->nx * p->ny * p->nz, sizeof(double));
        if (!h->sk_full) return -1;
    }
    return 0;
}
/* Mean over the samples of the full S(k), out [nz][ny][nx] (k = 0 included as
 * sampled: zero, since the mean is removed). */
long long or3_sk_full_get(const or3_lattice *h, double *out) {
    const or3_params *p = &h->p;
    size_t n = (size_t)p->nx * p->ny * p->nz;
    for (size_t s = 0; s < n; ++s)
        out[s] = (h->sk_full && h->sk_count) ? h->sk_full[s] / (double)h->sk_count : 0.0;
    return h->sk_count;
}

void or3_sk_config(or3_lattice *h, int every, long long start) {
    h->sk_every = every;
    h->sk_start = start;
}
long long or3_sk_get(const or3_lattice *h, double *out) {
    int nb = h->p.nx / 2 + h->p.ny / 2 + h->p.nz / 2;
    for (int b = 0; b < nb; ++b) out[b] = h->sk_count ? h->sk_acc[b] / (double)h->sk_count : 0.0;
    return h->sk_count;
}

static void step3(or3_lattice *h) {
    const or3_params *p = &h->p;
    int nx = p->nx, ny = p->ny, nz = p->nz;
    size_t n = (size_t)nx * ny * nz;
    setup3();
    /* 1. pull streaming: g_i(x) = f_i(x - c_i), periodic */
    for (int i = 0; i < 19; ++i)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x)
                    h->g[IDX3(i, x, y, z, p)] = h->f[IDX3(i, wrap3(x - C3[i][0], nx),
                                                          wrap3(y - C3[i][1], ny),
                                                          wrap3(z - C3[i][2], nz), p)];
    /* 2. density and pseudopotential on every site */
    for (size_t s = 0; s < n; ++s) {
        double v = 0.0;
        for (int i = 0; i < 19; ++i) v += h->g[(size_t)i * n + s];
        h->psi[s] = psi3(p, v);
    }
    /* 3. force (Eq. (1) with the D3Q19 neighbours), collision, noise */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double g[19], out[19], S[3] = {0, 0, 0}, F[3];
                size_t s = SITE3(x, y, z, p);
                for (int i = 0; i < 19; ++i) g[i] = h->g[(size_t)i * n + s];
                for (int a = 1; a < 19; ++a) {
                    double wa = C3[a][0] * C3[a][0] + C3[a][1] * C3[a][1] + C3[a][2] * C3[a][2] == 1
                                    ? 1.0 / 6.0 : 1.0 / 12.0;
                    double pn = h->psi[SITE3(wrap3(x + C3[a][0], nx), wrap3(y + C3[a][1], ny),
                                             wrap3(z + C3[a][2], nz), p)];
                    for (int b = 0; b < 3; ++b) S[b] += wa * pn * C3[a][b];
                }
                for (int b = 0; b < 3; ++b) F[b] = -p->G * CS2 * h->psi[s] * S[b];
                collide3(p, (uint32_t)s, (uint32_t)h->t, g, F, out);
                for (int i = 0; i < 19; ++i) h->f[(size_t)i * n + s] = out[i];
            }
    h->t += 1;
    if (h->sk_every > 0 && h->t >= h->sk_start && (h->t - h->sk_start) % h->sk_every == 0)
        sk_sample3(h);
}

/* One step evaluated at chosen sites only, from a full-lattice input state
 * f_in [19][nz][ny][nx] (full populations) at step t: the same pull, density,
 * pseudopotential, force and collision as step3, with the density of each
 * force neighbour computed on demand.  For checking large lattices site by
 * site.  Returns -1 if a site is out of range. */
static double density3_after_streaming(const or3_params *p, const double *f_in, int x, int y,
                                       int z) {
    double s = 0.0;
    for (int i = 0; i < 19; ++i)
        s += f_in[IDX3(i, wrap3(x - C3[i][0], p->nx), wrap3(y - C3[i][1], p->ny),
                       wrap3(z - C3[i][2], p->nz), p)];
    return s;
}

int or3_step_sites(const or3_params *p, long long t, const double *f_in, int nsites,
                   const int *xs, const int *ys, const int *zs, double *out) {
    setup3();
    int nx = p->nx, ny = p->ny, nz = p->nz;
    for (int k = 0; k < nsites; ++k) {
        int x = xs[k], y = ys[k], z = zs[k];
        if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) return -1;
        double g[19], S[3] = {0, 0, 0}, F[3];
        for (int i = 0; i < 19; ++i)
            g[i] = f_in[IDX3(i, wrap3(x - C3[i][0], nx), wrap3(y - C3[i][1], ny),
                             wrap3(z - C3[i][2], nz), p)];
        for (int a = 1; a < 19; ++a) {
            double wa = C3[a][0] * C3[a][0] + C3[a][1] * C3[a][1] + C3[a][2] * C3[a][2] == 1
                            ? 1.0 / 6.0 : 1.0 / 12.0;
            double pn = psi3(p, density3_after_streaming(p, f_in, wrap3(x + C3[a][0], nx),
                                                         wrap3(y + C3[a][1], ny),
                                                         wrap3(z + C3[a][2], nz)));
            for (int b = 0; b < 3; ++b) S[b] += wa * pn * C3[a][b];
        }
        double pc = psi3(p, density3_after_streaming(p, f_in, x, y, z));
        for (int b = 0; b < 3; ++b) F[b] = -p->G * CS2 * pc * S[b];
        collide3(p, (uint32_t)SITE3(x, y, z, p), (uint32_t)t, g, F, out + 19 * (size_t)k);
    }
    return 0;
}

int or3_step(or3_lattice *h, int nsteps) {
    for (int s = 0; s < nsteps; ++s) step3(h);
    return 0;
}

/* Shan-Chen force of Eq. (1) with the D3Q19 E4 neighbours, for the stored
 * state's density (diagnostic): F [3][nz][ny][nx]. */
void or3_force_field(const or3_lattice *h, double *F) {
    const or3_params *p = &h->p;
    int nx = p->nx, ny = p->ny, nz = p->nz;
    size_t n = (size_t)nx * ny * nz;
    double *rho = (double *)malloc(sizeof(double) * n), *ps = (double *)malloc(sizeof(double) * n);
    or3_density(h, rho);
    for (size_t s = 0; s < n; ++s) ps[s] = psi3(p, rho[s]);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double S[3] = {0, 0, 0};
                for (int a = 1; a < 19; ++a) {
                    double wa = C3[a][0] * C3[a][0] + C3[a][1] * C3[a][1] + C3[a][2] * C3[a][2] == 1
                                    ? 1.0 / 6.0 : 1.0 / 12.0;
                    double pn = ps[SITE3(wrap3(x + C3[a][0], nx), wrap3(y + C3[a][1], ny),
                                         wrap3(z + C3[a][2], nz), p)];
                    for (int b = 0; b < 3; ++b) S[b] += wa * pn * C3[a][b];
                }
                size_t s = SITE3(x, y, z, p);
                for (int b = 0; b < 3; ++b) F[(size_t)b * n + s] = -p->G * CS2 * ps[s] * S[b];
            }
    free(rho);
    free(ps);
}

/* Lattice tables for the tests: velocities [19][3], weights, basis [19][19], norms. */
void or3_lattice_constants(int c[57], double w[19]) {
    setup3();
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = C3[i][a];
        w[i] = W3[i];
    }
}
void or3_moment_basis(double m[361], double b[19]) {
    setup3();
    for (int k = 0; k < 19; ++k) {
        b[k] = B3[k];
        for (int i = 0; i < 19; ++i) m[19 * k + i] = E3[k][i];
    }
}
/* One ring pair from a single word (the 3D mapping: 22-bit radius, 10-bit angle). */
void or3_ring_pair22(uint32_t w, double z[2]) { ring_pair22(w, &z[0], &z[1]); }

void or3_normals(const or3_params *p, uint32_t site, uint32_t t, double z[15]) {
    site_normals3(p, site, t, z);
}
