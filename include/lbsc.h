/*
 * lbsc.h -- C ABI of the GB300 (sm_103a) fluctuating Shan-Chen D2Q9 lattice
 * Boltzmann library.
 *
 * Method: Lulli, Biferale, Falcucci, Sbragaglia, Yang and Shan, "Metastable
 * and Unstable Dynamics in multi-phase lattice Boltzmann" (arXiv:2212.07848).
 * One time step is the fluctuating lattice Boltzmann equation, Eq. (12):
 * pull streaming, BGK relaxation in moment space, Guo forcing of the
 * Shan-Chen force of Eq. (1), and Gaussian noise on the non-conserved
 * moments (the noise paragraph after Eq. (16)); the density structure
 * factor S(k) = <|delta n(k)|^2> (defined after Eq. (12)) is accumulated on
 * the device.
 *
 * Conventions shared by every entry point:
 *   - Lattice: periodic nx x ny, site index s = x + nx * y (x fastest).
 *     Host arrays of populations are [9][ny][nx] doubles in the velocity
 *     order 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1)
 *     7:(-1,-1) 8:(1,-1), weights 4/9, 1/9 (x4), 1/36 (x4), c_s^2 = 1/3.
 *   - Force: F = -G c_s^2 psi(x) sum_a w_a psi(x + e_a) e_a with the stencil
 *     weights normalised to sum_a w_a e_ax^2 = 1; G < 0 is attractive and the
 *     bulk pressure is p = rho c_s^2 + (G c_s^2 / 2) psi^2 (Eq. (2) with
 *     T = c_s^2).  For psi = 1 - exp(-rho) the critical point is
 *     rho_c = ln 2, G_c = -4.
 *   - Noise: each non-conserved Hermite moment k = 3..8 receives
 *     sqrt(mu rho b_k (1 - gamma^2)) z_k with mu = kT / c_s^2,
 *     gamma = 1 - 1/tau, rho the local density and z_k standard normals
 *     from Philox4x32-10 keyed by the 64-bit seed with counter
 *     (site, step, replica, block).
 *   - Ownership: the context owns every device buffer it allocates; the
 *     caller owns every host array passed in and must size it as stated.
 *   - Errors: every int-returning call returns LB_OK (0) or a negative
 *     LB_ERR_* code; nothing throws across the ABI and nothing aborts.
 *     Calls that synchronise report a non-finite state detected by the
 *     step kernel as LB_ERR_NONFINITE.
 *   - Streams: device work runs asynchronously on the context's stream
 *     (the caller's stream if one was given to lb_create_ex).  Calls that
 *     return host data synchronise that stream first.
 */
#ifndef LBSC_H
#define LBSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LB_OK 0
#define LB_ERR_ARG (-1)          /* invalid argument or size                */
#define LB_ERR_CUDA (-2)         /* a CUDA runtime call or launch failed    */
#define LB_ERR_NONFINITE (-3)    /* the step produced NaN or Inf            */
#define LB_ERR_TIMEOUT (-4)      /* a bounded device wait ran out           */
#define LB_ERR_UNSUPPORTED (-5)  /* valid request this build cannot serve   */
#define LB_ERR_IO (-6)           /* file open/read/write failed             */
#define LB_ERR_NOMEM (-7)        /* host or device allocation failed        */
#define LB_ERR_STATE (-8)        /* call out of order (e.g. step before init)*/

/* ---- pseudopotentials psi(rho) (p1, p2 are lb_params.psi_p1/psi_p2) ----- */
#define LB_PSI_EXP 0        /* psi = 1 - exp(-rho)                            */
#define LB_PSI_CRITICAL 1   /* psi = sqrt(Tc nc) exp(1 - nc/rho), Eq. (5);
                               p1 = Tc, p2 = nc                               */
#define LB_PSI_AEXP 2       /* psi = a exp(-b/rho) (the form before Eq. (3));
                               p1 = a, p2 = b                                 */

/* ---- storage precision of the populations --------------------------------- */
#define LB_FP32 0           /* deviations from w_i rho0 stored in FP32        */
#define LB_FP64 1           /* deviations stored in FP64                      */

/* ---- lb_device_ptr selectors -------------------------------------------- */
#define LB_PTR_POPULATIONS 0   /* current deviations [9][ny][nx] (T)        */
#define LB_PTR_DENSITY_SAMPLE 1/* last sampled delta rho [ny][nx] (T)       */
#define LB_PTR_SK_ACCUM 2      /* FP64 S(k) sums [ny][ldx], ldx = pad4(nx/2+1) */

typedef struct lb_ctx lb_ctx;

typedef struct lb_params {
    int nx, ny;          /* lattice size; multiples of 4, >= 4              */
    double G;            /* Shan-Chen coupling (G < 0 attractive)           */
    double tau;          /* BGK relaxation time, > 1/2                       */
    double kT;           /* fluctuation energy k_B theta, >= 0               */
    int psi_kind;        /* LB_PSI_*                                          */
    double psi_p1, psi_p2;
    int stencil;         /* force stencil isotropy order: 4, 6 or 8          */
    int precision;       /* LB_FP32 or LB_FP64                                */
    void *stream;        /* cudaStream_t to run on, or NULL for an owned one */
    int device;          /* CUDA device ordinal, or -1 for the current one   */
} lb_params;

/* Fill *p with defaults: 128x128, G = -3.6, tau = 1, kT = 0, LB_PSI_EXP,
 * E4, LB_FP32, own stream, current device.  Returns LB_ERR_ARG if p is NULL. */
int lb_params_init(lb_params *p);

/* Create a lattice context (FP32 storage, own stream, current device).
 * Step: Eq. (12) with the force of Eq. (1).  Sizes: nx, ny multiples of 4,
 * >= 4; tau > 1/2; kT >= 0; psi_kind LB_PSI_EXP/..; stencil 4, 6 or 8.
 * On success *out owns all device memory (about 2 x 9 x nx x ny x 4 bytes of
 * populations plus the S(k) buffers); free it with lb_destroy.
 * Errors: LB_ERR_ARG, LB_ERR_NOMEM, LB_ERR_CUDA (no usable GPU). */
int lb_create(lb_ctx **out, int nx, int ny, double G, double tau, double kT,
              int psi_kind, int stencil);

/* As lb_create with every parameter in *p (precision, stream, device). */
int lb_create_ex(lb_ctx **out, const lb_params *p);

/* Release the context and its device memory.  NULL is ignored. */
void lb_destroy(lb_ctx *h);

/* Homogeneous initial state of the paper's simulations (density n0 at rest,
 * periodic box; the simulation paragraph after Eq. (16)): f_i = w_i rho0, plus an
 * optional density kick rho0 + init_amp * z(site) with z from Philox block 2
 * of step 0.  Sets the Philox key to seed, the step counter to 0, and
 * clears S(k) sums.  rho0 > 0.  Errors: LB_ERR_ARG, LB_ERR_CUDA. */
int lb_init(lb_ctx *h, double rho0, uint64_t seed, double init_amp);

/* Philox counter word 2 (independent noise streams of replicas sharing a
 * seed).  Default 0. */
int lb_set_replica(lb_ctx *h, uint32_t replica);

/* Rows of the lattice swept by one CTA of the step kernel (launch-shape
 * tuning, 1 <= rows <= ny; the default depends on the lattice size).  Does
 * not change results. */
int lb_set_strip_height(lb_ctx *h, int rows);

/* Advance n >= 0 time steps of Eq. (12), asynchronously on the context
 * stream.  Sampling steps (lb_sk_config) also run the S(k) transform and
 * accumulation.  Returns the launch status (LB_ERR_CUDA if a launch failed,
 * LB_ERR_STATE before lb_init); NaN/Inf shows at the next synchronising
 * call. */
int lb_step(lb_ctx *h, int n);

/* Wait for the context stream; LB_ERR_NONFINITE if any step since the last
 * check produced a non-finite value (the flag is then cleared). */
int lb_sync(lb_ctx *h);

/* Completed steps since lb_init (or the value given to lb_set_step). */
long long lb_get_step(const lb_ctx *h);
int lb_set_step(lb_ctx *h, long long t);

/* Density rho(x) = sum_i f_i(x) of the current state into host_out[ny*nx]
 * (double, x fastest).  Synchronises. */
int lb_density(lb_ctx *h, double *host_out);

/* Full populations f_i = w_i rho0 + delta f_i into host_out[9*ny*nx]. */
int lb_populations(lb_ctx *h, double *host_out);

/* Replace the state by full populations host_in[9*ny*nx] (stored as
 * deviations from w_i rho0 in the context precision).  Requires lb_init. */
int lb_set_populations(lb_ctx *h, const double *host_in);

/* Replace the state by f_i = w_i rho(x) (rest) from host_rho[ny*nx]. */
int lb_set_density(lb_ctx *h, const double *host_rho);

/* Native-format state transfer: 9*ny*nx deviations in the context precision
 * (float for LB_FP32, double for LB_FP64).  Host memory may be pinned; the
 * copy runs on the context stream and these calls synchronise. */
int lb_upload_state(lb_ctx *h, const void *host_df);
int lb_download_state(lb_ctx *h, void *host_df);

/* S(k) sampling schedule: after completed step n, sample when
 * n >= start_step and (n - start_step) % sample_every == 0; sample_every = 0
 * turns sampling off.  Requires nx, ny powers of two (else
 * LB_ERR_UNSUPPORTED) and max(nx, ny) <= 8192 (FP32) / 4096 (FP64). */
int lb_sk_config(lb_ctx *h, int sample_every, long long start_step);

/* Clear the S(k) sums and the sample count. */
int lb_sk_reset(lb_ctx *h);

/* Sample S(k) from the current state now (outside the schedule). */
int lb_sk_sample_now(lb_ctx *h);

/* Mean structure factor S(k) = <|sum_x drho(x) e^{-ik.x}|^2> / (nx ny) over
 * the samples taken (k = 0 reported as 0).
 *   nbins == 0: host_out[ny * (nx/2+1)], ky-major half plane (kx = 0..nx/2).
 *   nbins  > 0: host_out[nbins], mean over the modes of the full plane with
 *               round(|k| / dk) == b, dk = 2 pi / max(nx, ny); empty bins NaN.
 * *nsamples_out (may be NULL) receives the sample count.  Synchronises. */
int lb_structure_factor(lb_ctx *h, double *host_out, int nbins,
                        long long *nsamples_out);

/* Number of full-plane modes in each radial bin of lb_structure_factor. */
int lb_structure_factor_counts(lb_ctx *h, long long *host_counts, int nbins);

/* Total mass sum rho and momentum sum j (FP64 device reduction, fixed
 * order, deterministic) into host out[3].  Synchronises. */
int lb_conserved(lb_ctx *h, double out[3]);

/* Checkpoint: parameters, step counter, seed, replica, populations and the
 * S(k) sums.  Because the noise is counter-based, a loaded run continues
 * bit-identically.  lb_load requires a context of the same size and
 * precision.  Errors: LB_ERR_IO, LB_ERR_ARG (mismatch). */
int lb_save(lb_ctx *h, const char *path);
int lb_load(lb_ctx *h, const char *path);

/* Device pointer to a context buffer (LB_PTR_*), valid until lb_destroy;
 * NULL for a bad selector.  The population buffer changes after each step. */
void *lb_device_ptr(lb_ctx *h, int which);

/* The cudaStream_t the context runs on. */
void *lb_stream(lb_ctx *h);

/* Allocation-free mass and momentum sums, for callers that must not call
 * cudaMalloc: a host application whose device memory all comes from its own
 * pool, or a loop that cannot take the device-wide synchronisation an
 * allocation brings.  The paper has no counterpart; this is a library
 * service.  Inputs: d_df, device pointer to deviations [9][ny][nx] in the
 * given precision (the layout of LB_PTR_POPULATIONS) and rho0, their
 * reference density.  Output: d_out3, a caller-owned device array of 3
 * doubles receiving (nx*ny*rho0 + sum delta rho, sum jx, sum jy), written
 * asynchronously on `stream` (cudaStream_t, NULL for the default stream).
 * Scratch: a fixed 96 KB device array inside the library (4096 partial
 * triples), held on every GPU that loads the library until the process
 * exits; lattices above 4096 x 4096 = 16,777,216 sites return
 * LB_ERR_UNSUPPORTED.  Every call shares that array and leaves its partial
 * sums there; each call rewrites every slot it reads, so nothing needs
 * clearing, but calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The first call on a
 * device looks up the array's device address (make that first call before
 * any stream capture).  Nothing here allocates device or host memory.
 * Errors: LB_ERR_ARG, LB_ERR_UNSUPPORTED, LB_ERR_CUDA. */
int lb_conserved_static(const void *d_df, int precision, int nx, int ny, double rho0,
                        double *d_out3, void *stream);

/* Static message for a status code. */
const char *lb_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LBSC_H */
