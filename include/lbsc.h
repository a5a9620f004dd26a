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
#define LB_ERR_UNSUPPORTED (-5)  /* valid request this library cannot serve */
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

/* ---- step kernel selection (lb_set_kernel) -------------------------------- */
#define LB_KERNEL_AUTO 0    /* the fastest kernel for this GPU and lattice: on
                               GB300 overlap for nx >= 1024, else plain          */
#define LB_KERNEL_PLAIN 1   /* coalesced global loads; strips of 128 columns and a
                               fifth warp for the halo columns' pseudopotential   */
#define LB_KERNEL_TMA 2     /* rows staged in shared memory by cp.async.bulk.tensor
                               (FP32 and nx a multiple of 128 only)               */
#define LB_KERNEL_OVERLAP 3 /* coalesced global loads; strips of 128 - 2H columns
                               whose halo columns are pulled by the CTA's own
                               threads (no separate halo warp)                    */

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
    double tau_bulk;     /* relaxation time of the bulk mode 3 (> 1/2), or 0 for tau */
    double tau_ghost;    /* relaxation time of the ghost modes 6-8 (> 1/2), or 0 for tau;
                            tau itself relaxes the shear modes 4-5.  All equal: the BGK
                            collision named after Eq. (12); otherwise the
                            multiple-relaxation-time variant with the same forcing
                            and fluctuation-dissipation noise per mode */
} lb_params;

/* Fill *p with defaults: 128x128, G = -3.6, tau = 1 (BGK: tau_bulk =
 * tau_ghost = 0), kT = 0, LB_PSI_EXP, E4, LB_FP32, own stream, current
 * device.  Returns LB_ERR_ARG if p is NULL. */
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

/* Choose the step kernel (LB_KERNEL_*).  All kernels perform the same
 * arithmetic per site and give the same results; they differ only in how rows
 * reach the SM and how the pseudopotential halo is exchanged.
 * LB_ERR_UNSUPPORTED if the requested kernel cannot serve the lattice
 * (LB_KERNEL_TMA: FP32 and nx % 128 == 0).
 * lb_get_kernel returns the kernel lb_step uses. */
int lb_set_kernel(lb_ctx *h, int mode);
int lb_get_kernel(const lb_ctx *h);

/* Bound, in nanoseconds of the device's global timer, on each mbarrier wait
 * of the staged kernel (LB_KERNEL_TMA) for a row copy to land (failure
 * detection).  ns < 0 restores the default of 2 s; ns = 0 makes a wait give
 * up at the first check that finds its copy in flight.  On a timeout every
 * thread of the CTA leaves through the same barrier, the CTA waits (with the
 * default bound) for the copies it issued, and lb_sync returns
 * LB_ERR_TIMEOUT; the steps launched since the last good sync are then
 * incomplete and the state must be restored (lb_init, lb_load or
 * lb_set_populations) before it is used again.  Errors: LB_ERR_ARG. */
int lb_set_wait_ns(lb_ctx *h, long long ns);

/* Advance n >= 0 time steps of Eq. (12), asynchronously on the context
 * stream.  Sampling steps (lb_sk_config) also run the S(k) transform and
 * accumulation.  Windows of 32 steps without a sampling step, and sampling
 * intervals ending with their sample, replay CUDA graphs captured on first
 * use (the step counter of the noise read from device memory; recaptured
 * after any setter that changes what they hold); other steps, the staged
 * kernel and streams that cannot be captured use single launches, with the
 * same results.  Returns the launch status (LB_ERR_CUDA if a launch failed,
 * LB_ERR_STATE before lb_init); NaN/Inf shows at the next synchronising
 * call. */
int lb_step(lb_ctx *h, int n);

/* Wait for the context stream; LB_ERR_NONFINITE if any step since the last
 * check produced a non-finite value, LB_ERR_TIMEOUT if a bounded device wait
 * of the staged kernel ran out (the flag is then cleared). */
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

/* First moments of the mean S(k) over the full plane, k = 0 excluded:
 * out[0] = sum_k S(k), out[1] = sum_k |k| S(k).  The characteristic domain
 * size of a coarsening quench is L = 2 pi out[0] / out[1] (a definition of
 * this library; the paper does not define L).  Synchronises. */
int lb_sk_moments(lb_ctx *h, double out[2]);

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
 * any stream capture) and keeps it for the life of the process: after a
 * cudaDeviceReset, or anything else that destroys the device's primary
 * context, the kept address is stale and this entry point must not be called
 * again on that device until the library is reloaded.  Nothing here
 * allocates device or host memory.
 * Errors: LB_ERR_ARG, LB_ERR_UNSUPPORTED, LB_ERR_CUDA. */
int lb_conserved_static(const void *d_df, int precision, int nx, int ny, double rho0,
                        double *d_out3, void *stream);

/* ---- batched ensembles ---------------------------------------------------
 * Many independent periodic lattices of uneven size, coupling and density
 * advanced together (the ensembles behind the S(k) statistics near the
 * critical point and the spinodal, Figs. 2-3 and the simulation paragraph).
 * One launch per step covers every replica (a tile list over all of them);
 * runs of steps are replayed from captured CUDA graphs.  FP32 storage.
 * Replica r draws its noise from Philox with key = seed and counter word 2 =
 * r, so it evolves exactly like a single lattice created with the same
 * parameters, lb_init(rho0, seed, amp) and lb_set_replica(r). */
typedef struct lb_ens lb_ens;

typedef struct lb_replica {
    int nx, ny;          /* multiples of 4 (powers of two for S(k))          */
    double G, tau, kT;   /* coupling, relaxation time (> 1/2), k_B theta      */
    double rho0;         /* homogeneous initial density (> 0)                 */
} lb_replica;

/* Create an ensemble of nrep (1..65536) replicas sharing the pseudopotential
 * and force stencil.  Memory: 2 x 9 x 4 bytes per site of every replica.
 * Errors: LB_ERR_ARG, LB_ERR_NOMEM, LB_ERR_CUDA. */
int lb_ens_create(lb_ens **out, const lb_replica *reps, int nrep, int psi_kind, double psi_p1,
                  double psi_p2, int stencil, uint64_t seed, void *stream);
void lb_ens_destroy(lb_ens *e);
/* Every replica to rho0_r at rest plus the optional Philox kick (block 2). */
int lb_ens_init(lb_ens *e, double init_amp);
/* Per-replica S(k) schedule, as lb_sk_config (all sizes powers of two). */
int lb_ens_sk_config(lb_ens *e, int sample_every, long long start_step);
/* Rows swept per CTA for every replica (tile shape). */
int lb_ens_set_strip_height(lb_ens *e, int rows);
/* Time candidate strip heights on a snapshot of the state (restored after),
 * keep the fastest, and cache it in cache_path ("key strip" lines; may be
 * NULL).  *chosen (may be NULL) receives the strip height. */
int lb_ens_autotune(lb_ens *e, int trial_steps, const char *cache_path, int *chosen);
/* How lb_ens_step launches the steps.  LB_ENS_PER_STEP: one launch per step
 * over every replica's tiles.  LB_ENS_PERSISTENT: each window of steps
 * (32 plain steps, or one S(k) sampling interval) is one cooperative
 * persistent launch whose CTAs take (step, tile) pairs in order from a
 * counter; a tile waits (bounded, 2 s) until the tiles it pulls from (its
 * neighbours within the stencil's reach, and itself) finished the previous
 * step; a timeout makes the next sync return LB_ERR_TIMEOUT.  A window's sampling step runs as a per-step launch.  Both
 * give the same bits.  LB_ERR_UNSUPPORTED if the device cannot launch
 * cooperatively. */
#define LB_ENS_PER_STEP 0
#define LB_ENS_PERSISTENT 1
int lb_ens_set_launch(lb_ens *e, int mode);
int lb_ens_get_launch(const lb_ens *e);
/* Bound, in nanoseconds of the device's global timer, on each dependency
 * wait of the persistent launch (failure detection, the bounded waits of a
 * persistent kernel).  ns < 0 restores the default of 2 s; ns = 0 makes a
 * wait give up at the first check that finds a tile it pulls from unfinished
 * with the previous step.  On a timeout the waiting CTA records it, every
 * other CTA stops at its next wait, the launch ends, and lb_ens_sync returns
 * LB_ERR_TIMEOUT; the replicas' state is then partly advanced and must be
 * re-initialised (lb_ens_init) before it is used again.  Synchronises the
 * ensemble's stream.  Errors: LB_ERR_ARG, LB_ERR_CUDA. */
int lb_ens_set_wait_ns(lb_ens *e, long long ns);
/* Strip layout of the ensemble's step kernels, as lb_set_kernel:
 * LB_KERNEL_PLAIN (128-column strips and a halo warp) or LB_KERNEL_OVERLAP
 * (strips of 128 - 2H columns whose halo the CTA's own threads pull);
 * LB_KERNEL_AUTO takes the faster one on this GPU.  Same results either way.
 * Synchronises the ensemble's stream and rebuilds the tile list.
 * lb_ens_get_kernel returns the layout in use.  Errors: LB_ERR_ARG, LB_ERR_CUDA. */
int lb_ens_set_kernel(lb_ens *e, int mode);
int lb_ens_get_kernel(const lb_ens *e);
/* Replicas resident in shared memory (the batched step of Eq. (12) kept on
 * chip for a window of steps).  A replica with nx in {32, 64, 128} whose
 * rows split into C = 1, 2, 4 or 8 equal parts of at most 4096 sites (64^2:
 * one CTA; 128^2: a cluster of four CTAs reading each other's boundary rows
 * through distributed shared memory) can live in shared memory for a whole
 * window of steps, reading and writing HBM only at the window's ends (and
 * delta rho at a sampling step).  LB_ENS_RESIDENT_OFF: none.
 * LB_ENS_RESIDENT_ON: every replica whose shape allows it; the others run
 * as tiles after them.  LB_ENS_RESIDENT_AUTO (the default): all replicas
 * when each fits one CTA (C = 1), else none.  Same bits as the tile path.
 * Synchronises the ensemble's stream and rebuilds the tile list.
 * lb_ens_num_resident returns how many replicas are resident.
 * Errors: LB_ERR_ARG, LB_ERR_CUDA. */
#define LB_ENS_RESIDENT_OFF 0
#define LB_ENS_RESIDENT_ON 1
#define LB_ENS_RESIDENT_AUTO 2
int lb_ens_set_resident(lb_ens *e, int mode);
int lb_ens_num_resident(const lb_ens *e);
/* Advance every replica n steps (asynchronous); windows of steps replay
 * captured CUDA graphs. */
int lb_ens_step(lb_ens *e, int n);
int lb_ens_sync(lb_ens *e);
long long lb_ens_get_step(const lb_ens *e);
int lb_ens_num_tiles(const lb_ens *e);
/* Read-outs of replica r, layouts as the single-lattice calls. */
int lb_ens_populations(lb_ens *e, int r, double *host_out);
int lb_ens_density(lb_ens *e, int r, double *host_out);
int lb_ens_conserved(lb_ens *e, int r, double out[3]);
int lb_ens_structure_factor(lb_ens *e, int r, double *host_out, int nbins,
                            long long *nsamples_out);

/* ---- three dimensions: D3Q19 ---------------------------------------------
 * The paper's own setting: Eq. (12) on a D3Q19 lattice (c_s^2 = 1/3; weights
 * 1/3, 1/18, 1/36; velocity order: rest; +x, -x, +y, -y, +z, -z; then the
 * face diagonals of the xy, xz and yz planes as (+,+), (-,-), (+,-), (-,+)),
 * psi of kind LB_PSI_* (default 1 - exp(-rho)), the Shan-Chen force of Eq. (1) over the 18 neighbours
 * with weights 1/6 (axes) and 1/12 (diagonals), BGK collision with Guo
 * forcing in the 19-moment basis (1, c, c^2-1, 3cx^2-c^2, cy^2-cz^2, cxcy,
 * cycz, czcx, (3c^2-5)c, (cy^2-cz^2)cx, (cz^2-cx^2)cy, (cx^2-cy^2)cz,
 * 3c^4-6c^2+1, (2c^2-3)(3cx^2-c^2), (2c^2-3)(cy^2-cz^2)), and noise
 * sqrt(mu rho b_k (1 - gamma^2)) z_k on the 15 modes k = 4..18 (the noise
 * paragraph after Eq. (16): modes a > 3), z from Philox4x32-10 blocks 0-2 of
 * counter (site, step, replica, block), site = x + nx (y + ny z).
 * Storage: deviations [19][nz][ny][nx], FP32 or FP64; the context owns its
 * device memory.  nx % 32 == 0, ny % 4 == 0, nz >= 3, 19 nx ny nz < 2^32,
 * tau > 1/2, kT >= 0 (LB_ERR_ARG otherwise).  Calls are asynchronous on the
 * context's stream except the read-outs, which synchronise. */
typedef struct lb3_ctx lb3_ctx;
int lb3_create(lb3_ctx **out, int nx, int ny, int nz, double G, double tau, double kT,
               int precision, void *stream);
void lb3_destroy(lb3_ctx *h);
/* Homogeneous rho0 at rest, plus an optional density kick init_amp z(site)
 * from Philox block 3 of step 0. */
int lb3_init(lb3_ctx *h, double rho0, uint64_t seed, double init_amp);
/* Pseudopotential (LB_PSI_*, parameters as in lb_params; default
 * LB_PSI_EXP); takes effect from the next step. */
int lb3_set_psi(lb3_ctx *h, int psi_kind, double psi_p1, double psi_p2);
int lb3_set_replica(lb3_ctx *h, uint32_t replica);
/* z planes marched by one CTA (performance only). */
int lb3_set_strip(lb3_ctx *h, int planes);
int lb3_step(lb3_ctx *h, int n);
int lb3_sync(lb3_ctx *h);
long long lb3_get_step(const lb3_ctx *h);
/* rho [nz][ny][nx] and full populations f [19][nz][ny][nx] (host, FP64). */
int lb3_density(lb3_ctx *h, double *host_out);
int lb3_populations(lb3_ctx *h, double *host_out);
int lb3_set_populations(lb3_ctx *h, const double *host_f);
/* Total mass and momentum (FP64). */
int lb3_conserved(lb3_ctx *h, double out[4]);
/* S(k) on the three lattice axes, sampled after completed step n when
 * n >= start and (n - start) % every == 0: S(k e_a) = |sum_x drho(x)
 * e^{-i k x_a}|^2 / N for k = 2 pi m / n_a, m = 1 .. n_a/2.  The read-out
 * host_out [nx/2 + ny/2 + nz/2] holds the means over the samples (x modes,
 * then y, then z); LB_ERR_STATE before lb3_sk_config. */
int lb3_sk_config(lb3_ctx *h, int every, long long start);
int lb3_sk_reset(lb3_ctx *h);
int lb3_structure_factor_axes(lb3_ctx *h, double *host_out, long long *nsamples_out);
/* The full S(k) in 3D (the structure factor defined after Eq. (12) on every
 * wave vector of the box): with enable != 0 each sampling step of
 * lb3_sk_config also transforms the density sample in three dimensions
 * (FFTs along x, y, z) and adds |delta rho(k)|^2 / N to FP64 sums over the
 * half spectrum (device memory about nz ny (nx/2+1) x 16 bytes, allocated on
 * the first call).  Call after lb3_sk_config(every > 0) (LB_ERR_STATE
 * otherwise); nx, ny, nz must be powers of two (LB_ERR_UNSUPPORTED
 * otherwise).  The sums are cleared by lb3_sk_reset and lb3_init. */
int lb3_sk_full(lb3_ctx *h, int enable);
/* Radial means of the full S(k) over the samples: host_bins[b], b = 0 ..
 * nbins-1, is the mean over the modes with round(|q|) = b, q_a = m_a max(n) /
 * n_a (m_a the folded wave-number index on axis a), k = 0 excluded; 0 for
 * empty shells.  *nsamples_out (may be NULL) = number of samples.
 * Synchronises.  LB_ERR_STATE without lb3_sk_full. */
int lb3_structure_factor(lb3_ctx *h, double *host_bins, int nbins, long long *nsamples_out);
/* First moments of the mean full S(k): out[0] = sum_k S(k), out[1] =
 * sum_k |k| S(k) over all k != 0 (|k| = 2 pi |(m_x/nx, m_y/ny, m_z/nz)|), so
 * the domain size is L = 2 pi out[0] / out[1].  Synchronises. */
int lb3_sk_moments(lb3_ctx *h, double *host_out2);

/* ---- learned surrogate building blocks ---------------------------------------
 * A small convolutional operator advances the 4x coarse-grained density of a
 * quench by a fixed stride; it is trained on trajectories of the solver
 * above, which stays its reference.  The paper has no such part.  All tensors
 * are caller-owned device buffers; activations are BF16 NHWC
 * [nb][h][w][c] with periodic boundaries, parameters FP32 with BF16 copies.
 * Calls are asynchronous on `stream` (cudaStream_t or NULL).
 *
 * 3x3 convolution on tensor cores (BF16 inputs, FP32 accumulation):
 *   dgrad = 0: y = act(bias + conv(x, w)), w [9][cout][cin] (tap-major,
 *              tap = 3 (dy+1) + (dx+1)), bias [cout] or NULL, act = ReLU if relu;
 *   dgrad = 1: the input gradient dx [..][cout] of a forward layer with
 *              weights w [9][cin][cout] from dy [..][cin] (bias NULL, relu 0).
 * Requires h * w % 128 == 0 and channel counts multiples of 16.  For w % 128
 * == 0 and 16/32/64/128 channels both cases run on the tcgen05 tensor cores
 * in a persistent kernel (accumulators in tensor memory, weights and input
 * rows staged by TMA); otherwise on mma.sync (the forward case with 32 or 64
 * input channels on a per-tile tcgen05 kernel when lb_nn_set_conv_path(2)). */
int lb_nn_conv3x3(const void *x, const void *w, const float *bias, void *y, int nb, int h, int w_,
                  int cin, int cout, int relu, int dgrad, void *stream);
/* Weight and bias gradients, accumulated (+=) into FP32 dw [9][cout][cin] and
 * dbias [cout] (may be NULL): dw[tap][n][c] += sum_p x[p + off(tap)][c] dy[p][n].
 * The sum is split over chunks of 128-pixel tiles whose partial sums go to the
 * caller's device workspace (16-byte aligned, at least
 * lb_nn_wgrad_workspace(...) bytes, which also holds the bias partials) and
 * are then added in a fixed order, so dw and dbias are deterministic (the same
 * inputs give the same bits).  Where image rows are a multiple of 128 pixels
 * and both channel counts are 16, 32, 64 or 128 the sums run on the tensor
 * cores (tcgen05; lb_nn_set_conv_path(1) forces the mma.sync kernel).
 * Requires h * w % 128 == 0, channel counts multiples of 16 and x, dy 16-byte
 * aligned (LB_ERR_ARG otherwise, or for a missing/short workspace). */
size_t lb_nn_wgrad_workspace(int nb, int h, int w_, int cin, int cout);
int lb_nn_conv3x3_wgrad(const void *x, const void *dy, float *dw, float *dbias, int nb, int h,
                        int w_, int cin, int cout, void *workspace, size_t workspace_bytes,
                        void *stream);
/* dz = dy where y > 0, else 0 (ReLU backward through the layer output y). */
int lb_nn_relu_mask(const void *dy, const void *y, void *dz, size_t n, void *stream);
/* 2x2 average pooling of [nb][h][w][c] (backward: spread dy/4). */
int lb_nn_pool2(const void *x, void *y, int nb, int h, int w_, int c, int backward, void *stream);
/* Nearest 2x upsampling of [nb][h][w][c] (backward: sum of the 2x2 block). */
int lb_nn_up2(const void *x, void *y, int nb, int h, int w_, int c, int backward, void *stream);
/* y = a + b elementwise (n values). */
int lb_nn_add(const void *a, const void *b, void *y, size_t n, void *stream);
/* Coarse-grained density of a lattice state: FP32 out [ny/f][nx/f] = (mean of
 * rho - rho0 over each f x f block) / scale, from FP32 deviations df [9][ny][nx]
 * (the populations buffer of an LB_FP32 lattice).  LB_ERR_ARG unless f divides
 * nx and ny and scale != 0. */
int lb_nn_coarse_grain(const float *df, int nx, int ny, int f, double scale, float *out,
                       void *stream);
/* Coarse-grained momentum of the same state: FP32 jx, jy [ny/f][nx/f] = (mean
 * of sum_i c_i df_i over each f x f block) / scale, the post-collision
 * momentum of the stored populations.  LB_ERR_ARG as lb_nn_coarse_grain. */
int lb_nn_coarse_momentum(const float *df, int nx, int ny, int f, double scale, float *jx,
                          float *jy, void *stream);
/* One more input channel: out[.][ch] = BF16(src[.]) and, with prev (may be
 * NULL), out[.][ch + 2] = BF16(src - prev), the layout lb_nn_residual keeps
 * (value at ch, last increment at ch + 2) when it is given out + ch.  Other
 * channels are untouched.  LB_ERR_ARG unless ch (and ch + 2 with prev) < c. */
int lb_nn_expand_channel(const float *src, const float *prev, void *out, int c, int ch, size_t n,
                         void *stream);
/* dst[.][dch] += src[.][sch] for BF16 buffers dst [n][dc] and src [n][sc]
 * (gradients gathered from several paths).  LB_ERR_ARG for a bad channel. */
int lb_nn_add_channel(void *dst, int dc, int dch, const void *src, int sc, int sch, size_t n,
                      void *stream);
/* Block MSE of the residual d = base + y[.][0] - target over images
 * [nb][h][w]: *loss += weight * mean over block x block tiles of (tile mean
 * of d)^2, a measure of the error at wavelengths longer than the tile; dy
 * (may be NULL) gets its gradient ADDED to channel 0 (call after lb_nn_mse,
 * which overwrites dy).  LB_ERR_ARG unless block divides h and w. */
int lb_nn_mse_blocks(const void *y, int c, const float *target, const float *base, int nb, int h,
                     int w_, int block, double weight, float *loss, void *dy, void *stream);
/* Weighted residual MSE of channel ch: prediction = base + y[.][ch];
 * *loss += weight * mean((prediction - target)^2); dy (may be NULL) gets
 * the gradient in channel ch only, every other channel of dy is untouched
 * (so several channels' losses add up after lb_nn_mse has zeroed the rest). */
int lb_nn_mse_channel(const void *y, int c, int ch, const float *target, const float *base,
                      size_t n, double weight, float *loss, void *dy, void *stream);
/* Residual MSE over n pixels: prediction = base + y[.][0] (FP32 base, BF16 y
 * [n][c]); *loss += mean((prediction - target)^2) (accumulates: zero it first);
 * dy (may be NULL) [n][c] = d loss / d y: 2 (prediction - target) / n on
 * channel 0, 0 elsewhere. */
int lb_nn_mse(const void *y, int c, const float *target, const float *base, size_t n, float *loss,
              void *dy, void *stream);
/* Rollout update: FP32 state [n] += y[.][0] - m, channel 0 of the network
 * input x [n][cx] = BF16(state), channel 2 (when cx > 2) = the increment just
 * applied, other channels of x untouched.  With mean_buf (a caller-owned
 * device buffer of at least 513 floats, or NULL for m = 0) m is the mean of
 * y[.][0] over the n pixels, written to mean_buf[0] first (mean_buf[1..] holds
 * partial sums; fixed summation order): the increment then has zero mean and
 * the field's mass is conserved as the lattice conserves it. */
int lb_nn_residual(float *state, const void *y, int c, void *x, int cx, size_t n, float *mean_buf,
                   void *stream);
/* Adam step (bias-corrected, `step` >= 1) on FP32 w with gradient g and moments
 * m, v; w_bf16 (may be NULL) receives the BF16 copy. */
int lb_nn_adam(float *w, const float *g, float *m, float *v, void *w_bf16, size_t n, double lr,
               double b1, double b2, double eps, long long step, void *stream);
/* Network input from an FP32 field src [n]: out [n][c] with channel 0 =
 * BF16(src), channel 1 = gfeat (the coupling feature), channel 2 =
 * BF16(src - prev) (the field's last increment; 0 when prev is NULL), others 0. */
int lb_nn_expand(const float *src, const float *prev, double gfeat, void *out, int c, size_t n,
                 void *stream);
/* Process-wide choice of the convolution kernel: 0 = automatic (default),
 * 1 = mma.sync always, 2 = the per-tile tcgen05 forward kernel wherever it
 * has one, 3 = the persistent tcgen05 kernel (forward and input gradient;
 * weights staged once per CTA, a ring of input rows, double-buffered tensor
 * memory) wherever it has one. */
int lb_nn_set_conv_path(int path);
/* Synchronises the device and reports whether a tensor-core convolution gave
 * up waiting on its mbarrier since the last call: LB_ERR_TIMEOUT (the flag is
 * then cleared), LB_ERR_CUDA if tensor memory had to be left allocated (see
 * lb_nn_set_wait_ns), or LB_OK. */
int lb_nn_status(void);
/* Bound, in nanoseconds of the device's global timer, on the tensor-core
 * convolution's wait for its MMAs (current device, process-wide).  ns < 0
 * restores the default of 1 s; ns = 0 makes the wait give up at the first
 * check that finds the MMAs unfinished.  On a timeout the CTA skips its
 * output tile, records the timeout for lb_nn_status, waits (with the
 * default bound) for the MMAs it committed, and only then frees its tensor
 * memory; if even that wait runs out it leaves the tensor memory allocated
 * and lb_nn_status returns LB_ERR_CUDA (the process should then be
 * restarted).  Errors: LB_ERR_CUDA. */
int lb_nn_set_wait_ns(long long ns);
/* BF16 copy of FP32 values. */
int lb_nn_to_bf16(const float *a, void *b, size_t n, void *stream);
/* Increment as the divergence of a predicted flux, so that the surrogate
 * conserves mass locally as the lattice does (the continuity equation behind
 * Eq. (12)'s conserved density): forward (backward = 0) reads J = (y[.][0],
 * y[.][1]) from BF16 y [nb][h][w][c] and writes BF16 out [nb][h][w]
 *   out[i][j] = -(Jx[i][j] - Jx[i][j-1] + Jy[i][j] - Jy[i-1][j])
 * (periodic wrap); backward (1) reads BF16 d out [nb][h][w] and writes the
 * adjoint into BF16 dy [nb][h][w][c] (channels 0 and 1; the others 0).
 * LB_ERR_ARG unless c >= 2 and the sizes are positive. */
int lb_nn_flux_div(const void *in, void *out, int c, int nb, int h, int w_, int backward,
                   void *stream);

/* Static message for a status code. */
const char *lb_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LBSC_H */
