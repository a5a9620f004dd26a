// Internal declarations shared by the translation units of liblbsc.so.
// Nothing here is part of the public ABI (include/lbsc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbsc {

// Launch shape of the fused step: one thread per lattice column inside a
// strip of kStepTX columns; each CTA sweeps strip_h rows of its strip.
constexpr int kStepTX = 128;

// Bits of the device status flag read by lb_sync.
constexpr int LB_STEP_NONFINITE = 1;
constexpr int LB_STEP_TIMEOUT = 2;

// Opaque storage for the CUDA tensor maps (CUtensorMap, 128 bytes each) of
// the two FP32 population buffers: row loads (136 columns x 9 planes) and
// row stores (128 columns x 9 planes).
struct TmaMaps {
    alignas(64) unsigned char load[2][128];
    alignas(64) unsigned char store[2][128];
    bool ok = false;
};

// Parameters of one fused time step (Eq. (12) with the force of Eq. (1)).
// Floating-point values are converted to the storage precision in the kernel.
struct StepArgs {
    const void *src;      // deviations delta f* [9][ny][nx] at time t
    void *dst;            // deviations delta f* [9][ny][nx] at time t+1
    void *drho_out;       // delta rho [ny][nx] of the new state, or nullptr
    int *flag;            // LB_STEP_* bits (non-finite value, wait timeout)
    int nx, ny;
    int strip_h;          // rows swept by one CTA
    double rho0;          // reference density of the stored deviations
    double force_pref;    // -G c_s^2
    double psi_kind;      // 0, 1, 2 (kept as double for packing)
    double psi_c;         // kind 0: exp(-rho0); kinds 1, 2: psi(rho0)
    double psi_b;         // kinds 1, 2: b (nc or b); unused for kind 0
    double psi0;          // psi(rho0)
    double gamma;         // 1 - 1/tau of the shear modes 4, 5
    double gamma_b;       // 1 - 1/tau_bulk of mode 3
    double gamma_g;       // 1 - 1/tau_ghost of modes 6, 7, 8
    double noise_amp[6];  // sqrt(mu b_k (1 - gamma_k^2)), k = 3..8 (times sqrt(rho))
    uint32_t round_keys[20];  // Philox4x32-10 key schedule (k0, k1) per round
    uint32_t step;        // counter word 1: number of completed steps
    uint32_t replica;     // counter word 2
    int noise;            // kT > 0
    long long wait_ns;    // staged kernel: bound on an mbarrier wait (< 0: default)
    int layout;           // plain kernel: 0 = halo warp, 1 = overlapped strips
    const uint32_t *clock;  // device step counter: the noise counter is *clock + step (or null)
};

// FFT / structure-factor buffers of one lattice.
struct SkArgs {
    const void *drho;     // [ny][nx] real input (storage precision)
    void *spec;           // complex [ny][ldx] half spectrum (storage precision)
    double *acc;          // [ny][ldx] running sum of |X|^2 / N
    const void *tw_x;     // complex table e^{-2 pi i m / nx}, m < nx/2
    const void *tw_y;     // complex table e^{-2 pi i m / ny}, m < ny/2
    int nx, ny, ldx;
};

cudaError_t launch_step(int precision, int stencil, const StepArgs &a, cudaStream_t s);
bool tma_eligible(int precision, int nx, int ny);
bool tma_encode_maps(TmaMaps *m, void *buf0, void *buf1, int nx, int ny);
// src_buf: index (0/1) of the buffer holding the current state.
cudaError_t launch_step_tma(int stencil, const StepArgs &a, const TmaMaps &m, int src_buf,
                            cudaStream_t s);
cudaError_t launch_init(int precision, void *df, int nx, int ny, double amp,
                        const uint32_t round_keys[20], uint32_t replica, cudaStream_t s);
cudaError_t launch_density(int precision, const void *df, double rho0, double *out,
                           int nx, int ny, cudaStream_t s);
cudaError_t launch_drho(int precision, const void *df, void *drho, int nx, int ny,
                        cudaStream_t s);
cudaError_t launch_sk_sample(int precision, const SkArgs &a, cudaStream_t s);
cudaError_t launch_twiddles(int precision, void *tw, int n, cudaStream_t s);
cudaError_t launch_sk_readout(const double *acc, double inv_count, double *out, int nx,
                              int ny, int ldx, cudaStream_t s);
cudaError_t launch_sk_bins(const double *acc, double inv_count, double *bins, double *counts,
                           int nbins, int nx, int ny, int ldx, cudaStream_t s);
cudaError_t launch_sk_moments(const double *acc, double inv_count, int nx, int ny, int ldx,
                              double *out2, cudaStream_t s);
cudaError_t launch_conserved(int precision, const void *df, double *partials, int nblocks,
                             double *out3, int nx, int ny, cudaStream_t s);
int conserved_blocks(int nx, int ny);

// Philox4x32-10 key schedule for a 64-bit seed (k0 = low word, k1 = high).
void philox_round_keys(uint64_t seed, uint32_t rk[20]);

}  // namespace lbsc
