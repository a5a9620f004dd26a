// Internal declarations shared by the ensemble translation units: the
// per-replica device records, the tile descriptors, the device clock and
// the launcher of the shared-memory-resident replica kernel.  Nothing here
// is part of the public ABI (include/lbsc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbsc_collide.cuh"

namespace lbsc {

// Per-replica state on the device.
struct EnsRep {
    float *buf[2];
    float *drho;
    float2 *spec;
    double *acc;
    const float2 *tw_x, *tw_y;
    int nx, ny, ldx, psi_kind;
    int noise;
    uint32_t replica;
    float rho0, force_pref, psi_c, psi_b, psi0, gamma;
    float c3a, c3b, c4a, c4b, c5a, c5b;
    float amp[6];
};   // single relaxation time per replica (BGK)
struct EnsTile {
    int r, x0, y0, y1;
};
struct EnsClock {
    uint32_t t;
    int cur;
    uint32_t done;
    uint32_t pad;
};
struct EnsKeys {
    uint32_t rk[20];
};

// Kernel parameters of one tile of replica R at step t (current buffer cur).
__device__ __forceinline__ void fill_tile_params(KParams<float> &sp, const EnsRep &R,
                                                 const EnsTile &tile, uint32_t t, int cur,
                                                 bool sample, int *flag) {
    sp.src = R.buf[cur];
    sp.dst = R.buf[cur ^ 1];
    sp.drho_out = sample ? R.drho : nullptr;
    sp.flag = flag;
    sp.nx = R.nx;
    sp.ny = R.ny;
    sp.strip_h = tile.y1 - tile.y0;
    sp.psi_kind = R.psi_kind;
    sp.noise = R.noise;
    sp.step = t;
    sp.clock = nullptr;
    sp.replica = R.replica;
    sp.rho0 = R.rho0;
    sp.force_pref = R.force_pref;
    sp.psi_c = R.psi_c;
    sp.psi_b = R.psi_b;
    sp.psi0 = R.psi0;
    sp.gamma = R.gamma;
    sp.gamma_b = R.gamma;
    sp.gamma_g = R.gamma;
    sp.c3a = R.c3a;
    sp.c3b = R.c3b;
    sp.c4a = R.c4a;
    sp.c4b = R.c4b;
    sp.c5a = R.c5a;
    sp.c5b = R.c5b;
    for (int k = 0; k < 6; ++k) sp.amp[k] = R.amp[k];
}

// Replicas small enough to live in shared memory for a whole window of
// steps: one CTA per replica, or a cluster of C CTAs sharing its rows
// through distributed shared memory.  All replicas of one launch have the
// same shape; the grid is nres * C CTAs.
struct ResLaunch {
    const EnsRep *reps;
    const int *list;        // replica indices of this shape, nres of them
    int nres;
    int nx, ny;             // the shape (nx in {32, 64, 128})
    int C;                  // CTAs per replica (cluster size: 1, 2, 4 or 8)
    int hb;                 // rows per band (one thread per column and band)
    int stencil;            // 4, 6, 8
    EnsClock *clk;
    int *flag;
    EnsKeys keys;
    int nsteps;
    int sample;             // the window's last step writes delta rho
};
// Dynamic shared memory of one CTA holding `rows` rows of nx columns in
// bands of hb rows, or 0 if the shape is not supported.
size_t resident_smem(int nx, int rows, int hb, int stencil);
// Opt the kernel of (stencil, C) in to `smem` bytes of dynamic shared memory.
cudaError_t resident_prepare(int stencil, int C, size_t smem);
// Clusters of C CTAs (CTAs per SM when C = 1) that can be resident at once.
int resident_max_clusters(int stencil, int C, int nx, int rows, int hb, size_t smem);
cudaError_t launch_ens_resident(const ResLaunch &a, cudaStream_t s);

}  // namespace lbsc
