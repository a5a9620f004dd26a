// Batched ensembles: many independent periodic lattices of uneven size,
// coupling G, density rho0 (and optionally tau, kT) advanced together.
//
// Statistics of S(k) near the critical point and the spinodal (the scaling
// of Figs. 2-3 of arXiv:2212.07848) need many independent realisations; one
// small lattice cannot fill a GB300 and a launch per replica per step is
// launch-bound.  Here every step of every replica is one launch over a tile
// list (replica, strip of 128 - 2H columns, row strip) sorted largest
// replica first (the overlapped layout of the single-lattice kernel: 128
// threads per CTA pull the strip and its halo columns);
// each CTA copies its replica's parameters into shared memory and runs the
// same per-strip code as the single-lattice kernel, so a replica evolves
// bit-identically to a single lattice with the same seed and replica index.
// The step counter and the current-buffer index live on the device and are
// advanced by the last CTA to finish, so a captured CUDA graph of several
// steps can be replayed for any step range.  S(k) of all replicas is sampled
// by batched FFT kernels over (replica, row pair) and (replica, column tile)
// descriptors.  An autotuner times candidate strip heights on a snapshot of
// the state and caches the choice.  Alternatively (lb_ens_set_launch) a
// window of steps runs as one persistent cooperative launch with per-replica
// completion barriers, captured in the same graphs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "lbsc.h"
#include "lbsc_fft.cuh"
#include "lbsc_ens.cuh"
#include "lbsc_internal.cuh"
#include "lbsc_strip.cuh"

namespace lbsc {
namespace {

// OV: the overlapped layout (kStepTX threads, strips of kStepTX - 2H
// columns); otherwise strips of kStepTX columns and a halo warp.
template <int ORDER, bool OV>
__global__ void __launch_bounds__(OV ? kStepTX : kStepTX + 32, OV ? (ORDER == 4 ? 8 : 5)
                                                                  : (ORDER == 4 ? 6 : 4))
ens_step_kernel(const EnsRep *__restrict__ reps, const EnsTile *__restrict__ tiles, int ntiles,
                EnsClock *clk, int *flag, const EnsKeys keys, int sk_every, long long sk_start) {
    __shared__ KParams<float> sp;
    __shared__ int s_sample;
    __shared__ uint32_t s_t;
    __shared__ int s_cur;
    const EnsTile tile = tiles[blockIdx.x];
    if (threadIdx.x == 0) {
        const uint32_t t = __ldcg(&clk->t);
        const int cur = __ldcg(&clk->cur);
        const EnsRep &R = reps[tile.r];
        const long long tn = (long long)t + 1;
        const bool sample =
            R.drho && sk_every > 0 && tn >= sk_start && (tn - sk_start) % sk_every == 0;
        fill_tile_params(sp, R, tile, t, cur, sample, flag);
        s_sample = sample ? 1 : 0;
        s_t = t;
        s_cur = cur;
    }
    __syncthreads();
    // replicas with every relaxation rate 1 (tau = 1) take the unit path,
    // which keeps only the conserved moments of the pulled rows
    const bool unit = sp.gamma == 0.f;
    if (OV) {
        if (unit) {
            if (s_sample) step_strip_ov<float, ORDER, true, false, true>(sp, keys.rk, tile.x0, tile.y0, tile.y1);
            else step_strip_ov<float, ORDER, false, false, true>(sp, keys.rk, tile.x0, tile.y0, tile.y1);
        } else {
            if (s_sample) step_strip_ov<float, ORDER, true>(sp, keys.rk, tile.x0, tile.y0, tile.y1);
            else step_strip_ov<float, ORDER, false>(sp, keys.rk, tile.x0, tile.y0, tile.y1);
        }
    } else {
        if (unit) {
            if (s_sample) step_strip<float, ORDER, true, false, true>(sp, keys.rk, tile.x0, tile.y0, tile.y1);
            else step_strip<float, ORDER, false, false, true>(sp, keys.rk, tile.x0, tile.y0, tile.y1);
        } else {
            if (s_sample) step_strip<float, ORDER, true>(sp, keys.rk, tile.x0, tile.y0, tile.y1);
            else step_strip<float, ORDER, false>(sp, keys.rk, tile.x0, tile.y0, tile.y1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        // every CTA read the clock before finishing, so the last one to
        // finish may advance it
        if (atomicAdd(&clk->done, 1u) == (uint32_t)ntiles - 1) {
            clk->done = 0;
            clk->t = s_t + 1;
            clk->cur = s_cur ^ 1;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// Persistent variant: one cooperative launch advances every replica by
// `nsteps` steps.  The (step, tile) pairs are handed out in order, step-major,
// from one atomic counter: a CTA that finishes a tile takes the next pair, so
// the work balances itself across CTAs and the tiles of step s + 1 start
// while the last tiles of step s run.  A tile at step s may start once the
// tiles whose cells it pulls (itself and its neighbours within the stencil's
// reach) have finished step s - 1 (per-tile completion counters, bounded
// wait): they wrote what it reads, and its stores overwrite what they read.
// Those pairs were handed out earlier, so the waits always end.
// The buffers alternate inside the launch, so pulls go through L2
// (ld.global.cg), not the read-only path.  The last CTA to finish resets the
// counters and advances the device clock.
// ---------------------------------------------------------------------------
struct EnsCtl {
    uint32_t finished;
    int abort;
    unsigned long long wait_ns;   // bound on a replica barrier (lb_ens_set_wait_ns)
    uint32_t next;                // next (step, tile) pair to hand out
};
constexpr uint64_t kEnsWaitNs = 2000000000ull;   // default: 2 s

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ens_global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait, as one warp, until counter nbr[q0 + q] of tdone reaches target for
// every q < cnt: lane l checks q = l, l + 32, ... and the warp decides
// together (one round trip to L2 per check, not one per counter).  Every
// lane returns 1 when they did, 0 when another CTA aborted, -1 on a timeout;
// a limit of 0 gives up at the first check that finds a counter short.
__device__ int wait_tiles(const uint32_t *tdone, const int *__restrict__ nbr, int q0, int cnt,
                          uint32_t target, const int *abort, uint64_t limit_ns) {
    const int lane = threadIdx.x & 31;
    auto ready = [&]() {
        bool ok = true;
        for (int q = lane; q < cnt; q += 32) ok = ok && ld_acquire_u32(&tdone[nbr[q0 + q]]) >= target;
        return __all_sync(0xffffffffu, ok);
    };
    if (ready()) return 1;
    if (limit_ns == 0) return -1;
    const uint64_t t0 = ens_global_ns();
    for (;;) {
        if (ready()) return 1;
        int stop = 2;   // lane 0 decides: 0 another CTA aborted, -1 timed out
        if (lane == 0) {
            if (*(volatile const int *)abort) stop = 0;
            else if (ens_global_ns() - t0 > limit_ns) stop = -1;
        }
        stop = __shfl_sync(0xffffffffu, stop, 0);
        if (stop != 2) return stop;
        __nanosleep(100);
    }
}

// UM: 1 every replica takes the unit path (all rates 1), 0 none does, 2 each
// replica by its own rates.  One strip variant per kernel (two for UM 2):
// more inlined variants in the loop push the strip past the register budget
// the launch bounds leave, and it spills.  The persistent launch never
// samples; a sampling step runs through the per-step kernel.
template <int ORDER, bool OV, int UM>
__global__ void __launch_bounds__(OV ? kStepTX : kStepTX + 32, OV ? (ORDER == 4 ? 8 : 5)
                                                                  : (ORDER == 4 ? 6 : 4))
ens_persist_kernel(const EnsRep *__restrict__ reps, const EnsTile *__restrict__ tiles,
                   int ntiles, const int *__restrict__ nbr_off, const int *__restrict__ nbr,
                   uint32_t *tdone, EnsCtl *ctl, EnsClock *clk, int *flag, const EnsKeys keys,
                   int nsteps) {
    __shared__ KParams<float> sp;
    __shared__ EnsTile s_tile;
    __shared__ int s_go, s_last, s_cur0, s_ti;
    __shared__ uint32_t s_k[2], s_t0;
    // what lives across the strip sits in shared memory: the strip needs
    // every register the launch bounds leave
    if (threadIdx.x == 0) {
        s_t0 = __ldcg(&clk->t);
        s_cur0 = __ldcg(&clk->cur);
    }
    const uint32_t npairs = (uint32_t)nsteps * (uint32_t)ntiles;
    // Thread 0 claims the next pair while the current one runs, and another
    // thread posts a finished tile while thread 0 sets up the next one, so
    // neither round trip to L2 idles the CTA.  Pairs are still claimed in
    // order and a CTA starts a claimed pair as soon as its current one ends,
    // so the lowest unfinished pair always runs and every wait below ends.
    constexpr int kPoster = 32;
    if (threadIdx.x == 0) s_k[0] = atomicAdd(&ctl->next, 1u);
    __syncthreads();
    for (int it = 0;; it ^= 1) {
        const uint32_t k = s_k[it];
        if (k >= npairs) break;
        uint32_t knext = 0;
        if (threadIdx.x < 32) {   // warp 0 sets the tile up
            const int s = (int)(k / (uint32_t)ntiles), i = (int)(k % (uint32_t)ntiles);
            if (threadIdx.x == 0) knext = atomicAdd(&ctl->next, 1u);
            // the tiles whose cells this one pulls (itself included) must have
            // finished step s - 1: they wrote what it reads, and its stores
            // overwrite what they read in step s - 1
            int w = 1;
            if (s > 0) {
                const int q0 = nbr_off[i];
                w = wait_tiles(tdone, nbr, q0, nbr_off[i + 1] - q0, (uint32_t)s, &ctl->abort,
                               __ldcg(&ctl->wait_ns));
            }
            if (threadIdx.x == 0) {
                const EnsTile tile = tiles[i];
                s_tile = tile;
                s_ti = i;
                if (w < 0) {
                    atomicOr(flag, LB_STEP_TIMEOUT);
                    atomicExch(&ctl->abort, 1);
                }
                if (w > 0)
                    fill_tile_params(sp, reps[tile.r], tile, s_t0 + (uint32_t)s,
                                     s_cur0 ^ (s & 1), false, flag);
                s_go = w > 0;
            }
        }
        __syncthreads();
        if (!s_go) break;
#define ENS_STRIP(FN, U) FN<float, ORDER, false, true, U>(sp, keys.rk, s_tile.x0, s_tile.y0, s_tile.y1)
        if (UM == 2) {
            if (sp.gamma == 0.f) {
                if (OV) ENS_STRIP(step_strip_ov, true); else ENS_STRIP(step_strip, true);
            } else {
                if (OV) ENS_STRIP(step_strip_ov, false); else ENS_STRIP(step_strip, false);
            }
        } else {
            if (OV) ENS_STRIP(step_strip_ov, UM == 1); else ENS_STRIP(step_strip, UM == 1);
        }
#undef ENS_STRIP
        if (threadIdx.x == 0) s_k[it ^ 1] = knext;
        // read before the barrier: thread 0 overwrites s_ti after it
        const int ti = s_ti;
        __syncthreads();   // the tile's stores are done, and sp may be refilled
        if (threadIdx.x == kPoster) {
            __threadfence();
            atomicAdd(&tdone[ti], 1u);   // one step more of tile ti is done
        }
    }
    // the last CTA to finish resets the barriers and advances the clock
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&ctl->finished, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        for (int i = threadIdx.x; i < ntiles; i += blockDim.x) tdone[i] = 0;
        if (threadIdx.x == 0) {
            ctl->finished = 0;
            ctl->abort = 0;
            ctl->next = 0;
            clk->t = s_t0 + (uint32_t)nsteps;
            clk->cur = s_cur0 ^ (nsteps & 1);
            clk->done = 0;
        }
        __threadfence();
    }
}

__device__ __forceinline__ int ilog2_dev(int n) { return __ffs(n) - 1; }

__global__ void ens_rows_kernel(const EnsRep *__restrict__ reps, const int2 *__restrict__ desc) {
    const int2 d = desc[blockIdx.x];
    const EnsRep &R = reps[d.x];
    sk_rows_block<float>(R.drho, R.spec, R.tw_x, R.nx, ilog2_dev(R.nx), R.ldx, d.y);
}

__global__ void ens_cols_kernel(const EnsRep *__restrict__ reps, const int2 *__restrict__ desc,
                                int cpb) {
    const int2 d = desc[blockIdx.x];
    const EnsRep &R = reps[d.x];
    sk_cols_block<float>(R.spec, R.acc, R.tw_y, R.nx, R.ny, ilog2_dev(R.ny), R.ldx, cpb,
                         1.0 / ((double)R.nx * R.ny), d.y);
}

__global__ void clock_set_kernel(EnsClock *clk, uint32_t t, int cur) {
    clk->t = t;
    clk->cur = cur;
    clk->done = 0;
}
// The clock of an ensemble whose replicas are all resident (no tile kernel
// advances it).
__global__ void clock_advance_kernel(EnsClock *clk, int n) {
    clk->t += (uint32_t)n;
    clk->cur ^= n & 1;
}

constexpr double kCs2 = 1.0 / 3.0;
constexpr double kB[6] = {4.0, 4.0 / 9.0, 1.0 / 9.0, 2.0 / 3.0, 2.0 / 3.0, 16.0};
constexpr double kW[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                          1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace lbsc

using namespace lbsc;

// Resident replicas of one shape: C CTAs of hb-row bands per replica.
struct ResClass {
    int nx, ny, C, hb;
    size_t smem;
    std::vector<int> reps;
    int *d_list = nullptr;
};

struct lb_ens {
    int nrep = 0, stencil = 4, psi_kind = 0, dev = 0;
    double p1 = 0, p2 = 0;
    uint64_t seed = 0;
    std::vector<lb_replica> reps;
    std::vector<EnsRep> h_reps;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    unsigned char *pool = nullptr;      // populations of every replica (two buffers)
    unsigned char *sk_pool = nullptr;   // delta rho, spectra, accumulators, twiddles
    EnsRep *d_reps = nullptr;
    EnsTile *d_tiles = nullptr;
    int ntiles = 0;
    int2 *d_rows = nullptr, *d_cols = nullptr;
    int nrows = 0, ncols = 0, cpb = 4, max_nx = 0, max_ny = 0;
    EnsClock *d_clk = nullptr;
    int *d_flag = nullptr;
    double *d_io = nullptr, *d_partials = nullptr, *d_out = nullptr;
    size_t io_elems = 0;
    int nred = 0;
    EnsKeys keys;
    long long t = 0;
    int cur = 0;
    bool inited = false;
    int strip_h = 32;
    int sk_every = 0;
    long long sk_start = 0, sk_count = 0;
    cudaGraphExec_t graph_plain = nullptr;     // kGraphSteps steps, no sampling
    cudaGraphExec_t graph_window = nullptr;    // sk_every steps, sampling at the last
    int launch_mode = LB_ENS_PER_STEP;         // LB_ENS_PER_STEP or LB_ENS_PERSISTENT
    int *d_nbr_off = nullptr, *d_nbr = nullptr;   // tiles each tile pulls from (CSR)
    uint32_t *d_tdone = nullptr;               // steps each tile has finished (persistent)
    EnsCtl *d_ctl = nullptr;
    int persist_grid = 0;                      // co-resident CTAs of the persistent kernel
    int kernel_mode = LB_KERNEL_AUTO;          // LB_KERNEL_PLAIN or _OVERLAP (strip layout)
    bool ov = false;                           // the layout in use
    int umode = 2;                             // unit path: 1 every replica, 0 none, 2 mixed
    int resident_mode = LB_ENS_RESIDENT_AUTO;  // which replicas live in shared memory
    std::vector<ResClass> rclasses;            // resident replicas, one launch per shape
    std::vector<char> is_res;                  // replica r is resident
    int nres = 0;
};

namespace {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return LB_OK;
    if (e == cudaErrorMemoryAllocation) return LB_ERR_NOMEM;
    return LB_ERR_CUDA;
}
#define ENS_CHECK(call)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_status(e_);   \
    } while (0)

double psi_of(int kind, double p1, double p2, double rho) {
    switch (kind) {
    case LB_PSI_EXP: return -expm1(-rho);
    case LB_PSI_CRITICAL: return sqrt(p1 * p2) * exp(1.0 - p2 / rho);
    default: return p1 * exp(-p2 / rho);
    }
}

void fill_rep_params(lb_ens *e, int r) {
    const lb_replica &q = e->reps[r];
    EnsRep &R = e->h_reps[r];
    const double gam = 1.0 - 1.0 / q.tau, hs = 1.0 - 0.5 / q.tau;
    R.psi_kind = e->psi_kind;
    R.noise = q.kT > 0.0 ? 1 : 0;
    R.replica = (uint32_t)r;
    R.rho0 = (float)q.rho0;
    R.force_pref = (float)(-q.G * kCs2);
    R.psi0 = (float)psi_of(e->psi_kind, e->p1, e->p2, q.rho0);
    R.psi_c = e->psi_kind == LB_PSI_EXP ? (float)exp(-q.rho0) : R.psi0;
    R.psi_b = e->psi_kind == LB_PSI_EXP ? 0.0f : (float)e->p2;
    R.gamma = (float)gam;
    R.c3a = (float)(3.0 * (1.0 - gam));
    R.c3b = (float)(6.0 * hs);
    R.c4a = (float)(1.0 - gam);
    R.c4b = (float)(2.0 * hs);
    R.c5a = (float)(1.0 - gam);
    R.c5b = (float)hs;
    const double mu = q.kT / kCs2;
    for (int k = 0; k < 6; ++k) R.amp[k] = (float)sqrt(mu * kB[k] * (1.0 - gam * gam));
}

void drop_graphs(lb_ens *e) {
    if (e->graph_plain) cudaGraphExecDestroy(e->graph_plain);
    if (e->graph_window) cudaGraphExecDestroy(e->graph_window);
    e->graph_plain = e->graph_window = nullptr;
}

// Tiles of 128 columns x strip rows, largest replicas first.
// Launch shape of a resident replica of nx x ny sites: the fewest CTAs per
// replica (C, at most max_c) and then the shortest bands (hb) whose shared
// memory fits one CTA and whose clusters can be resident; false if there is
// none.
bool resident_shape(const lb_ens *e, int nx, int ny, int max_c, ResClass *out) {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, e->dev) !=
        cudaSuccess)
        return false;
    const size_t limit = optin > 1024 ? (size_t)optin - 1024 : 0;   // static shared memory
    for (int c : {1, 2, 4, 8}) {
        if (c > max_c || ny % c) continue;
        const int rows = ny / c;
        for (int hb : {8, 16, 32}) {
            if (rows % hb) continue;
            const size_t sm = resident_smem(nx, rows, hb, e->stencil);
            if (!sm || sm > limit) continue;
            if (resident_prepare(e->stencil, c, limit) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            if (resident_max_clusters(e->stencil, c, nx, rows, hb, sm) < 1) {
                cudaGetLastError();
                continue;
            }
            out->nx = nx;
            out->ny = ny;
            out->C = c;
            out->hb = hb;
            out->smem = sm;
            return true;
        }
    }
    return false;
}

// Which replicas live in shared memory (resident_mode): none; every one
// whose shape allows it; or, AUTO, all of them when each fits one CTA.
// AUTO leaves out the clusters (128^2 over four CTAs measured 42 against 63
// GLUPS tiled: a tile already fills its 128 columns, clusters of four
// 200 KB CTAs leave SMs of each GPC idle and each step waits at two cluster
// barriers) and mixed ensembles (the resident launch runs before the tiles,
// so its few CTAs would hold up the rest of the GPU).
int setup_resident(lb_ens *e) {
    for (auto &c : e->rclasses) cudaFree(c.d_list);
    e->rclasses.clear();
    e->is_res.assign(e->nrep, 0);
    e->nres = 0;
    if (e->resident_mode == LB_ENS_RESIDENT_OFF) return LB_OK;
    std::vector<ResClass> cls;
    std::vector<std::pair<long, int>> tried;   // shape -> class index or -1
    int n = 0;
    for (int r = 0; r < e->nrep; ++r) {
        const int nx = e->reps[r].nx, ny = e->reps[r].ny;
        const long key = (long)nx * 1000003L + ny;
        int k = -2;
        for (const auto &t : tried)
            if (t.first == key) k = t.second;
        if (k == -2) {
            ResClass c;
            const int max_c = e->resident_mode == LB_ENS_RESIDENT_AUTO ? 1 : 8;
            if (resident_shape(e, nx, ny, max_c, &c)) {
                cls.push_back(c);
                k = (int)cls.size() - 1;
            } else {
                k = -1;
            }
            tried.push_back({key, k});
        }
        if (k < 0) {
            if (e->resident_mode == LB_ENS_RESIDENT_AUTO) return LB_OK;
            continue;
        }
        cls[k].reps.push_back(r);
        ++n;
    }
    for (auto &c : cls) {
        ENS_CHECK(cudaMalloc(&c.d_list, c.reps.size() * sizeof(int)));
        ENS_CHECK(cudaMemcpy(c.d_list, c.reps.data(), c.reps.size() * sizeof(int),
                             cudaMemcpyHostToDevice));
        for (int r : c.reps) e->is_res[r] = 1;
    }
    e->rclasses = std::move(cls);
    e->nres = n;
    return LB_OK;
}

int build_tiles(lb_ens *e) {
    std::vector<EnsTile> tiles;
    std::vector<int> order(e->nrep);
    for (int r = 0; r < e->nrep; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long)e->reps[a].nx * e->reps[a].ny > (long)e->reps[b].nx * e->reps[b].ny;
    });
    // Tiles of a replica form a grid of row strips x column strips.  A tile
    // pulls rows y0 - H - 1 .. y1 + H and columns x0 - H - 1 .. x1 + H
    // (periodic); the tiles holding those cells are its dependencies in the
    // persistent launch (CSR: nbr_off, nbr).
    const int H = e->stencil == 4 ? 1 : 2;
    std::vector<int> nbr_off(1, 0), nbr;
    for (int r : order) {
        if (e->is_res[r]) continue;   // advanced by the resident kernel
        const int nx = e->reps[r].nx, ny = e->reps[r].ny;
        const int h = std::min(e->strip_h, ny);
        const int cols = e->ov ? kStepTX - 2 * H : kStepTX;
        const int nry = (ny + h - 1) / h, ncx = (nx + cols - 1) / cols;
        const int base = (int)tiles.size();
        // strips whose cells the tiles of one row (column) strip read
        auto strips = [](int a0, int a1, int n, int w, int halo) {
            std::vector<int> out;
            for (int a = a0 - halo - 1; a <= a1 - 1 + halo + 1; ++a) {
                const int idx = (((a % n) + n) % n) / w;
                if (std::find(out.begin(), out.end(), idx) == out.end()) out.push_back(idx);
            }
            return out;
        };
        std::vector<std::vector<int>> rset(nry), cset(ncx);
        for (int ry = 0; ry < nry; ++ry) rset[ry] = strips(ry * h, std::min(ry * h + h, ny), ny, h, H);
        for (int cx = 0; cx < ncx; ++cx)
            cset[cx] = strips(cx * cols, std::min(cx * cols + cols, nx), nx, cols, H);
        for (int ry = 0; ry < nry; ++ry)
            for (int cx = 0; cx < ncx; ++cx) {
                const int y0 = ry * h, x0 = cx * cols;
                tiles.push_back({r, x0, y0, std::min(y0 + h, ny)});
                for (int a : rset[ry])
                    for (int b : cset[cx]) nbr.push_back(base + a * ncx + b);
                nbr_off.push_back((int)nbr.size());
            }
    }
    cudaFree(e->d_tiles);
    cudaFree(e->d_nbr_off);
    cudaFree(e->d_nbr);
    cudaFree(e->d_tdone);
    e->d_tiles = nullptr;
    e->d_nbr_off = e->d_nbr = nullptr;
    e->d_tdone = nullptr;
    e->ntiles = 0;
    if (!tiles.empty()) {
        ENS_CHECK(cudaMalloc(&e->d_tiles, tiles.size() * sizeof(EnsTile)));
        ENS_CHECK(cudaMemcpy(e->d_tiles, tiles.data(), tiles.size() * sizeof(EnsTile),
                             cudaMemcpyHostToDevice));
        ENS_CHECK(cudaMalloc(&e->d_nbr_off, nbr_off.size() * sizeof(int)));
        ENS_CHECK(cudaMemcpy(e->d_nbr_off, nbr_off.data(), nbr_off.size() * sizeof(int),
                             cudaMemcpyHostToDevice));
        ENS_CHECK(cudaMalloc(&e->d_nbr, nbr.size() * sizeof(int)));
        ENS_CHECK(cudaMemcpy(e->d_nbr, nbr.data(), nbr.size() * sizeof(int),
                             cudaMemcpyHostToDevice));
        ENS_CHECK(cudaMalloc(&e->d_tdone, tiles.size() * sizeof(uint32_t)));
        ENS_CHECK(cudaMemset(e->d_tdone, 0, tiles.size() * sizeof(uint32_t)));
    }
    e->ntiles = (int)tiles.size();
    drop_graphs(e);
    return LB_OK;
}

template <int ORDER, bool OV, int UM>
cudaError_t launch_persist_t(lb_ens *e, int nsteps) {
    void *args[] = {&e->d_reps,  &e->d_tiles, &e->ntiles, &e->d_nbr_off, &e->d_nbr,
                    &e->d_tdone, &e->d_ctl,   &e->d_clk,  &e->d_flag,    &e->keys,
                    &nsteps};
    const int grid = std::min(e->persist_grid, e->ntiles);
    return cudaLaunchCooperativeKernel((const void *)ens_persist_kernel<ORDER, OV, UM>,
                                       dim3(grid), dim3(OV ? kStepTX : kStepTX + 32), args, 0,
                                       e->stream);
}

// The persistent kernel of the ensemble's stencil, layout and unit mode.
template <int ORDER, bool OV>
const void *persist_fn_ov(int um) {
    return um == 1   ? (const void *)ens_persist_kernel<ORDER, OV, 1>
           : um == 0 ? (const void *)ens_persist_kernel<ORDER, OV, 0>
                     : (const void *)ens_persist_kernel<ORDER, OV, 2>;
}
template <int ORDER>
const void *persist_fn_o(const lb_ens *e) {
    return e->ov ? persist_fn_ov<ORDER, true>(e->umode) : persist_fn_ov<ORDER, false>(e->umode);
}
const void *persist_fn(const lb_ens *e) {
    return e->stencil == 4   ? persist_fn_o<4>(e)
           : e->stencil == 6 ? persist_fn_o<6>(e)
                             : persist_fn_o<8>(e);
}

template <int ORDER, bool OV>
cudaError_t launch_persist_ov(lb_ens *e, int nsteps) {
    return e->umode == 1   ? launch_persist_t<ORDER, OV, 1>(e, nsteps)
           : e->umode == 0 ? launch_persist_t<ORDER, OV, 0>(e, nsteps)
                           : launch_persist_t<ORDER, OV, 2>(e, nsteps);
}
template <int ORDER>
cudaError_t launch_persist_o(lb_ens *e, int nsteps) {
    return e->ov ? launch_persist_ov<ORDER, true>(e, nsteps)
                 : launch_persist_ov<ORDER, false>(e, nsteps);
}

// Co-resident CTAs of the persistent kernel in use.
cudaError_t persist_occupancy(lb_ens *e) {
    int per_sm = 0, nsm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, persist_fn(e), e->ov ? kStepTX : kStepTX + 32, 0);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, e->dev);
    e->persist_grid = per_sm * nsm;
    return err;
}

cudaError_t launch_ens_step(lb_ens *e, bool sample);

// `nsteps` steps of every replica: one persistent launch, except that a
// sampling last step runs through the per-step kernel, which also takes the
// S(k) sample.
cudaError_t launch_ens_persistent(lb_ens *e, int nsteps, bool sample_last) {
    const int n = sample_last ? nsteps - 1 : nsteps;
    cudaError_t err = cudaSuccess;
    if (n > 0 && e->ntiles == 0) {
        clock_advance_kernel<<<1, 1, 0, e->stream>>>(e->d_clk, n);
        err = cudaGetLastError();
    } else if (n > 0)
        err = e->stencil == 4   ? launch_persist_o<4>(e, n)
              : e->stencil == 6 ? launch_persist_o<6>(e, n)
                                : launch_persist_o<8>(e, n);
    if (err != cudaSuccess || !sample_last) return err;
    return launch_ens_step(e, true);
}

// One step of every replica; `sample` also runs the S(k) sample of all
// replicas (the step kernel then writes delta rho: the device decides from
// its own step counter, which agrees with the host's).
cudaError_t launch_ens_step(lb_ens *e, bool sample) {
    const int sk_every = sample ? e->sk_every : 0;
#define ENS_STEP(O, V, B)                                                                     \
    ens_step_kernel<O, V><<<e->ntiles, B, 0, e->stream>>>(e->d_reps, e->d_tiles, e->ntiles,   \
                                                          e->d_clk, e->d_flag, e->keys,       \
                                                          sk_every, e->sk_start)
    if (e->ntiles == 0) {
        clock_advance_kernel<<<1, 1, 0, e->stream>>>(e->d_clk, 1);
    } else if (e->ov) {
        if (e->stencil == 4) ENS_STEP(4, true, kStepTX);
        else if (e->stencil == 6) ENS_STEP(6, true, kStepTX);
        else ENS_STEP(8, true, kStepTX);
    } else {
        if (e->stencil == 4) ENS_STEP(4, false, kStepTX + 32);
        else if (e->stencil == 6) ENS_STEP(6, false, kStepTX + 32);
        else ENS_STEP(8, false, kStepTX + 32);
    }
#undef ENS_STEP
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || !sample) return err;
    ens_rows_kernel<<<e->nrows, 512, (size_t)e->max_nx * sizeof(float2), e->stream>>>(e->d_reps,
                                                                                       e->d_rows);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    ens_cols_kernel<<<e->ncols, 512, (size_t)e->cpb * e->max_ny * sizeof(float2), e->stream>>>(
        e->d_reps, e->d_cols, e->cpb);
    return cudaGetLastError();
}

bool is_sample_step(const lb_ens *e, long long tn) {
    return e->sk_every > 0 && e->sk_pool && tn >= e->sk_start &&
           (tn - e->sk_start) % e->sk_every == 0;
}

// `steps` consecutive steps of every replica, the last one sampling if
// sample_last: the resident replicas in one launch per shape, then the
// tiles (which advance the device clock and take the S(k) sample).
cudaError_t launch_window(lb_ens *e, int steps, bool sample_last) {
    cudaError_t err = cudaSuccess;
    for (const auto &c : e->rclasses) {
        ResLaunch a;
        a.reps = e->d_reps;
        a.list = c.d_list;
        a.nres = (int)c.reps.size();
        a.nx = c.nx;
        a.ny = c.ny;
        a.C = c.C;
        a.hb = c.hb;
        a.stencil = e->stencil;
        a.clk = e->d_clk;
        a.flag = e->d_flag;
        a.keys = e->keys;
        a.nsteps = steps;
        a.sample = sample_last ? 1 : 0;
        if ((err = launch_ens_resident(a, e->stream)) != cudaSuccess) return err;
    }
    if (e->launch_mode == LB_ENS_PERSISTENT) return launch_ens_persistent(e, steps, sample_last);
    for (int s = 0; s < steps && err == cudaSuccess; ++s)
        err = launch_ens_step(e, sample_last && s == steps - 1);
    return err;
}

// Capture `steps` consecutive steps, the last one sampling if sample_last.
int capture(lb_ens *e, int steps, bool sample_last, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    ENS_CHECK(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = launch_window(e, steps, sample_last);
    cudaError_t err2 = cudaStreamEndCapture(e->stream, &g);
    if (err != cudaSuccess || err2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_status(err != cudaSuccess ? err : err2);
    }
    err = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    ENS_CHECK(err);
    return LB_OK;
}

void free_ens(lb_ens *e) {
    drop_graphs(e);
    for (auto &c : e->rclasses) cudaFree(c.d_list);
    e->rclasses.clear();
    cudaFree(e->pool);
    cudaFree(e->sk_pool);
    cudaFree(e->d_reps);
    cudaFree(e->d_tiles);
    cudaFree(e->d_rows);
    cudaFree(e->d_cols);
    cudaFree(e->d_clk);
    cudaFree(e->d_flag);
    cudaFree(e->d_io);
    cudaFree(e->d_partials);
    cudaFree(e->d_out);
    cudaFree(e->d_nbr_off);
    cudaFree(e->d_nbr);
    cudaFree(e->d_tdone);
    cudaFree(e->d_ctl);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
}

int rep_arg(const lb_ens *e, int r) {
    if (!e || r < 0 || r >= e->nrep) return LB_ERR_ARG;
    if (!e->inited) return LB_ERR_STATE;
    return LB_OK;
}

int ens_sync(lb_ens *e) {
    ENS_CHECK(cudaStreamSynchronize(e->stream));
    int flag = 0;
    ENS_CHECK(cudaMemcpy(&flag, e->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        ENS_CHECK(cudaMemset(e->d_flag, 0, sizeof(int)));
        return (flag & LB_STEP_TIMEOUT) ? LB_ERR_TIMEOUT : LB_ERR_NONFINITE;
    }
    return LB_OK;
}

}  // namespace

extern "C" {

int lb_ens_create(lb_ens **out, const lb_replica *reps, int nrep, int psi_kind, double psi_p1,
                  double psi_p2, int stencil, uint64_t seed, void *stream) {
    if (!out || !reps || nrep < 1 || nrep > 65536) return LB_ERR_ARG;
    *out = nullptr;
    if (stencil != 4 && stencil != 6 && stencil != 8) return LB_ERR_ARG;
    if (psi_kind != LB_PSI_EXP && !(psi_p1 > 0.0 && psi_p2 > 0.0)) return LB_ERR_ARG;
    if (psi_kind < 0 || psi_kind > 2) return LB_ERR_ARG;
    for (int r = 0; r < nrep; ++r) {
        const lb_replica &q = reps[r];
        if (q.nx < 4 || q.ny < 4 || q.nx % 4 || q.ny % 4) return LB_ERR_ARG;
        if (9.0 * (double)q.nx * q.ny >= 4294967296.0) return LB_ERR_ARG;
        if (!(q.tau > 0.5) || !(q.kT >= 0.0) || !isfinite(q.G) || !(q.rho0 > 0.0)) return LB_ERR_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return LB_ERR_CUDA;
    lb_ens *e = new (std::nothrow) lb_ens();
    if (!e) return LB_ERR_NOMEM;
    cudaGetDevice(&e->dev);
    e->nrep = nrep;
    e->stencil = stencil;
    e->psi_kind = psi_kind;
    e->p1 = psi_p1;
    e->p2 = psi_p2;
    e->seed = seed;
    e->reps.assign(reps, reps + nrep);
    e->h_reps.resize(nrep);
    philox_round_keys(seed, e->keys.rk);
    if (stream) {
        e->stream = (cudaStream_t)stream;
    } else if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) == cudaSuccess) {
        e->own_stream = true;
    } else {
        delete e;
        return LB_ERR_CUDA;
    }
    size_t bytes = 0, max_sites = 0;
    std::vector<size_t> off(nrep);
    for (int r = 0; r < nrep; ++r) {
        const size_t n = (size_t)reps[r].nx * reps[r].ny;
        off[r] = bytes;
        bytes += align256(2 * 9 * n * sizeof(float));
        max_sites = std::max(max_sites, n);
    }
    cudaError_t err = cudaMalloc(&e->pool, bytes);
    if (err == cudaSuccess) err = cudaMalloc(&e->d_reps, nrep * sizeof(EnsRep));
    if (err == cudaSuccess) err = cudaMalloc(&e->d_clk, sizeof(EnsClock));
    if (err == cudaSuccess) err = cudaMalloc(&e->d_flag, sizeof(int));
    e->io_elems = std::max(max_sites, (size_t)8192);
    if (err == cudaSuccess) err = cudaMalloc(&e->d_io, e->io_elems * sizeof(double));
    e->nred = conserved_blocks(4096, 4096);
    if (err == cudaSuccess) err = cudaMalloc(&e->d_partials, 3 * (size_t)e->nred * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&e->d_out, 4 * sizeof(double));
    if (err == cudaSuccess) err = cudaMemset(e->d_flag, 0, sizeof(int));
    if (err == cudaSuccess) err = cudaMalloc(&e->d_ctl, sizeof(EnsCtl));
    if (err == cudaSuccess) {
        const EnsCtl c0 = {0u, 0, (unsigned long long)kEnsWaitNs, 0u};
        err = cudaMemcpy(e->d_ctl, &c0, sizeof(EnsCtl), cudaMemcpyHostToDevice);
    }
    {
        // a replica takes the unit path when its rate gamma rounds to 0 in
        // FP32, the test the kernels make
        int nunit = 0;
        for (int r = 0; r < nrep; ++r) nunit += (float)(1.0 - 1.0 / reps[r].tau) == 0.0f;
        e->umode = nunit == nrep ? 1 : nunit == 0 ? 0 : 2;
    }
    if (err == cudaSuccess) err = persist_occupancy(e);
    if (err != cudaSuccess) {
        free_ens(e);
        delete e;
        return cuda_status(err);
    }
    for (int r = 0; r < nrep; ++r) {
        EnsRep &R = e->h_reps[r];
        memset(&R, 0, sizeof(R));
        const size_t n = (size_t)reps[r].nx * reps[r].ny;
        R.buf[0] = (float *)(e->pool + off[r]);
        R.buf[1] = R.buf[0] + 9 * n;
        R.nx = reps[r].nx;
        R.ny = reps[r].ny;
        fill_rep_params(e, r);
        e->max_nx = std::max(e->max_nx, R.nx);
        e->max_ny = std::max(e->max_ny, R.ny);
    }
    int rc = setup_resident(e);
    if (rc == LB_OK) rc = build_tiles(e);
    if (rc == LB_OK && cudaMemcpy(e->d_reps, e->h_reps.data(), nrep * sizeof(EnsRep),
                                  cudaMemcpyHostToDevice) != cudaSuccess)
        rc = LB_ERR_CUDA;
    if (rc != LB_OK) {
        free_ens(e);
        delete e;
        return rc;
    }
    *out = e;
    return LB_OK;
}

void lb_ens_destroy(lb_ens *e) {
    if (!e) return;
    cudaSetDevice(e->dev);
    if (e->stream) cudaStreamSynchronize(e->stream);
    free_ens(e);
    delete e;
}

int lb_ens_init(lb_ens *e, double init_amp) {
    if (!e || !isfinite(init_amp)) return LB_ERR_ARG;
    ENS_CHECK(cudaSetDevice(e->dev));
    for (int r = 0; r < e->nrep; ++r)
        ENS_CHECK(launch_init(0, e->h_reps[r].buf[0], e->h_reps[r].nx, e->h_reps[r].ny, init_amp,
                              e->keys.rk, (uint32_t)r, e->stream));
    e->t = 0;
    e->cur = 0;
    clock_set_kernel<<<1, 1, 0, e->stream>>>(e->d_clk, 0, 0);
    ENS_CHECK(cudaGetLastError());
    if (e->sk_pool) {
        for (int r = 0; r < e->nrep; ++r) {
            const EnsRep &R = e->h_reps[r];
            ENS_CHECK(cudaMemsetAsync(R.acc, 0, (size_t)R.ny * R.ldx * sizeof(double), e->stream));
        }
    }
    e->sk_count = 0;
    e->inited = true;
    return LB_OK;
}

int lb_ens_sk_config(lb_ens *e, int sample_every, long long start_step) {
    if (!e || sample_every < 0 || start_step < 0) return LB_ERR_ARG;
    ENS_CHECK(cudaSetDevice(e->dev));
    if (sample_every > 0 && !e->sk_pool) {
        for (int r = 0; r < e->nrep; ++r) {
            const lb_replica &q = e->reps[r];
            if (!is_pow2(q.nx) || !is_pow2(q.ny) || q.nx > 8192 || q.ny > 8192)
                return LB_ERR_UNSUPPORTED;
        }
        size_t bytes = 0;
        std::vector<size_t> o_drho(e->nrep), o_spec(e->nrep), o_acc(e->nrep), o_tx(e->nrep),
            o_ty(e->nrep);
        for (int r = 0; r < e->nrep; ++r) {
            const int nx = e->reps[r].nx, ny = e->reps[r].ny, ldx = ((nx / 2 + 1) + 3) / 4 * 4;
            e->h_reps[r].ldx = ldx;
            o_drho[r] = bytes;
            bytes += align256((size_t)nx * ny * sizeof(float));
            o_spec[r] = bytes;
            bytes += align256((size_t)ny * ldx * sizeof(float2));
            o_acc[r] = bytes;
            bytes += align256((size_t)ny * ldx * sizeof(double));
            o_tx[r] = bytes;
            bytes += align256((size_t)(nx / 2) * sizeof(float2));
            o_ty[r] = bytes;
            bytes += align256((size_t)(ny / 2) * sizeof(float2));
        }
        ENS_CHECK(cudaMalloc(&e->sk_pool, bytes));
        ENS_CHECK(cudaMemsetAsync(e->sk_pool, 0, bytes, e->stream));
        std::vector<int2> rows, cols;
        const int cpb = cols_per_block(e->max_ny, sizeof(float2));
        e->cpb = cpb;
        for (int r = 0; r < e->nrep; ++r) {
            EnsRep &R = e->h_reps[r];
            R.drho = (float *)(e->sk_pool + o_drho[r]);
            R.spec = (float2 *)(e->sk_pool + o_spec[r]);
            R.acc = (double *)(e->sk_pool + o_acc[r]);
            R.tw_x = (const float2 *)(e->sk_pool + o_tx[r]);
            R.tw_y = (const float2 *)(e->sk_pool + o_ty[r]);
            ENS_CHECK(launch_twiddles(0, (void *)R.tw_x, R.nx, e->stream));
            ENS_CHECK(launch_twiddles(0, (void *)R.tw_y, R.ny, e->stream));
            for (int pr = 0; pr < R.ny / 2; ++pr) rows.push_back(make_int2(r, pr));
            for (int kx = 0; kx < R.nx / 2 + 1; kx += cpb) cols.push_back(make_int2(r, kx));
        }
        e->nrows = (int)rows.size();
        e->ncols = (int)cols.size();
        ENS_CHECK(cudaMalloc(&e->d_rows, rows.size() * sizeof(int2)));
        ENS_CHECK(cudaMalloc(&e->d_cols, cols.size() * sizeof(int2)));
        ENS_CHECK(cudaMemcpy(e->d_rows, rows.data(), rows.size() * sizeof(int2),
                             cudaMemcpyHostToDevice));
        ENS_CHECK(cudaMemcpy(e->d_cols, cols.data(), cols.size() * sizeof(int2),
                             cudaMemcpyHostToDevice));
        ENS_CHECK(cudaMemcpy(e->d_reps, e->h_reps.data(), e->nrep * sizeof(EnsRep),
                             cudaMemcpyHostToDevice));
        ENS_CHECK(cudaFuncSetAttribute(ens_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((size_t)e->max_nx * sizeof(float2))));
        ENS_CHECK(cudaFuncSetAttribute(ens_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((size_t)cpb * e->max_ny * sizeof(float2))));
        e->sk_count = 0;
    }
    e->sk_every = sample_every;
    e->sk_start = start_step;
    drop_graphs(e);
    return LB_OK;
}

int lb_ens_set_strip_height(lb_ens *e, int rows) {
    if (!e || rows < 1) return LB_ERR_ARG;
    ENS_CHECK(cudaSetDevice(e->dev));
    e->strip_h = rows;
    return build_tiles(e);
}

int lb_ens_set_launch(lb_ens *e, int mode) {
    if (!e || (mode != LB_ENS_PER_STEP && mode != LB_ENS_PERSISTENT)) return LB_ERR_ARG;
    ENS_CHECK(cudaSetDevice(e->dev));
    if (mode == LB_ENS_PERSISTENT) {
        int coop = 0;
        ENS_CHECK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, e->dev));
        if (!coop || e->persist_grid < 1) return LB_ERR_UNSUPPORTED;
    }
    e->launch_mode = mode;
    drop_graphs(e);
    return LB_OK;
}

int lb_ens_get_launch(const lb_ens *e) { return e ? e->launch_mode : LB_ERR_ARG; }

int lb_ens_set_kernel(lb_ens *e, int mode) {
    if (!e || (mode != LB_KERNEL_AUTO && mode != LB_KERNEL_PLAIN && mode != LB_KERNEL_OVERLAP))
        return LB_ERR_ARG;
    ENS_CHECK(cudaSetDevice(e->dev));
    ENS_CHECK(cudaStreamSynchronize(e->stream));
    e->kernel_mode = mode;
    // AUTO: the halo-warp layout.  Replica widths are powers of two up to a
    // few hundred columns, where the overlapped layout's last strip holds
    // only a few columns (256 replicas of {64..512}^2: 61 against 56 GLUPS).
    e->ov = mode == LB_KERNEL_OVERLAP;
    ENS_CHECK(persist_occupancy(e));
    return build_tiles(e);
}

int lb_ens_set_resident(lb_ens *e, int mode) {
    if (!e || (mode != LB_ENS_RESIDENT_OFF && mode != LB_ENS_RESIDENT_ON &&
               mode != LB_ENS_RESIDENT_AUTO))
        return LB_ERR_ARG;
    ENS_CHECK(cudaSetDevice(e->dev));
    ENS_CHECK(cudaStreamSynchronize(e->stream));
    e->resident_mode = mode;
    const int rc = setup_resident(e);
    return rc != LB_OK ? rc : build_tiles(e);
}

int lb_ens_num_resident(const lb_ens *e) { return e ? e->nres : LB_ERR_ARG; }

int lb_ens_get_kernel(const lb_ens *e) {
    if (!e) return LB_ERR_ARG;
    return e->ov ? LB_KERNEL_OVERLAP : LB_KERNEL_PLAIN;
}

int lb_ens_set_wait_ns(lb_ens *e, long long ns) {
    if (!e) return LB_ERR_ARG;
    ENS_CHECK(cudaSetDevice(e->dev));
    const unsigned long long v = ns < 0 ? (unsigned long long)kEnsWaitNs : (unsigned long long)ns;
    ENS_CHECK(cudaStreamSynchronize(e->stream));
    ENS_CHECK(cudaMemcpy(&e->d_ctl->wait_ns, &v, sizeof(v), cudaMemcpyHostToDevice));
    return LB_OK;
}

int lb_ens_step(lb_ens *e, int n) {
    if (!e || n < 0) return LB_ERR_ARG;
    if (!e->inited) return LB_ERR_STATE;
    ENS_CHECK(cudaSetDevice(e->dev));
    constexpr int kGraphSteps = 32;
    const bool sk = e->sk_every > 0 && e->sk_pool;
    while (n > 0) {
        const long long t = e->t;
        // a window of kGraphSteps steps with no sampling step inside
        const bool plain_ok = n >= kGraphSteps &&
                              (!sk || t + kGraphSteps < e->sk_start);
        // a window t+1 .. t+every whose only sampling step is its last
        // (one launch per step: intervals of at most 1024 steps are captured whole)
        const bool window_ok = sk && e->sk_every >= 2 && n >= e->sk_every && t >= e->sk_start &&
                               (t - e->sk_start) % e->sk_every == 0 &&
                               (e->launch_mode == LB_ENS_PERSISTENT || e->sk_every <= 1024);
        if (plain_ok || window_ok) {
            cudaGraphExec_t *g = plain_ok ? &e->graph_plain : &e->graph_window;
            const int len = plain_ok ? kGraphSteps : e->sk_every;
            if (!*g) {
                int rc = capture(e, len, !plain_ok, g);
                if (rc != LB_OK) return rc;
            }
            ENS_CHECK(cudaGraphLaunch(*g, e->stream));
            e->t += len;
            e->cur = (int)((e->cur + len) & 1);
            if (!plain_ok) e->sk_count += 1;
            n -= len;
            continue;
        }
        const bool sample = is_sample_step(e, t + 1);
        ENS_CHECK(launch_window(e, 1, sample));
        e->t += 1;
        e->cur ^= 1;
        if (sample) e->sk_count += 1;
        n -= 1;
    }
    return LB_OK;
}

int lb_ens_sync(lb_ens *e) {
    if (!e) return LB_ERR_ARG;
    ENS_CHECK(cudaSetDevice(e->dev));
    return ens_sync(e);
}

long long lb_ens_get_step(const lb_ens *e) { return e ? e->t : -1; }

int lb_ens_num_tiles(const lb_ens *e) { return e ? e->ntiles : LB_ERR_ARG; }

int lb_ens_populations(lb_ens *e, int r, double *host_out) {
    int rc = rep_arg(e, r);
    if (rc || !host_out) return rc ? rc : LB_ERR_ARG;
    ENS_CHECK(cudaSetDevice(e->dev));
    const EnsRep &R = e->h_reps[r];
    const size_t n = (size_t)R.nx * R.ny;
    std::vector<float> tmp;
    try {
        tmp.resize(9 * n);
    } catch (...) {
        return LB_ERR_NOMEM;
    }
    ENS_CHECK(cudaMemcpyAsync(tmp.data(), R.buf[e->cur], 9 * n * sizeof(float),
                              cudaMemcpyDeviceToHost, e->stream));
    rc = ens_sync(e);
    if (rc) return rc;
    for (int i = 0; i < 9; ++i)
        for (size_t s = 0; s < n; ++s) host_out[i * n + s] = kW[i] * e->reps[r].rho0 + tmp[i * n + s];
    return LB_OK;
}

int lb_ens_density(lb_ens *e, int r, double *host_out) {
    int rc = rep_arg(e, r);
    if (rc || !host_out) return rc ? rc : LB_ERR_ARG;
    ENS_CHECK(cudaSetDevice(e->dev));
    const EnsRep &R = e->h_reps[r];
    ENS_CHECK(launch_density(0, R.buf[e->cur], e->reps[r].rho0, e->d_io, R.nx, R.ny, e->stream));
    ENS_CHECK(cudaMemcpyAsync(host_out, e->d_io, (size_t)R.nx * R.ny * sizeof(double),
                              cudaMemcpyDeviceToHost, e->stream));
    return ens_sync(e);
}

int lb_ens_conserved(lb_ens *e, int r, double out[3]) {
    int rc = rep_arg(e, r);
    if (rc || !out) return rc ? rc : LB_ERR_ARG;
    ENS_CHECK(cudaSetDevice(e->dev));
    const EnsRep &R = e->h_reps[r];
    const int nb = std::min(e->nred, conserved_blocks(R.nx, R.ny));
    ENS_CHECK(launch_conserved(0, R.buf[e->cur], e->d_partials, nb, e->d_out, R.nx, R.ny,
                               e->stream));
    double tmp[3];
    ENS_CHECK(cudaMemcpyAsync(tmp, e->d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, e->stream));
    rc = ens_sync(e);
    if (rc) return rc;
    out[0] = (double)R.nx * R.ny * e->reps[r].rho0 + tmp[0];
    out[1] = tmp[1];
    out[2] = tmp[2];
    return LB_OK;
}

int lb_ens_structure_factor(lb_ens *e, int r, double *host_out, int nbins,
                            long long *nsamples_out) {
    int rc = rep_arg(e, r);
    if (rc || !host_out || nbins < 0 || nbins > 4096) return rc ? rc : LB_ERR_ARG;
    if (!e->sk_pool) return LB_ERR_STATE;
    ENS_CHECK(cudaSetDevice(e->dev));
    const EnsRep &R = e->h_reps[r];
    const double inv = e->sk_count > 0 ? 1.0 / (double)e->sk_count : 0.0;
    if (nbins == 0) {
        ENS_CHECK(launch_sk_readout(R.acc, inv, e->d_io, R.nx, R.ny, R.ldx, e->stream));
        ENS_CHECK(cudaMemcpyAsync(host_out, e->d_io, (size_t)(R.nx / 2 + 1) * R.ny * sizeof(double),
                                  cudaMemcpyDeviceToHost, e->stream));
        rc = ens_sync(e);
        if (rc) return rc;
    } else {
        ENS_CHECK(cudaMemsetAsync(e->d_io, 0, 2 * (size_t)nbins * sizeof(double), e->stream));
        ENS_CHECK(launch_sk_bins(R.acc, inv, e->d_io, e->d_io + nbins, nbins, R.nx, R.ny, R.ldx,
                                 e->stream));
        std::vector<double> tmp(2 * (size_t)nbins);
        ENS_CHECK(cudaMemcpyAsync(tmp.data(), e->d_io, tmp.size() * sizeof(double),
                                  cudaMemcpyDeviceToHost, e->stream));
        rc = ens_sync(e);
        if (rc) return rc;
        for (int b = 0; b < nbins; ++b)
            host_out[b] = tmp[nbins + b] > 0 ? tmp[b] / tmp[nbins + b] : NAN;
    }
    if (nsamples_out) *nsamples_out = e->sk_count;
    return LB_OK;
}

// Autotuner: time each candidate strip height on a snapshot of the state and
// keep the fastest; the state, clock and S(k) sums are restored afterwards.
// The candidates run in the launch mode and strip layout in use.  The choice
// is cached in `cache_path` (one "key strip" line per ensemble shape, launch
// mode, layout and device) when the path is not NULL.
int lb_ens_autotune(lb_ens *e, int trial_steps, const char *cache_path, int *chosen) {
    if (!e || trial_steps < 1) return LB_ERR_ARG;
    if (!e->inited) return LB_ERR_STATE;
    ENS_CHECK(cudaSetDevice(e->dev));
    if (e->ntiles == 0) {   // every replica resident: there is no tile shape to tune
        if (chosen) *chosen = e->strip_h;
        return LB_OK;
    }
    cudaDeviceProp prop;
    ENS_CHECK(cudaGetDeviceProperties(&prop, e->dev));
    std::string key = std::string(prop.name) + "|E" + std::to_string(e->stencil) +
                      (e->launch_mode == LB_ENS_PERSISTENT ? "|P" : "|S") +
                      (e->ov ? "|ov" : "|hw") + "|R" + std::to_string(e->nres);
    {
        std::vector<long> sizes;
        for (const auto &q : e->reps) sizes.push_back((long)q.nx * 100000 + q.ny);
        std::sort(sizes.begin(), sizes.end());
        unsigned long long h = 1469598103934665603ull;
        for (long v : sizes) h = (h ^ (unsigned long long)v) * 1099511628211ull;
        char buf[64];
        snprintf(buf, sizeof(buf), "|n%d|%016llx", e->nrep, h);
        key += buf;
        for (auto &c : key)
            if (c == ' ') c = '_';
    }
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char k[512];
            int v = 0;
            while (fscanf(f, "%511s %d", k, &v) == 2) {
                if (key == k && v > 0) {
                    fclose(f);
                    if (chosen) *chosen = v;
                    return lb_ens_set_strip_height(e, v);
                }
            }
            fclose(f);
        }
    }
    // snapshot
    size_t pool_bytes = 0;
    for (int r = 0; r < e->nrep; ++r)
        pool_bytes += align256(2 * 9 * (size_t)e->reps[r].nx * e->reps[r].ny * sizeof(float));
    unsigned char *snap = nullptr;
    ENS_CHECK(cudaMalloc(&snap, pool_bytes));
    ENS_CHECK(cudaMemcpyAsync(snap, e->pool, pool_bytes, cudaMemcpyDeviceToDevice, e->stream));
    const long long t0 = e->t, count0 = e->sk_count;
    const int cur0 = e->cur, every0 = e->sk_every;
    const int cand[] = {8, 12, 16, 24, 32, 48};
    float best_ms = 1e30f;
    int best = e->strip_h;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    e->sk_every = 0;
    int rc = LB_OK;
    // each candidate runs the way steps will run: one launch per step, or
    // one persistent launch for the whole trial
    const bool persist = e->launch_mode == LB_ENS_PERSISTENT;
    for (int c : cand) {
        if ((rc = lb_ens_set_strip_height(e, c)) != LB_OK) break;
        if (persist) rc = cuda_status(launch_ens_persistent(e, 2, false));
        else
            for (int w = 0; w < 2 && rc == LB_OK; ++w) rc = cuda_status(launch_ens_step(e, false));
        cudaEventRecord(a, e->stream);
        if (persist && rc == LB_OK) rc = cuda_status(launch_ens_persistent(e, trial_steps, false));
        for (int s = 0; s < trial_steps && rc == LB_OK && !persist; ++s)
            rc = cuda_status(launch_ens_step(e, false));
        cudaEventRecord(b, e->stream);
        if (rc != LB_OK) break;
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    // restore
    e->sk_every = every0;
    ENS_CHECK(cudaMemcpyAsync(e->pool, snap, pool_bytes, cudaMemcpyDeviceToDevice, e->stream));
    e->t = t0;
    e->cur = cur0;
    e->sk_count = count0;
    clock_set_kernel<<<1, 1, 0, e->stream>>>(e->d_clk, (uint32_t)t0, cur0);
    ENS_CHECK(cudaStreamSynchronize(e->stream));
    cudaFree(snap);
    if (rc != LB_OK) return rc;
    rc = lb_ens_set_strip_height(e, best);
    if (rc != LB_OK) return rc;
    if (chosen) *chosen = best;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s %d\n", key.c_str(), best);
            fclose(f);
        }
    }
    return LB_OK;
}

}  // extern "C"
