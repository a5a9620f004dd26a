// C ABI of liblbsc.so (declared in include/lbsc.h): context management,
// argument checking, the time loop and host <-> device transfers.  Every
// computation on the lattice runs in the kernels of lbsc_step.cu,
// lbsc_sk.cu and lbsc_reduce.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <limits.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "lbsc.h"
#include "lbsc_internal.cuh"

using namespace lbsc;

struct lb_ctx {
    lb_params p;
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t esize = 4;               // bytes per stored value
    size_t n = 0;                   // nx * ny
    void *df[2] = {nullptr, nullptr};
    int cur = 0;
    int *d_flag = nullptr;
    double *d_partials = nullptr;
    double *d_out = nullptr;        // small device results (conserved sums, bins)
    int nred = 0;
    double *d_io = nullptr;         // nx*ny doubles for density / read-outs (lazy)
    // structure factor (lazy, powers of two only)
    void *drho = nullptr;
    void *spec = nullptr;
    double *acc = nullptr;
    void *tw_x = nullptr, *tw_y = nullptr;
    int ldx = 0;
    int sk_every = 0;
    long long sk_start = 0, sk_count = 0;
    // state
    bool inited = false;
    double rho0 = 0.0;
    uint64_t seed = 0;
    uint32_t replica = 0;
    long long t = 0;
    int strip_h = 32;
    int kernel_mode = 0;            // LB_KERNEL_*
    TmaMaps maps;                   // tensor maps of df[0], df[1] (FP32 only)
    long long wait_ns = -1;         // staged kernel's mbarrier bound (< 0: default)
    StepArgs base;
    // captured windows of steps: [starting buffer][0: 32 plain steps, 1: one
    // S(k) interval ending with its sample, 2: 32 steps sampling at every
    // step]; the step counter of the noise is read from d_clock, set before
    // each replay
    uint32_t *d_clock = nullptr;
    cudaGraphExec_t graph[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    int graph_len[2][3] = {{0, 0, 0}, {0, 0, 0}};
    long long graph_ver[2][3] = {{-1, -1, -1}, {-1, -1, -1}};
    long long ver = 0;              // bumped by every change that a captured window bakes in
    bool graphs_ok = true;          // false once a capture failed (e.g. the legacy stream)
};

namespace {

constexpr double kCs2 = 1.0 / 3.0;
// Norms b_k = sum_i w_i e_ki^2 of the Hermite modes k = 3..8 (basis in the header).
constexpr double kB[6] = {4.0, 4.0 / 9.0, 1.0 / 9.0, 2.0 / 3.0, 2.0 / 3.0, 16.0};
constexpr double kW[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                          1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return LB_OK;
    if (e == cudaErrorMemoryAllocation) return LB_ERR_NOMEM;
    return LB_ERR_CUDA;
}

#define LB_CHECK(call)                          \
    do {                                        \
        cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

int validate(const lb_params *p) {
    if (!p) return LB_ERR_ARG;
    if (p->nx < 4 || p->ny < 4 || p->nx % 4 || p->ny % 4) return LB_ERR_ARG;
    // 32-bit element indices in the kernels: 9 nx ny < 2^32
    if (9.0 * (double)p->nx * (double)p->ny >= 4294967296.0) return LB_ERR_ARG;
    if (!(p->tau > 0.5) || !isfinite(p->tau)) return LB_ERR_ARG;
    if (p->tau_bulk != 0.0 && (!(p->tau_bulk > 0.5) || !isfinite(p->tau_bulk))) return LB_ERR_ARG;
    if (p->tau_ghost != 0.0 && (!(p->tau_ghost > 0.5) || !isfinite(p->tau_ghost))) return LB_ERR_ARG;
    if (!(p->kT >= 0.0) || !isfinite(p->kT)) return LB_ERR_ARG;
    if (!isfinite(p->G)) return LB_ERR_ARG;
    if (p->stencil != 4 && p->stencil != 6 && p->stencil != 8) return LB_ERR_ARG;
    if (p->precision != LB_FP32 && p->precision != LB_FP64) return LB_ERR_ARG;
    if (p->psi_kind == LB_PSI_EXP) return LB_OK;
    if (p->psi_kind == LB_PSI_CRITICAL || p->psi_kind == LB_PSI_AEXP) {
        if (!(p->psi_p1 > 0.0) || !(p->psi_p2 > 0.0)) return LB_ERR_ARG;
        return LB_OK;
    }
    return LB_ERR_ARG;
}

int default_strip(int nx, int ny) {
    const bool ov = nx >= 1024;   // the overlapped kernel (see lb_get_kernel)
    const long gx = ov ? (nx + kStepTX - 3) / (kStepTX - 2) : (nx + kStepTX - 1) / kStepTX;
    long target = (long)ny * gx / (152 * 4);
    int h = 8;
    while (h < 32 && h * 2 <= target) h *= 2;
    // the overlapped kernel measured fastest at 24 rows per CTA (4096^2)
    if (ov && h == 32) h = 24;
    if (h > ny) h = ny;
    return h;
}

double psi_of(const lb_params &p, double rho) {
    switch (p.psi_kind) {
    case LB_PSI_EXP: return -expm1(-rho);
    case LB_PSI_CRITICAL: return sqrt(p.psi_p1 * p.psi_p2) * exp(1.0 - p.psi_p2 / rho);
    default: return p.psi_p1 * exp(-p.psi_p2 / rho);
    }
}

void fill_base(lb_ctx *h) {
    StepArgs &a = h->base;
    const lb_params &p = h->p;
    memset(&a, 0, sizeof(a));
    a.nx = p.nx;
    a.ny = p.ny;
    a.strip_h = h->strip_h;
    a.rho0 = h->rho0;
    a.force_pref = -p.G * kCs2;
    a.psi_kind = p.psi_kind;
    a.psi0 = psi_of(p, h->rho0);
    a.psi_c = p.psi_kind == LB_PSI_EXP ? exp(-h->rho0) : a.psi0;
    a.psi_b = p.psi_kind == LB_PSI_EXP ? 0.0 : p.psi_p2;
    const double tb = p.tau_bulk > 0.0 ? p.tau_bulk : p.tau;
    const double tg = p.tau_ghost > 0.0 ? p.tau_ghost : p.tau;
    a.gamma = 1.0 - 1.0 / p.tau;
    a.gamma_b = 1.0 - 1.0 / tb;
    a.gamma_g = 1.0 - 1.0 / tg;
    const double mu = p.kT / kCs2;
    const double gk[6] = {a.gamma_b, a.gamma, a.gamma, a.gamma_g, a.gamma_g, a.gamma_g};
    for (int k = 0; k < 6; ++k) a.noise_amp[k] = sqrt(mu * kB[k] * (1.0 - gk[k] * gk[k]));
    philox_round_keys(h->seed, a.round_keys);
    a.replica = h->replica;
    a.noise = p.kT > 0.0 ? 1 : 0;
    a.flag = h->d_flag;
}

int ensure_io(lb_ctx *h) {
    if (h->d_io) return LB_OK;
    const size_t n = h->n > 8192 ? h->n : 8192;   // also holds 2 x 4096 radial bins
    LB_CHECK(cudaMalloc(&h->d_io, n * sizeof(double)));
    return LB_OK;
}

int ensure_sk(lb_ctx *h) {
    if (h->acc) return LB_OK;
    const int nx = h->p.nx, ny = h->p.ny;
    if (!is_pow2(nx) || !is_pow2(ny)) return LB_ERR_UNSUPPORTED;
    const int maxn = h->p.precision == LB_FP32 ? 8192 : 4096;
    if (nx > maxn || ny > maxn) return LB_ERR_UNSUPPORTED;
    h->ldx = ((nx / 2 + 1) + 3) / 4 * 4;
    const size_t cs = 2 * h->esize;
    LB_CHECK(cudaMalloc(&h->drho, h->n * h->esize));
    LB_CHECK(cudaMalloc(&h->spec, (size_t)ny * h->ldx * cs));
    LB_CHECK(cudaMalloc(&h->acc, (size_t)ny * h->ldx * sizeof(double)));
    LB_CHECK(cudaMalloc(&h->tw_x, (size_t)(nx / 2) * cs));
    LB_CHECK(cudaMalloc(&h->tw_y, (size_t)(ny / 2) * cs));
    LB_CHECK(cudaMemsetAsync(h->acc, 0, (size_t)ny * h->ldx * sizeof(double), h->stream));
    LB_CHECK(launch_twiddles(h->p.precision, h->tw_x, nx, h->stream));
    LB_CHECK(launch_twiddles(h->p.precision, h->tw_y, ny, h->stream));
    h->sk_count = 0;
    return LB_OK;
}

int sample_sk(lb_ctx *h) {
    SkArgs s;
    s.drho = h->drho;
    s.spec = h->spec;
    s.acc = h->acc;
    s.tw_x = h->tw_x;
    s.tw_y = h->tw_y;
    s.nx = h->p.nx;
    s.ny = h->p.ny;
    s.ldx = h->ldx;
    LB_CHECK(launch_sk_sample(h->p.precision, s, h->stream));
    h->sk_count += 1;
    return LB_OK;
}

int select_device(lb_ctx *h) {
    LB_CHECK(cudaSetDevice(h->dev));
    return LB_OK;
}

void drop_step_graphs(lb_ctx *h) {
    for (auto &row : h->graph)
        for (auto &g : row) {
            if (g) cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

void free_all(lb_ctx *h) {
    drop_step_graphs(h);
    cudaFree(h->d_clock);
    cudaFree(h->df[0]);
    cudaFree(h->df[1]);
    cudaFree(h->d_flag);
    cudaFree(h->d_partials);
    cudaFree(h->d_out);
    cudaFree(h->d_io);
    cudaFree(h->drho);
    cudaFree(h->spec);
    cudaFree(h->acc);
    cudaFree(h->tw_x);
    cudaFree(h->tw_y);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

}  // namespace

namespace lbsc {
void philox_round_keys(uint64_t seed, uint32_t rk[20]) {
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0;
        rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;   // golden ratio, 2^32 (phi - 1)
        k1 += 0xBB67AE85u;   // 2^32 (sqrt(3) - 1)
    }
}
}  // namespace lbsc

extern "C" {

int lb_params_init(lb_params *p) {
    if (!p) return LB_ERR_ARG;
    memset(p, 0, sizeof(*p));
    p->nx = 128;
    p->ny = 128;
    p->G = -3.6;
    p->tau = 1.0;
    p->kT = 0.0;
    p->psi_kind = LB_PSI_EXP;
    p->stencil = 4;
    p->precision = LB_FP32;
    p->stream = nullptr;
    p->device = -1;
    return LB_OK;
}

int lb_create_ex(lb_ctx **out, const lb_params *p) {
    if (!out) return LB_ERR_ARG;
    *out = nullptr;
    int rc = validate(p);
    if (rc != LB_OK) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return LB_ERR_CUDA;
    lb_ctx *h = new (std::nothrow) lb_ctx();
    if (!h) return LB_ERR_NOMEM;
    h->p = *p;
    if (p->device >= 0) {
        if (p->device >= ndev || cudaSetDevice(p->device) != cudaSuccess) {
            delete h;
            return LB_ERR_ARG;
        }
    }
    cudaGetDevice(&h->dev);
    h->esize = p->precision == LB_FP32 ? sizeof(float) : sizeof(double);
    h->n = (size_t)p->nx * p->ny;
    if (p->stream) {
        h->stream = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return LB_ERR_CUDA;
        }
        h->own_stream = true;
    }
    h->nred = conserved_blocks(p->nx, p->ny);
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&h->df[b], 9 * h->n * h->esize);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_clock, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_partials, 3 * (size_t)h->nred * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_out, 4096 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) {
        free_all(h);
        delete h;
        return cuda_status(e);
    }
    h->strip_h = default_strip(p->nx, p->ny);
    if (tma_eligible(p->precision, p->nx, p->ny))
        tma_encode_maps(&h->maps, h->df[0], h->df[1], p->nx, p->ny);
    fill_base(h);
    *out = h;
    return LB_OK;
}

int lb_create(lb_ctx **out, int nx, int ny, double G, double tau, double kT, int psi_kind,
              int stencil) {
    lb_params p;
    lb_params_init(&p);
    p.nx = nx;
    p.ny = ny;
    p.G = G;
    p.tau = tau;
    p.kT = kT;
    p.psi_kind = psi_kind;
    p.stencil = stencil;
    return lb_create_ex(out, &p);
}

void lb_destroy(lb_ctx *h) {
    if (!h) return;
    cudaSetDevice(h->dev);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

int lb_init(lb_ctx *h, double rho0, uint64_t seed, double init_amp) {
    if (!h || !(rho0 > 0.0) || !isfinite(rho0) || !isfinite(init_amp)) return LB_ERR_ARG;
    int rc = select_device(h);
    if (rc) return rc;
    h->rho0 = rho0;
    h->seed = seed;
    h->t = 0;
    h->cur = 0;
    fill_base(h);
    ++h->ver;
    LB_CHECK(launch_init(h->p.precision, h->df[0], h->p.nx, h->p.ny, init_amp,
                         h->base.round_keys, h->replica, h->stream));
    if (h->acc) {
        LB_CHECK(cudaMemsetAsync(h->acc, 0, (size_t)h->p.ny * h->ldx * sizeof(double), h->stream));
    }
    h->sk_count = 0;
    h->inited = true;
    return LB_OK;
}

int lb_set_replica(lb_ctx *h, uint32_t replica) {
    if (!h) return LB_ERR_ARG;
    h->replica = replica;
    h->base.replica = replica;
    ++h->ver;
    return LB_OK;
}

int lb_set_strip_height(lb_ctx *h, int rows) {
    if (!h || rows < 1 || rows > h->p.ny) return LB_ERR_ARG;
    h->strip_h = rows;
    h->base.strip_h = rows;
    ++h->ver;
    return LB_OK;
}

int lb_set_kernel(lb_ctx *h, int mode) {
    if (!h || mode < LB_KERNEL_AUTO || mode > LB_KERNEL_OVERLAP) return LB_ERR_ARG;
    if (mode == LB_KERNEL_TMA && !h->maps.ok) return LB_ERR_UNSUPPORTED;
    h->kernel_mode = mode;
    ++h->ver;
    return LB_OK;
}

int lb_set_wait_ns(lb_ctx *h, long long ns) {
    if (!h) return LB_ERR_ARG;
    h->wait_ns = ns < 0 ? -1 : ns;
    ++h->ver;
    return LB_OK;
}

int lb_get_kernel(const lb_ctx *h) {
    if (!h) return LB_ERR_ARG;
    // AUTO: on GB300 the overlapped-strip kernel is the fastest for lattices
    // at least 1024 columns wide (the step is issue-bound; without a halo warp
    // every resident warp collides, 8 CTAs of 4 warps per SM instead of 6 of
    // 5: 73 against 67 GLUPS at 4096^2), while narrower lattices lose more to
    // its partly filled last strip (a power-of-two width leaves a strip of a
    // few columns) and take the halo-warp kernel.  The staged kernel's per-row
    // mbarrier hand-off costs more than the loads it saves.
    if (h->kernel_mode == LB_KERNEL_TMA && h->maps.ok) return LB_KERNEL_TMA;
    if (h->kernel_mode == LB_KERNEL_PLAIN) return LB_KERNEL_PLAIN;
    if (h->kernel_mode == LB_KERNEL_OVERLAP) return LB_KERNEL_OVERLAP;
    return h->p.nx >= 1024 ? LB_KERNEL_OVERLAP : LB_KERNEL_PLAIN;
}

namespace {

__global__ void clock_set_kernel(uint32_t *clock, uint32_t t) { *clock = t; }

// The first step after t that takes an S(k) sample (LLONG_MAX: none).
long long next_sample(const lb_ctx *h, long long t) {
    if (h->sk_every <= 0 || !h->acc) return LLONG_MAX;
    if (t + 1 <= h->sk_start) return h->sk_start;
    const long long r = (t + 1 - h->sk_start) % h->sk_every;
    return r == 0 ? t + 1 : t + 1 + (h->sk_every - r);
}

// One step on the stream (the launch loop's body; len-step windows capture
// the same launches with the step counter read from d_clock).
cudaError_t launch_one(lb_ctx *h, int kern, int buf, bool sample, uint32_t step,
                       const uint32_t *clock) {
    StepArgs a = h->base;
    a.src = h->df[buf];
    a.dst = h->df[buf ^ 1];
    a.drho_out = sample ? h->drho : nullptr;
    a.step = step;
    a.clock = clock;
    a.wait_ns = h->wait_ns;
    a.layout = kern == LB_KERNEL_OVERLAP ? 1 : 0;
    if (kern == LB_KERNEL_TMA) return launch_step_tma(h->p.stencil, a, h->maps, buf, h->stream);
    return launch_step(h->p.precision, h->p.stencil, a, h->stream);
}

// Capture `len` steps from buffer h->cur; sampling S(k) at the last step
// (kind 1) or at every step (kind 2); LB_ERR_UNSUPPORTED if the stream
// cannot be captured.
int capture_steps(lb_ctx *h, int kern, int len, int kind, cudaGraphExec_t *out) {
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return LB_ERR_UNSUPPORTED;
    }
    SkArgs sk;
    sk.drho = h->drho;
    sk.spec = h->spec;
    sk.acc = h->acc;
    sk.tw_x = h->tw_x;
    sk.tw_y = h->tw_y;
    sk.nx = h->p.nx;
    sk.ny = h->p.ny;
    sk.ldx = h->ldx;
    cudaError_t err = cudaSuccess;
    int buf = h->cur;
    for (int j = 0; j < len && err == cudaSuccess; ++j, buf ^= 1) {
        const bool sample = kind == 2 || (kind == 1 && j == len - 1);
        err = launch_one(h, kern, buf, sample, (uint32_t)j, h->d_clock);
        if (err == cudaSuccess && sample) err = launch_sk_sample(h->p.precision, sk, h->stream);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (err != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return LB_ERR_UNSUPPORTED;
    }
    err = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    LB_CHECK(err);
    return LB_OK;
}

}  // namespace

// Steps run as replays of captured windows where they can: 32 steps with no
// sampling step inside, one sampling interval ending with its sample, or 32
// steps that all sample (bit-identical to the launch loop: the same kernels,
// with the noise counter read from the device).  The rest, and the staged
// kernel, are single launches.
int lb_step(lb_ctx *h, int n) {
    if (!h || n < 0) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    int rc = select_device(h);
    if (rc) return rc;
    const int kern = lb_get_kernel(h);
    constexpr int kWindow = 32;
    constexpr int kMaxWindow = 1024;   // longest sampling interval captured whole
    while (n > 0) {
        const long long t = h->t, ns = next_sample(h, t);
        int kind = -1, len = 0;
        if (h->graphs_ok && kern != LB_KERNEL_TMA) {
            if (n >= kWindow && ns > t + kWindow) {
                kind = 0;
                len = kWindow;
            } else if (h->sk_every >= 2 && h->sk_every <= kMaxWindow && n >= h->sk_every &&
                       ns == t + h->sk_every) {
                kind = 1;
                len = h->sk_every;
            } else if (h->sk_every == 1 && n >= kWindow && ns == t + 1) {
                kind = 2;
                len = kWindow;
            }
        }
        if (kind >= 0) {
            cudaGraphExec_t &g = h->graph[h->cur][kind];
            if (!g || h->graph_ver[h->cur][kind] != h->ver || h->graph_len[h->cur][kind] != len) {
                if (g) cudaGraphExecDestroy(g);
                g = nullptr;
                rc = capture_steps(h, kern, len, kind, &g);
                if (rc == LB_ERR_UNSUPPORTED) {
                    h->graphs_ok = false;   // take single launches from now on
                    continue;
                }
                if (rc) return rc;
                h->graph_ver[h->cur][kind] = h->ver;
                h->graph_len[h->cur][kind] = len;
            }
            clock_set_kernel<<<1, 1, 0, h->stream>>>(h->d_clock, (uint32_t)t);
            LB_CHECK(cudaGetLastError());
            LB_CHECK(cudaGraphLaunch(g, h->stream));
            h->t = t + len;
            h->cur ^= len & 1;
            if (kind == 1) h->sk_count += 1;
            if (kind == 2) h->sk_count += len;
            n -= len;
            continue;
        }
        const bool sample = ns == t + 1;
        LB_CHECK(launch_one(h, kern, h->cur, sample, (uint32_t)t, nullptr));
        h->cur ^= 1;
        h->t = t + 1;
        if (sample) {
            rc = sample_sk(h);
            if (rc) return rc;
        }
        n -= 1;
    }
    return LB_OK;
}

int lb_sync(lb_ctx *h) {
    if (!h) return LB_ERR_ARG;
    int rc = select_device(h);
    if (rc) return rc;
    LB_CHECK(cudaStreamSynchronize(h->stream));
    int flag = 0;
    LB_CHECK(cudaMemcpy(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        LB_CHECK(cudaMemset(h->d_flag, 0, sizeof(int)));
        return (flag & LB_STEP_TIMEOUT) ? LB_ERR_TIMEOUT : LB_ERR_NONFINITE;
    }
    return LB_OK;
}

long long lb_get_step(const lb_ctx *h) { return h ? h->t : -1; }

int lb_set_step(lb_ctx *h, long long t) {
    if (!h || t < 0) return LB_ERR_ARG;
    h->t = t;
    return LB_OK;
}

int lb_density(lb_ctx *h, double *host_out) {
    if (!h || !host_out) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    int rc = select_device(h);
    if (rc) return rc;
    rc = ensure_io(h);
    if (rc) return rc;
    LB_CHECK(launch_density(h->p.precision, h->df[h->cur], h->rho0, h->d_io, h->p.nx, h->p.ny,
                            h->stream));
    LB_CHECK(cudaMemcpyAsync(host_out, h->d_io, h->n * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    return lb_sync(h);
}

int lb_download_state(lb_ctx *h, void *host_df) {
    if (!h || !host_df) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    int rc = select_device(h);
    if (rc) return rc;
    LB_CHECK(cudaMemcpyAsync(host_df, h->df[h->cur], 9 * h->n * h->esize, cudaMemcpyDeviceToHost,
                             h->stream));
    return lb_sync(h);
}

int lb_upload_state(lb_ctx *h, const void *host_df) {
    if (!h || !host_df) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    int rc = select_device(h);
    if (rc) return rc;
    LB_CHECK(cudaMemcpyAsync(h->df[h->cur], host_df, 9 * h->n * h->esize, cudaMemcpyHostToDevice,
                             h->stream));
    LB_CHECK(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb_populations(lb_ctx *h, double *host_out) {
    if (!h || !host_out) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    const size_t n = h->n;
    std::vector<unsigned char> tmp;
    try {
        tmp.resize(9 * n * h->esize);
    } catch (...) {
        return LB_ERR_NOMEM;
    }
    int rc = lb_download_state(h, tmp.data());
    if (rc) return rc;
    for (int i = 0; i < 9; ++i) {
        const double base = kW[i] * h->rho0;
        if (h->p.precision == LB_FP32) {
            const float *d = (const float *)tmp.data() + i * n;
            for (size_t s = 0; s < n; ++s) host_out[i * n + s] = base + (double)d[s];
        } else {
            const double *d = (const double *)tmp.data() + i * n;
            for (size_t s = 0; s < n; ++s) host_out[i * n + s] = base + d[s];
        }
    }
    return LB_OK;
}

int lb_set_populations(lb_ctx *h, const double *host_in) {
    if (!h || !host_in) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    const size_t n = h->n;
    std::vector<unsigned char> tmp;
    try {
        tmp.resize(9 * n * h->esize);
    } catch (...) {
        return LB_ERR_NOMEM;
    }
    for (int i = 0; i < 9; ++i) {
        const double base = kW[i] * h->rho0;
        if (h->p.precision == LB_FP32) {
            float *d = (float *)tmp.data() + i * n;
            for (size_t s = 0; s < n; ++s) d[s] = (float)(host_in[i * n + s] - base);
        } else {
            double *d = (double *)tmp.data() + i * n;
            for (size_t s = 0; s < n; ++s) d[s] = host_in[i * n + s] - base;
        }
    }
    return lb_upload_state(h, tmp.data());
}

int lb_set_density(lb_ctx *h, const double *host_rho) {
    if (!h || !host_rho) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    const size_t n = h->n;
    std::vector<double> f;
    try {
        f.resize(9 * n);
    } catch (...) {
        return LB_ERR_NOMEM;
    }
    for (int i = 0; i < 9; ++i)
        for (size_t s = 0; s < n; ++s) f[i * n + s] = kW[i] * host_rho[s];
    return lb_set_populations(h, f.data());
}

int lb_sk_config(lb_ctx *h, int sample_every, long long start_step) {
    if (!h || sample_every < 0 || start_step < 0) return LB_ERR_ARG;
    int rc = select_device(h);
    if (rc) return rc;
    if (sample_every > 0) {
        rc = ensure_sk(h);
        if (rc) return rc;
    }
    h->sk_every = sample_every;
    h->sk_start = start_step;
    ++h->ver;
    return LB_OK;
}

int lb_sk_reset(lb_ctx *h) {
    if (!h) return LB_ERR_ARG;
    int rc = select_device(h);
    if (rc) return rc;
    if (h->acc) {
        LB_CHECK(cudaMemsetAsync(h->acc, 0, (size_t)h->p.ny * h->ldx * sizeof(double), h->stream));
    }
    h->sk_count = 0;
    return LB_OK;
}

int lb_sk_sample_now(lb_ctx *h) {
    if (!h) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    int rc = select_device(h);
    if (rc) return rc;
    rc = ensure_sk(h);
    if (rc) return rc;
    LB_CHECK(launch_drho(h->p.precision, h->df[h->cur], h->drho, h->p.nx, h->p.ny, h->stream));
    return sample_sk(h);
}

int lb_structure_factor(lb_ctx *h, double *host_out, int nbins, long long *nsamples_out) {
    if (!h || !host_out || nbins < 0 || nbins > 4096) return LB_ERR_ARG;
    int rc = select_device(h);
    if (rc) return rc;
    if (!h->acc) return LB_ERR_STATE;
    const double inv = h->sk_count > 0 ? 1.0 / (double)h->sk_count : 0.0;
    const int nx = h->p.nx, ny = h->p.ny;
    if (nbins == 0) {
        rc = ensure_io(h);
        if (rc) return rc;
        LB_CHECK(launch_sk_readout(h->acc, inv, h->d_io, nx, ny, h->ldx, h->stream));
        LB_CHECK(cudaMemcpyAsync(host_out, h->d_io, (size_t)(nx / 2 + 1) * ny * sizeof(double),
                                 cudaMemcpyDeviceToHost, h->stream));
    } else {
        rc = ensure_io(h);
        if (rc) return rc;
        double *bins = h->d_io, *counts = h->d_io + nbins;
        LB_CHECK(cudaMemsetAsync(h->d_io, 0, 2 * (size_t)nbins * sizeof(double), h->stream));
        LB_CHECK(launch_sk_bins(h->acc, inv, bins, counts, nbins, nx, ny, h->ldx, h->stream));
        std::vector<double> tmp(2 * (size_t)nbins);
        LB_CHECK(cudaMemcpyAsync(tmp.data(), h->d_io, 2 * (size_t)nbins * sizeof(double),
                                 cudaMemcpyDeviceToHost, h->stream));
        rc = lb_sync(h);
        if (rc) return rc;
        for (int b = 0; b < nbins; ++b)
            host_out[b] = tmp[nbins + b] > 0 ? tmp[b] / tmp[nbins + b] : NAN;
    }
    if (nsamples_out) *nsamples_out = h->sk_count;
    return lb_sync(h);
}

int lb_sk_moments(lb_ctx *h, double out[2]) {
    if (!h || !out) return LB_ERR_ARG;
    int rc = select_device(h);
    if (rc) return rc;
    if (!h->acc) return LB_ERR_STATE;
    const double inv = h->sk_count > 0 ? 1.0 / (double)h->sk_count : 0.0;
    LB_CHECK(launch_sk_moments(h->acc, inv, h->p.nx, h->p.ny, h->ldx, h->d_out, h->stream));
    LB_CHECK(cudaMemcpyAsync(out, h->d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return lb_sync(h);
}

int lb_structure_factor_counts(lb_ctx *h, long long *host_counts, int nbins) {
    if (!h || !host_counts || nbins <= 0 || nbins > 4096) return LB_ERR_ARG;
    const int nx = h->p.nx, ny = h->p.ny;
    const double L = (double)(nx > ny ? nx : ny);
    for (int b = 0; b < nbins; ++b) host_counts[b] = 0;
    for (int ky = 0; ky < ny; ++ky) {
        const int my = ky <= ny / 2 ? ky : ky - ny;
        for (int kx = 0; kx <= nx / 2; ++kx) {
            if (kx == 0 && ky == 0) continue;
            const double qx = (double)kx * (L / nx), qy = (double)my * (L / ny);
            const int b = (int)rint(sqrt(qx * qx + qy * qy));
            if (b >= nbins) continue;
            host_counts[b] += (kx == 0 || 2 * kx == nx) ? 1 : 2;
        }
    }
    return LB_OK;
}

int lb_conserved(lb_ctx *h, double out[3]) {
    if (!h || !out) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    int rc = select_device(h);
    if (rc) return rc;
    LB_CHECK(launch_conserved(h->p.precision, h->df[h->cur], h->d_partials, h->nred, h->d_out,
                              h->p.nx, h->p.ny, h->stream));
    double tmp[3];
    LB_CHECK(cudaMemcpyAsync(tmp, h->d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    rc = lb_sync(h);
    if (rc) return rc;
    out[0] = (double)h->n * h->rho0 + tmp[0];
    out[1] = tmp[1];
    out[2] = tmp[2];
    return LB_OK;
}

// ---- checkpoint -----------------------------------------------------------
namespace {
const char kMagic[8] = {'L', 'B', 'S', 'C', '0', '0', '0', '2'};
struct CkptHeader {
    char magic[8];
    int32_t nx, ny, precision, stencil, psi_kind, sk_every, has_acc, pad;
    double G, tau, kT, p1, p2, rho0, tau_bulk, tau_ghost;
    uint64_t seed;
    uint32_t replica, pad2;
    int64_t t, sk_start, sk_count;
};
}  // namespace

int lb_save(lb_ctx *h, const char *path) {
    if (!h || !path) return LB_ERR_ARG;
    if (!h->inited) return LB_ERR_STATE;
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, kMagic, 8);
    hd.nx = h->p.nx;
    hd.ny = h->p.ny;
    hd.precision = h->p.precision;
    hd.stencil = h->p.stencil;
    hd.psi_kind = h->p.psi_kind;
    hd.sk_every = h->sk_every;
    hd.has_acc = h->acc ? 1 : 0;
    hd.G = h->p.G;
    hd.tau = h->p.tau;
    hd.kT = h->p.kT;
    hd.p1 = h->p.psi_p1;
    hd.p2 = h->p.psi_p2;
    hd.rho0 = h->rho0;
    hd.tau_bulk = h->p.tau_bulk;
    hd.tau_ghost = h->p.tau_ghost;
    hd.seed = h->seed;
    hd.replica = h->replica;
    hd.t = h->t;
    hd.sk_start = h->sk_start;
    hd.sk_count = h->sk_count;
    std::vector<unsigned char> df;
    std::vector<double> acc;
    try {
        df.resize(9 * h->n * h->esize);
        if (h->acc) acc.resize((size_t)h->p.ny * h->ldx);
    } catch (...) {
        return LB_ERR_NOMEM;
    }
    int rc = lb_download_state(h, df.data());
    if (rc) return rc;
    if (h->acc) {
        LB_CHECK(cudaMemcpy(acc.data(), h->acc, acc.size() * sizeof(double),
                            cudaMemcpyDeviceToHost));
    }
    FILE *f = fopen(path, "wb");
    if (!f) return LB_ERR_IO;
    bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(df.data(), 1, df.size(), f) == df.size();
    if (ok && h->acc) ok = fwrite(acc.data(), sizeof(double), acc.size(), f) == acc.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? LB_OK : LB_ERR_IO;
}

int lb_load(lb_ctx *h, const char *path) {
    if (!h || !path) return LB_ERR_ARG;
    int rc = select_device(h);
    if (rc) return rc;
    FILE *f = fopen(path, "rb");
    if (!f) return LB_ERR_IO;
    CkptHeader hd;
    if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, kMagic, 8) != 0) {
        fclose(f);
        return LB_ERR_IO;
    }
    if (hd.nx != h->p.nx || hd.ny != h->p.ny || hd.precision != h->p.precision) {
        fclose(f);
        return LB_ERR_ARG;
    }
    lb_params np = h->p;
    np.stencil = hd.stencil;
    np.psi_kind = hd.psi_kind;
    np.G = hd.G;
    np.tau = hd.tau;
    np.kT = hd.kT;
    np.psi_p1 = hd.p1;
    np.psi_p2 = hd.p2;
    np.tau_bulk = hd.tau_bulk;
    np.tau_ghost = hd.tau_ghost;
    if (validate(&np) != LB_OK) {
        fclose(f);
        return LB_ERR_IO;
    }
    std::vector<unsigned char> df;
    std::vector<double> acc;
    try {
        df.resize(9 * h->n * h->esize);
    } catch (...) {
        fclose(f);
        return LB_ERR_NOMEM;
    }
    bool ok = fread(df.data(), 1, df.size(), f) == df.size();
    if (ok && hd.has_acc) {
        if (ensure_sk(h) != LB_OK) {
            fclose(f);
            return LB_ERR_UNSUPPORTED;
        }
        acc.resize((size_t)h->p.ny * h->ldx);
        ok = fread(acc.data(), sizeof(double), acc.size(), f) == acc.size();
    }
    fclose(f);
    if (!ok) return LB_ERR_IO;
    h->p = np;
    h->rho0 = hd.rho0;
    h->seed = hd.seed;
    h->replica = hd.replica;
    h->t = hd.t;
    h->sk_every = hd.sk_every;
    h->sk_start = hd.sk_start;
    h->sk_count = hd.sk_count;
    h->cur = 0;
    h->inited = true;
    fill_base(h);
    ++h->ver;
    LB_CHECK(cudaMemcpyAsync(h->df[0], df.data(), df.size(), cudaMemcpyHostToDevice, h->stream));
    if (hd.has_acc) {
        LB_CHECK(cudaMemcpyAsync(h->acc, acc.data(), acc.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, h->stream));
    }
    LB_CHECK(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

void *lb_device_ptr(lb_ctx *h, int which) {
    if (!h) return nullptr;
    switch (which) {
    case LB_PTR_POPULATIONS: return h->df[h->cur];
    case LB_PTR_DENSITY_SAMPLE: return h->drho;
    case LB_PTR_SK_ACCUM: return h->acc;
    }
    return nullptr;
}

void *lb_stream(lb_ctx *h) { return h ? (void *)h->stream : nullptr; }

const char *lb_strerror(int code) {
    switch (code) {
    case LB_OK: return "ok";
    case LB_ERR_ARG: return "invalid argument";
    case LB_ERR_CUDA: return "CUDA error";
    case LB_ERR_NONFINITE: return "non-finite value produced by the step";
    case LB_ERR_TIMEOUT: return "bounded device wait timed out";
    case LB_ERR_UNSUPPORTED: return "unsupported configuration";
    case LB_ERR_IO: return "file input/output error";
    case LB_ERR_NOMEM: return "out of memory";
    case LB_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

}  // extern "C"
