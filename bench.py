"""Throughput of the fluctuating Shan-Chen D2Q9 hot path on GB300.

Workload (synthetic, the paper's kind of run): a periodic 4096 x 4096 lattice,
FP32 deviation storage, psi = 1 - exp(-rho), E4 force stencil, G = -5.0
(T_hat = 0.8), tau = 1, rho0 = ln 2 (critical quench on the unstable branch),
kT = 1e-6, seed 100.  One benchmark step is one sampling interval of that
run: 500 fused lattice steps, one S(k) sample (row + column FFT and FP64
accumulation), the FP64 mass/momentum reduction and the radial S(k) read-out.
The populations (1.2 GB for both buffers) exceed the 129 MB L2, so no flush is
needed between timed iterations.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
import argparse
import ctypes as C
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fluctuating Shan-Chen D2Q9 MLUPS, % HBM roofline; ensemble & surrogate speedup"
WORKLOAD = "d2q9_4096sq_fp32_G-5.0_quench"
NX = NY = 4096
G, TAU, KT, SEED = -5.0, 1.0, 1e-6, 100
RHO0 = float(np.log(2.0))
LB_PER_STEP = 500            # lattice steps per benchmark step (the S(k) interval)
NBINS = NX // 2
BYTES_PER_SITE = 72          # 9 FP32 loads + 9 FP32 stores per site update
ORACLE_SAMPLE = (512, 512, 240)  # CPU baseline: lattice and steps of the bounded sample (~20 s of CPU time)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _step_kernel_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    valid only while the kernel source is unchanged (else None)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_4096sq_fp32_E4.json")
    try:
        with open(path) as f:
            d = json.load(f)
        h = hashlib.sha256()
        for name in d["source_files"]:
            with open(os.path.join(ROOT, "paper_2212_07848_gb300", "csrc", name), "rb") as f:
                h.update(f.read())
        if d.get("source_sha256") != h.hexdigest():
            return None
        return float(d["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock and throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline():
    """The FP64 oracle as it stands on the host cores, on a bounded sample of
    the workload: ORACLE_SAMPLE lattice and steps, then one S(k) sample."""
    from oracle import oracle as O
    nx, ny, steps = ORACLE_SAMPLE
    o = O.OracleLattice(nx, ny, G, TAU, KT)
    o.init(RHO0, SEED, 0.0)
    t0 = time.perf_counter()
    o.step(steps)
    o.sk_sample_now()
    dt = time.perf_counter() - t0
    cores = O.threads()
    # one core: a quarter of the sample (the site loops are the same code)
    O.set_threads(1)
    try:
        o1 = O.OracleLattice(nx // 2, ny // 2, G, TAU, KT)
        o1.init(RHO0, SEED, 0.0)
        t1 = time.perf_counter()
        o1.step(steps)
        dt1 = time.perf_counter() - t1
    finally:
        O.set_threads(cores)
    return {"value": nx * ny * steps / dt / 1e6, "unit": "MLUPS", "cores": cores,
            "kind": "oracle",
            "single_core_mlups": (nx // 2) * (ny // 2) * steps / dt1 / 1e6,
            "sample": f"{nx}x{ny} lattice, {steps} steps of the same physics (G=-5.0, "
                      f"rho0=ln2, kT=1e-6, E4, FP64) plus one direct-DFT S(k) sample; "
                      f"{dt:.1f} s on {cores} threads; one thread: {nx // 2}x{ny // 2}, "
                      f"{steps} steps, {dt1:.1f} s"}


def ensemble_leg(stream_ptr, steps=20000, seq_steps=200, nrep=256, seed=7):
    """Batched ensemble vs the plain per-replica method on the same GPU: 256
    replicas with sides drawn from {64, 128, 256, 512}, G ~ U[-4.8, -3.6],
    rho0 = ln2 (1 + U[-0.1, 0.1]), kT = 1e-6, S(k) every 50 steps.  The
    ensemble runs the whole 2e4-step workload with an autotuned strip
    height, once with one launch per step and once with one persistent
    launch per window of steps (both from captured graphs; the faster
    counts); the plain method steps each replica's own context in turn on
    one stream, timed over the first `seq_steps` steps of the same runs (its
    rate per site update does not change along the run).  All draw the same
    noise, so every replica's S(k) over those first steps must agree."""
    import torch

    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.ensemble import Ensemble
    from paper_2212_07848_gb300.lattice import Lattice
    rng = np.random.default_rng(seed)
    sizes = rng.choice([64, 128, 256, 512], size=nrep)
    Gs = rng.uniform(-4.8, -3.6, nrep)
    rhos = RHO0 * (1.0 + rng.uniform(-0.1, 0.1, nrep))
    reps = [(int(n), int(n), float(g), 1.0, 1e-6, float(r)) for n, g, r in zip(sizes, Gs, rhos)]
    sites = sum(r[0] * r[1] for r in reps)
    stream = torch.cuda.ExternalStream(stream_ptr)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    timings = {}
    for mode in (abi.LB_ENS_PER_STEP, abi.LB_ENS_PERSISTENT):
        e = Ensemble(reps, seed=seed, stream=stream_ptr)
        e.set_launch(mode)
        e.init(0.0)
        e.sk_config(50, 50)
        strip = e.autotune(10)
        e.sync()
        a.record(stream)
        e.step(steps)
        b.record(stream)
        b.synchronize()
        e.sync()
        timings[mode] = a.elapsed_time(b)
        e.close()
    ens_ms = min(timings.values())
    # the S(k) check: the first seq_steps + 50 steps of the ensemble against
    # the per-replica runs below
    ens = Ensemble(reps, seed=seed, stream=stream_ptr)
    ens.init(0.0)
    ens.sk_config(50, 50)
    ens.step(50 + seq_steps)
    lats = []
    for r, (nx, ny, g, tau, kT, rho0) in enumerate(reps):
        lat = Lattice(nx, ny, g, tau, kT, stream=stream_ptr)
        lat.set_replica(r)
        lat.init(rho0, seed, 0.0)
        lat.sk_config(50, 50)
        lat.step(50)
        lats.append(lat)
    torch.cuda.synchronize()
    a.record(stream)
    for lat in lats:
        lat.step(seq_steps)
    b.record(stream)
    b.synchronize()
    seq_ms = a.elapsed_time(b)
    worst = 0.0
    for r, lat in enumerate(lats):
        se, _ = ens.structure_factor(r)
        sq, _ = lat.structure_factor()
        worst = max(worst, float(np.max(np.abs(se - sq) / (np.abs(sq) + 1e-300))))
        lat.close()
    ens.close()
    ens_rate = sites * steps / (ens_ms * 1e-3)
    seq_rate = sites * seq_steps / (seq_ms * 1e-3)
    return {"replicas": nrep, "sites": sites, "steps": steps, "strip_h": strip,
            "per_step_launch_mlups": sites * steps / (timings[abi.LB_ENS_PER_STEP] * 1e-3) / 1e6,
            "persistent_launch_mlups":
                sites * steps / (timings[abi.LB_ENS_PERSISTENT] * 1e-3) / 1e6,
            "ensemble_mlups": ens_rate / 1e6, "ensemble_run_s": ens_ms * 1e-3,
            "sequential_mlups": seq_rate / 1e6, "sequential_steps_timed": seq_steps,
            "speedup": ens_rate / seq_rate, "sk_max_rel_diff": worst,
            "sizes": "uniform {64,128,256,512}^2, G~U[-4.8,-3.6], rho0=ln2(1+U[-0.1,0.1])"}


def ensemble_small_leg(stream_ptr, steps=2000, seed=7):
    """Ensembles of small replicas (4.2 M sites each: 1024 x 64^2, 4096 x
    32^2, 256 x 128^2; G ~ U[-4.8, -3.6], rho0 = ln2, kT = 1e-6, S(k) every
    50 steps, persistent launches): replicas resident in shared memory for
    each window of steps against the same replicas as tiles.  The 128^2
    replicas are resident over clusters of four CTAs (distributed shared
    memory); the others in one CTA each."""
    import torch

    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.ensemble import Ensemble
    stream = torch.cuda.ExternalStream(stream_ptr)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for side, nrep in ((64, 1024), (32, 4096), (128, 256)):
        rng = np.random.default_rng(seed)
        reps = [(side, side, float(g), 1.0, 1e-6, RHO0) for g in rng.uniform(-4.8, -3.6, nrep)]
        sites = side * side * nrep
        row = {"replicas": nrep, "sites": sites, "steps": steps}
        for name, mode in (("resident", abi.LB_ENS_RESIDENT_ON),
                           ("tiled", abi.LB_ENS_RESIDENT_OFF)):
            e = Ensemble(reps, seed=seed, stream=stream_ptr)
            e.set_resident(mode)
            e.set_launch(abi.LB_ENS_PERSISTENT)
            e.init(0.0)
            e.sk_config(50, 50)
            e.autotune(10)
            e.step(50)
            e.sync()
            a.record(stream)
            e.step(steps)
            b.record(stream)
            b.synchronize()
            e.sync()
            row[name + "_mlups"] = sites * steps / (a.elapsed_time(b) * 1e-3) / 1e6
            if mode == abi.LB_ENS_RESIDENT_ON:
                row["resident_replicas"] = e.num_resident
            e.close()
        row["speedup"] = row["resident_mlups"] / row["tiled_mlups"]
        out[f"{side}sq"] = row
    return out


def conv_layer_leg(nb=8, h=128, cin=64, cout=128, reps=20):
    """The surrogate's widest convolution (64 -> 128 channels on 8 images of
    128^2, BF16 operands, FP32 accumulation, bias + ReLU) on the path the
    network takes, forward and input gradient: mean time per call over
    `reps` calls replayed from a captured CUDA graph (no host gaps), TFLOP/s
    at 2 * 9 * cin * cout FLOP per output pixel, and the fraction of the
    measured BF16 peak (burst: the layer is timed alone)."""
    import torch

    from paper_2212_07848_gb300 import abi
    L = abi.load()
    p = lambda t: C.c_void_p(t.data_ptr())
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn((nb, h, h, cin), generator=g).to(torch.bfloat16).cuda()
    w = (0.1 * torch.randn((9, cout, cin), generator=g)).to(torch.bfloat16).cuda()
    b = torch.zeros(cout, device="cuda")
    y = torch.empty((nb, h, h, cout), dtype=torch.bfloat16, device="cuda")
    dy = torch.randn((nb, h, h, cout), generator=g).to(torch.bfloat16).cuda()
    dx = torch.empty_like(x)
    st = torch.cuda.Stream()
    fwd = lambda: L.lb_nn_conv3x3(p(x), p(w), p(b), p(y), nb, h, h, cin, cout, 1, 0,
                                  C.c_void_p(st.cuda_stream))
    bwd = lambda: L.lb_nn_conv3x3(p(dy), p(w), None, p(dx), nb, h, h, cout, cin, 0, 1,
                                  C.c_void_p(st.cuda_stream))
    peak = _bf16_peak()
    flop = 2.0 * 9 * cin * cout * nb * h * h
    out = {"layer": f"{nb}x{h}^2 {cin}->{cout}", "peak_tflops": peak[0], "peak_kind": peak[1]}
    for name, call in (("forward", fwd), ("input_gradient", bwd)):
        with torch.cuda.stream(st):
            for _ in range(3):
                if call() != 0:
                    raise RuntimeError("lb_nn_conv3x3 failed")
            st.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=st):
                for _ in range(reps):
                    call()
            graph.replay()
            st.synchronize()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            graph.replay()
            e.record(st)
            e.synchronize()
        us = a.elapsed_time(e) * 1e3 / reps
        out[name] = {"us": us, "tflops": flop / (us * 1e-6) / 1e12,
                     "frac": flop / (us * 1e-6) / 1e12 / peak[0]}
    if L.lb_nn_status() != 0:
        raise RuntimeError("a tensor-core wait gave up")
    return out


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured burst"
    except Exception:
        return 1900.0, "fallback"


def surrogate_leg(ntraj=64, ntest=8, size=2048, steps=6000, stride=200, iters=9000, batch=8,
                  seed=11):
    """Learned surrogate against the solver it stands in for: quench
    trajectories at size^2 (G ~ U[-5.2, -4.4], rho0 = ln2, kT = 1e-6)
    coarse-grained 4x every `stride` steps; the network is trained (Adam,
    cosine learning rate, pushforward over one or two strides) on all but `ntest`, which score
    it: one-stride MSE against persistence, and rollouts scored by the solver
    on the ensemble-mean L(t) and radial S(k, t), next to the same metrics for
    the solver itself continued on an independent noise stream (the floor of
    any predictor of a stochastic run).  The speedup is the solver's
    time for `stride` steps at size^2 over the surrogate's time for one stride
    at (size/4)^2."""
    import torch

    from paper_2212_07848_gb300 import surrogate as S
    from paper_2212_07848_gb300.lattice import Lattice
    frames, Gs, gen_s = S.generate(ntraj, size, steps, stride, seed0=seed * 1000)
    m = size // 4
    net = S.SurrogateNet(m, batch, seed=seed)
    train_ids, test_ids = list(range(ntraj - ntest)), list(range(ntraj - ntest, ntraj))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.train(net, frames, Gs, train_ids, iters, lr=2e-3, lr_end=1e-5, seed=seed, pushforward=0.5,
            pf_depth=2)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    mse, persist = S.one_step_mse(net, frames, Gs, test_ids)
    rollouts = {}
    for f0, nroll in ((5, 10), (10, 20)):
        ev = S.evaluate_rollouts(net, frames, Gs, test_ids, f0, nroll)
        rollouts[f"t={f0 * stride}..{(f0 + nroll) * stride}"] = {
            "L_mean_max_rel_err": ev["L_mean_max_rel_err"],
            "L_traj_max_rel_err": ev["L_traj_max_rel_err"],
            "Sk_peak_max_rel_err": ev["Sk_peak_max_rel_err"],
            "Sk_l1_rel_err": ev["Sk_l1_rel_err"]}
    # the floor: the solver itself continued from the same states on an
    # independent noise stream, scored by the same ensemble metrics
    floor = {}
    for f0, nroll in ((5, 10), (10, 20)):
        ev = S.solver_reseeded(frames, Gs, test_ids, f0, nroll, size, stride, seed * 1000)
        floor[f"t={f0 * stride}..{(f0 + nroll) * stride}"] = {
            "L_mean_max_rel_err": ev["L_mean_max_rel_err"],
            "L_traj_max_rel_err": ev["L_traj_max_rel_err"],
            "Sk_peak_max_rel_err": ev["Sk_peak_max_rel_err"],
            "Sk_l1_rel_err": ev["Sk_l1_rel_err"]}
    k, f0 = test_ids[0], 5
    x0, p0 = frames[k, f0].clone(), frames[k, f0 - 1].clone()
    S.rollout(net, x0, float(Gs[k]), 3, p0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    S.rollout(net, x0, float(Gs[k]), 20, p0)
    b.record()
    b.synchronize()
    sur_ms = a.elapsed_time(b) / 20
    lat = Lattice(size, size, float(Gs[k]), 1.0, 1e-6)
    lat.init(RHO0, 5, 0.0)
    lat.step(stride)
    lat.sync()
    st = torch.cuda.ExternalStream(lat.stream())
    a.record(st)
    lat.step(5 * stride)
    b.record(st)
    b.synchronize()
    lb_ms = a.elapsed_time(b) / 5
    lat.close()
    return {"lattice": f"{size}^2 -> {m}^2 (4x coarse)", "stride": stride,
            "trajectories": ntraj, "test_trajectories": ntest, "train_iters": iters,
            "batch": batch, "generate_s": gen_s, "train_s": train_s,
            "heldout_mse": mse, "persistence_mse": persist, "mse_ratio": mse / persist,
            "rollouts": rollouts, "solver_reseeded": floor,
            "surrogate_ms_per_stride": sur_ms, "solver_ms_per_stride": lb_ms,
            "speedup": lb_ms / sur_ms}


def d3q19_leg(n=256, steps=40, strips=(16, 32, 64)):
    """The D3Q19 step (the paper's three-dimensional setting) on an n^3 FP32
    lattice (G = -5.0, rho0 = ln 2, kT = 1e-6): MLUPS and the fraction of the
    measured HBM bandwidth at 152 algorithmic bytes per site (19 FP32 loads +
    19 stores), for the fastest of a few z-strip heights."""
    import torch

    from paper_2212_07848_gb300.lattice3 import Lattice3
    st = torch.cuda.Stream()
    lat = Lattice3(n, n, n, G, TAU, KT, stream=st.cuda_stream)
    lat.init(RHO0, SEED, 0.0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for strip in strips:
        lat.set_strip(strip)
        lat.step(5)
        lat.sync()
        a.record(st)
        lat.step(steps)
        b.record(st)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        if best is None or ms < best[1]:
            best = (strip, ms)
    lat.close()
    sites = n ** 3
    peak, kind = _peaks()
    gbs = 152.0 * sites / (best[1] * 1e-3) / 1e9
    return {"lattice": f"{n}^3 FP32 D3Q19", "strip_z": best[0], "ms_per_step": best[1],
            "mlups": sites / (best[1] * 1e-3) / 1e6, "bytes_per_site": 152,
            "achieved_gbs": gbs, "hbm_frac": gbs / peak, "peak_kind": kind}


def l2_assisted_leg(n=1024, steps=2000, strips=(8, 9, 12, 16, 32)):
    """The 1024^2 lattice of the metastable density sweep (FP32, E4, G = -4.5,
    rho0 = 0.33 on the gas branch between coexistence and spinodal, kT =
    1e-6): its 75 MB of populations fit the 129 MB L2, so its rate is
    L2-assisted and is reported apart from the HBM-bound headline; the
    fastest of a few strip heights (a 1024^2 lattice fills only about one
    wave of CTAs, so the strip height decides the halo share and the tail)."""
    import torch

    from paper_2212_07848_gb300.lattice import Lattice
    lat = Lattice(n, n, -4.5, TAU, KT, stencil=4, precision="fp32")
    lat.init(0.33, SEED, 0.0)
    lat.step(200)
    lat.sync()
    st = torch.cuda.ExternalStream(lat.stream())
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for strip in strips:
        lat.set_strip_height(strip)
        lat.step(50)
        a.record(st)
        lat.step(steps)
        b.record(st)
        b.synchronize()
        t = a.elapsed_time(b) / steps
        if best is None or t < best[1]:
            best = (strip, t)
    lat.close()
    ms = best[1]
    sites = n * n
    # the same lattice as a one-replica ensemble in persistent windows: tiles
    # start a step as soon as their neighbours finished the previous one, so
    # there is no launch boundary or tail per step
    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.ensemble import Ensemble
    pbest = None
    est = torch.cuda.Stream()
    e = Ensemble([(n, n, -4.5, TAU, KT, 0.33)], seed=SEED, stream=est.cuda_stream)
    e.set_launch(abi.LB_ENS_PERSISTENT)
    e.set_kernel(abi.LB_KERNEL_OVERLAP)
    e.init(0.0)
    for strip in (4, 6, 8):
        e.set_strip_height(strip)
        e.step(64)
        e.sync()
        a.record(est)
        e.step(steps)
        b.record(est)
        b.synchronize()
        e.sync()
        t = a.elapsed_time(b) / steps
        if pbest is None or t < pbest[1]:
            pbest = (strip, t)
    e.close()
    return {"lattice": f"{n}^2 FP32 E4, G=-4.5, rho0=0.33", "strip_h": best[0], "ms_per_step": ms,
            "mlups": sites / (ms * 1e-3) / 1e6,
            "equivalent_gbs": BYTES_PER_SITE * sites / (ms * 1e-3) / 1e9,
            "persistent_windows": {"strip_h": pbest[0], "ms_per_step": pbest[1],
                                   "mlups": sites / (pbest[1] * 1e-3) / 1e6},
            "note": "populations (75 MB) resident in L2; not an HBM figure"}


def c1_fp64_leg(n=128, steps=2000, sample_from=1001, strips=(1, 2, 4, 8)):
    """The 128^2 FP64 configuration (psi = 1 - exp(-rho), E4, G = -3.6, rho0 =
    ln 2, tau = 1, kT = 1e-5, seed 0): the whole run, 2000 steps with S(k)
    sampled every step over the last 1000 and the radial read-out, timed
    with CUDA events for the fastest of a few strip heights, plus the step
    kernel alone over the first 1000 steps.  144 algorithmic bytes per site
    (9 FP64 loads + 9 stores); the 2.4 MB of populations stay in L2 and a
    128^2 lattice gives only 4 to 64 CTAs, so the bound is launch latency and
    the FP64 pipe, not HBM."""
    import torch

    from paper_2212_07848_gb300.lattice import Lattice
    best = None
    bins = np.empty(n // 2 + 2)
    for strip in strips:
        lat = Lattice(n, n, -3.6, 1.0, 1e-5, stencil=4, precision="fp64")
        lat.set_strip_height(strip)
        st = torch.cuda.ExternalStream(lat.stream())
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        for rep in range(2):                      # the first pass warms up
            lat.init(RHO0, 0, 0.0)
            lat.sk_config(1, sample_from)
            lat.sync()
            ev[0].record(st)
            lat.step(sample_from - 1)
            ev[1].record(st)
            lat.step(steps - sample_from + 1)
            lat.structure_factor(nbins=len(bins))
            ev[2].record(st)
            ev[2].synchronize()
        lat.close()
        total = ev[0].elapsed_time(ev[2])
        plain = ev[0].elapsed_time(ev[1]) / (sample_from - 1)
        if best is None or total < best[1]:
            best = (strip, total, plain)
    strip, total, plain = best
    sites = n * n
    peak, kind = _peaks()
    gbs = 144.0 * sites / (plain * 1e-3) / 1e9
    return {"lattice": f"{n}^2 FP64 E4, G=-3.6, rho0=ln2, kT=1e-5", "strip_h": strip,
            "run_ms": total, "run_mlups": sites * steps / (total * 1e-3) / 1e6,
            "step_ms": plain, "step_mlups": sites / (plain * 1e-3) / 1e6,
            "bytes_per_site": 144, "equivalent_gbs": gbs, "hbm_frac": gbs / peak,
            "peak_kind": kind,
            "bound": "FP64 arithmetic latency (2.4 MB L2-resident lattice: 128 CTAs of one row, a few warps per SM; steps replayed from captured windows)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    per = []
    cb = None
    for _ in range(args.warmup):
        cpu_baseline()
    for _ in range(args.steps):
        cb = cpu_baseline()
        per.append(cb["value"])
    value = statistics.median(per)
    cb["value"] = value
    nx, ny, steps = ORACLE_SAMPLE
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": nx * ny * steps / (value * 1e6) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "sample_lattice": [nx, ny],
                   "sample_steps": steps},
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300 import replicas as R
    from paper_2212_07848_gb300.lattice import Lattice

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    lat = Lattice(NX, NY, G, TAU, KT, stencil=4, precision="fp32", device=local_rank)
    lat.init(RHO0, R.replica_seed(SEED, rank), 0.0)
    lat.sk_config(LB_PER_STEP, LB_PER_STEP)
    stream = torch.cuda.ExternalStream(lat.stream())
    bins = np.empty(NBINS)
    h = lat.handle
    L = abi.load()
    conserved = np.zeros(3)
    dptr = conserved.ctypes.data_as(C.POINTER(C.c_double))

    def one_step(ev_k1=None):
        # 499 plain steps, then the sampling step (writes delta rho) + S(k) sample
        if ev_k1 is not None:
            ev_k1[0].record(stream)
        rc = L.lb_step(h, LB_PER_STEP - 1)
        if ev_k1 is not None:
            ev_k1[1].record(stream)
        rc |= L.lb_step(h, 1)
        rc |= L.lb_conserved(h, conserved)
        if rc != 0:
            raise abi.LbError(rc, "bench step")
        abi.lb_structure_factor(h, bins, NBINS)

    for _ in range(args.warmup):
        one_step()
    lat.sync()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    k1_events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local_rank) as clk:
        start.record(stream)
        for k in range(args.steps):
            one_step(k1_events[k])
        end.record(stream)
        end.synchronize()
    lat.sync()
    ms = start.elapsed_time(end)
    k1_ms = sum(a.elapsed_time(b) for a, b in k1_events) / (args.steps * (LB_PER_STEP - 1))
    ms_max = R.max_over_ranks(ms, dist, device="cuda")
    sites = NX * NY
    value = R.whole_job_rate(sites * LB_PER_STEP * args.steps, world, ms_max * 1e-3) / 1e6

    # end-to-end through the C ABI with host buffers: per step, upload the
    # state from pinned host memory, run the interval, read back the density
    # and the radial S(k).
    state = torch.empty(9 * sites, dtype=torch.float32, pin_memory=True)
    dens = torch.empty(sites, dtype=torch.float64, pin_memory=True)
    state_np, dens_np = state.numpy(), dens.numpy()
    lat.download_state(state_np.reshape(9, NY, NX))
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        abi.lb_upload_state(h, state_np.ctypes.data_as(C.c_void_p))
        rc = L.lb_step(h, LB_PER_STEP)
        if rc != 0:
            raise abi.LbError(rc, "e2e step")
        abi.lb_density(h, dens_np)
        abi.lb_structure_factor(h, bins, NBINS)
    lat.sync()
    e2e_s = time.perf_counter() - t0
    e2e_max = R.max_over_ranks(e2e_s, dist, device="cuda")
    e2e_value = R.whole_job_rate(sites * LB_PER_STEP * e2e_steps, world, e2e_max) / 1e6

    peak, peak_kind = _peaks()
    achieved = BYTES_PER_SITE * sites / (k1_ms * 1e-3) / 1e9
    cb = cpu_baseline() if (rank == 0 and world == 1) else None
    ens = None
    if rank == 0 and world == 1 and not args.no_ensemble:
        ens = ensemble_leg(lat.stream())
    sur = None
    if rank == 0 and world == 1 and not args.no_surrogate:
        sur = surrogate_leg()
        sur["conv_layer"] = conv_layer_leg()
    d3 = None
    if rank == 0 and world == 1 and not args.no_3d:
        d3 = d3q19_leg()
    extras = rank == 0 and world == 1 and not args.no_extras
    small = ensemble_small_leg(lat.stream()) if extras else None
    l2 = l2_assisted_leg() if extras else None
    c1 = c1_fp64_leg() if extras else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "G": G, "tau": TAU, "kT": KT,
                       "rho0": "ln2", "stencil": "E4", "lb_steps_per_step": LB_PER_STEP,
                       "sk_sample_every": LB_PER_STEP, "nbins": NBINS,
                       "l2": "inputs larger than L2 (1.21 GB of populations), no flush",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "kernel": "step_kernel_ov<float,4> (unit relaxation)",
                         "kernel_ms": k1_ms, "bytes_per_site": BYTES_PER_SITE,
                         "traffic": _step_kernel_traffic()},
            "e2e": {"value": e2e_value, "unit": "MLUPS",
                    "h2d_bytes_per_step": state_np.nbytes,
                    "d2h_bytes_per_step": dens_np.nbytes + bins.nbytes,
                    "steps": e2e_steps},
            "clocks": clk.summary(),
            # per step: the lattice steps, one device-clock set per captured
            # 32-step window, the S(k) sample (2), the reduction (2), the bins (1)
            "gpu_launches": args.steps * (LB_PER_STEP + (LB_PER_STEP - 1) // 32 + 2 + 2 + 1),
        }
        if cb is not None:
            line["cpu_baseline"] = cb
        if ens is not None:
            line["ensemble"] = ens
        if sur is not None:
            line["surrogate"] = sur
        if d3 is not None:
            line["d3q19"] = d3
        if small is not None:
            line["ensemble_small"] = small
        if l2 is not None:
            line["l2_assisted_1024sq"] = l2
        if c1 is not None:
            line["c1_fp64_128sq"] = c1
        print(json.dumps(line), flush=True)
    lat.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the batched-ensemble vs per-replica leg")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the learned-surrogate leg")
    ap.add_argument("--no-3d", action="store_true", help="skip the D3Q19 leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the small-replica ensembles, 1024^2 L2-resident and 128^2 "
                         "FP64 legs")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    from paper_2212_07848_gb300.replicas import rank_info
    rank, world, local_rank = rank_info(1)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        from paper_2212_07848_gb300 import build
        if world == 1:
            build.build()   # under torchrun the library is built before launch
        run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
