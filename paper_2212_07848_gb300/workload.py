"""Run one synthetic lattice for a number of steps (profiling and sizing).

    python -m paper_2212_07848_gb300.workload --nx 2048 --ny 2048 --steps 5
    python -m paper_2212_07848_gb300.workload --nx 256 --ny 256 --nz 256 --steps 5   # D3Q19
    python -m paper_2212_07848_gb300.workload --nx 64 --ny 64 --replicas 1024 --steps 64  # ensemble

Defaults to the critical quench of the benchmark (G = -5.0, rho0 = ln 2,
kT = 1e-6, E4, FP32) on a smaller square lattice.  Prints the wall time.
"""
import argparse
import math
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--G", type=float, default=-5.0)
    ap.add_argument("--tau", type=float, default=1.0)
    ap.add_argument("--kT", type=float, default=1e-6)
    ap.add_argument("--rho0", type=float, default=math.log(2.0))
    ap.add_argument("--stencil", type=int, default=4)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--sk-every", type=int, default=0)
    ap.add_argument("--strip", type=int, default=0)
    ap.add_argument("--nz", type=int, default=0, help="> 0: a D3Q19 lattice nx x ny x nz")
    ap.add_argument("--replicas", type=int, default=0,
                    help="> 0: an ensemble of that many nx x ny replicas (G spread over "
                         "[-4.8, -3.6])")
    ap.add_argument("--resident", default="auto", choices=["auto", "on", "off"],
                    help="ensemble replicas in shared memory")
    ap.add_argument("--launch", default="step", choices=["step", "persistent"],
                    help="ensemble launch mode")
    a = ap.parse_args()
    if a.replicas > 0:
        from . import abi
        from .ensemble import Ensemble
        n = a.replicas
        reps = [(a.nx, a.ny, -4.8 + 1.2 * r / max(n - 1, 1), a.tau, a.kT, a.rho0)
                for r in range(n)]
        e = Ensemble(reps, stencil=a.stencil, seed=100)
        e.set_resident({"auto": abi.LB_ENS_RESIDENT_AUTO, "on": abi.LB_ENS_RESIDENT_ON,
                        "off": abi.LB_ENS_RESIDENT_OFF}[a.resident])
        e.set_launch(abi.LB_ENS_PERSISTENT if a.launch == "persistent" else abi.LB_ENS_PER_STEP)
        if a.strip:
            e.set_strip_height(a.strip)
        e.init(0.0)
        if a.sk_every:
            e.sk_config(a.sk_every, a.sk_every)
        t0 = time.perf_counter()
        e.step(a.steps)
        e.sync()
        dt = time.perf_counter() - t0
        print(f"{n} x {a.nx}x{a.ny} ensemble ({e.num_resident} resident, {e.num_tiles} tiles): "
              f"{a.steps} steps in {dt * 1e3:.2f} ms")
        e.close()
        return
    if a.nz > 0:
        from .lattice3 import Lattice3
        lat = Lattice3(a.nx, a.ny, a.nz, a.G, a.tau, a.kT, precision=a.precision)
        if a.strip:
            lat.set_strip(a.strip)
        lat.init(a.rho0, 100, 0.0)
        t0 = time.perf_counter()
        lat.step(a.steps)
        lat.sync()
        dt = time.perf_counter() - t0
        print(f"{a.nx}x{a.ny}x{a.nz} {a.precision} D3Q19: {a.steps} steps in {dt * 1e3:.2f} ms")
        lat.close()
        return
    from .lattice import Lattice
    lat = Lattice(a.nx, a.ny, a.G, a.tau, a.kT, stencil=a.stencil, precision=a.precision)
    if a.strip:
        lat.set_strip_height(a.strip)
    lat.init(a.rho0, 100, 0.0)
    if a.sk_every:
        lat.sk_config(a.sk_every, a.sk_every)
    t0 = time.perf_counter()
    lat.step(a.steps)
    lat.sync()
    dt = time.perf_counter() - t0
    print(f"{a.nx}x{a.ny} {a.precision} E{a.stencil}: {a.steps} steps in {dt * 1e3:.2f} ms")
    lat.close()


if __name__ == "__main__":
    main()
