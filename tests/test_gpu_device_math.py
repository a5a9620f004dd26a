"""The FP32 device math of the step kernel against FP64 references: the
expm1 used for the pseudopotential deviation, the hardware Box-Muller pair
(same 32-bit Philox words as the FP64 path), and the ring Box-Muller of the
step kernels against the oracle's FP64 pair."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2212_07848_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("devmath") / "libdevmath.so")
    subprocess.run(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-O3", "-shared", "-Xcompiler", "-fPIC", "-I", CSRC, "-o", out,
                    os.path.join(HERE, "device_math_probe.cu")], check=True)
    L = C.CDLL(out)
    f32 = np.ctypeslib.ndpointer(np.float32)
    L.probe_expm1.argtypes = [f32, f32, C.c_int]
    L.probe_box_muller.argtypes = [np.ctypeslib.ndpointer(np.uint32), f32, C.c_int]
    L.probe_box_ring.argtypes = [np.ctypeslib.ndpointer(np.uint32), f32, C.c_int]
    return L


def test_expm1_relative_error(probe):
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-0.25, 0.25, 200000), rng.uniform(-3, 3, 200000),
                        np.array([0.0, 1e-30, -1e-30, 0.25, -0.25, 0.2500001, -0.2500001])])
    x = x.astype(np.float32)
    y = np.zeros_like(x)
    assert probe.probe_expm1(x, y, len(x)) == 0
    ref = np.expm1(x.astype(np.float64))
    nz = ref != 0
    rel = np.abs(y[nz] - ref[nz]) / np.abs(ref[nz])
    small = np.abs(x[nz]) <= 0.25
    assert rel[small].max() < 4e-7
    assert rel[~small].max() < 3e-6
    assert y[np.flatnonzero(x == 0.0)[0]] == 0.0


def test_box_muller_against_fp64(probe):
    rng = np.random.default_rng(1)
    n = 400000
    r = rng.integers(0, 2 ** 32, size=2 * n, dtype=np.uint64).astype(np.uint32)
    # include the extreme words on both inputs
    r[:8] = np.array([0, 0, 0xFFFFFFFF, 0xFFFFFFFF, 0, 0xFFFFFFFF, 0xFFFFFF00, 12345], np.uint32)
    z = np.zeros(2 * n, np.float32)
    assert probe.probe_box_muller(r, z, n) == 0
    u1 = (r[0::2].astype(np.float64) + 0.5) * 2.0 ** -32
    u2 = (r[1::2].astype(np.float64) + 0.5) * 2.0 ** -32
    rad = np.sqrt(-2.0 * np.log(u1))
    ref = np.empty(2 * n)
    ref[0::2] = rad * np.cos(2 * np.pi * u2)
    ref[1::2] = rad * np.sin(2 * np.pi * u2)
    err = np.abs(z - ref)
    assert np.quantile(err, 0.9999) < 1e-5
    assert err.max() < 1e-3
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_ring_box_muller_against_oracle(probe):
    from oracle import oracle as O
    rng = np.random.default_rng(2)
    n = 200000
    r = np.empty(2 * n, np.uint32)
    r[0::2] = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    r[1::2] = rng.integers(0, 1024, size=n).astype(np.uint32)
    r[0:8] = np.array([0, 0, 0xFFFFFFFF, 1023, 0xFFFFFF00, 512, 12345, 255], np.uint32)
    z = np.zeros(2 * n, np.float32)
    assert probe.probe_box_ring(r, z, n) == 0
    ref = np.array([O.box_muller_ring(int(r[2 * i]), int(r[2 * i + 1])) for i in range(4000)])
    err = np.abs(z[:8000].reshape(-1, 2) - ref)
    assert err.max() < 1e-3 and np.quantile(err, 0.999) < 1e-5
    # full sample against the FP64 closed form of the same mapping
    u1 = (r[0::2].astype(np.float64) + 0.5) * 2.0 ** -32
    th = 2 * np.pi * (r[1::2].astype(np.float64) + 0.5) / 1024
    rad = np.sqrt(-2.0 * np.log(u1))
    e2 = np.abs(z.reshape(-1, 2) - np.stack([rad * np.cos(th), rad * np.sin(th)], axis=1))
    assert np.quantile(e2, 0.9999) < 1e-5 and e2.max() < 1e-3
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
