"""Pin the oracle's Philox4x32-10 (and so the shared noise stream) against
cuRAND's device Philox4_32_10: with key = seed and counter
(0, 0, subsequence), the first two blocks must agree word for word."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("curand") / "libcurand_probe.so")
    subprocess.run(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-shared", "-Xcompiler", "-fPIC", "-o", out,
                    os.path.join(HERE, "curand_probe.cu")], check=True)
    L = C.CDLL(out)
    L.curand_philox_first.argtypes = [C.c_ulonglong, C.c_ulonglong,
                                      np.ctypeslib.ndpointer(np.uint32)]
    return L


@pytest.mark.parametrize("seed,sub", [(0, 0), (1, 0), (0x123456789ABCDEF, 42),
                                      (2 ** 64 - 1, 2 ** 40 + 7)])
def test_oracle_philox_matches_curand(probe, seed, sub):
    got = np.zeros(8, np.uint32)
    assert probe.curand_philox_first(seed, sub, got) == 0
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for blk in range(2):
        ctr = (blk, 0, sub & 0xFFFFFFFF, sub >> 32)
        assert list(O.philox4x32(ctr, key)) == list(got[4 * blk:4 * blk + 4])
