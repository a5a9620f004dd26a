"""lb_conserved_static: the allocation-free mass/momentum entry point for
callers that cannot call cudaMalloc (its partial sums live in a fixed device
array inside the library).  Checked through the C ABI against lb_conserved on
two calls in a row.  Kept in a file of its own that collects last.  The
size and argument checks, which return before any device call, are tested
on the CPU (tests/test_abi_cpu.py)."""
import ctypes as C

import numpy as np
import pytest

from pairs import LN2

pytestmark = pytest.mark.gpu


# The last case is the largest lattice the fixed scratch array takes: all
# 4096 partial triples in use (4096 x 4096 FP32 sites, 604 MB per buffer).
@pytest.mark.parametrize("precision,nx,ny", [("fp32", 256, 128), ("fp64", 132, 36),
                                             ("fp32", 4096, 4096)])
def test_static_scratch_sums_match_lb_conserved(precision, nx, ny):
    torch = pytest.importorskip("torch")
    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.lattice import Lattice
    lat = Lattice(nx, ny, -3.6, 0.9, 1e-4, stencil=4, precision=precision)
    lat.init(LN2, 5, 0.01)
    lat.step(10 if nx * ny < 1 << 20 else 2)
    lat.sync()
    ref = lat.conserved()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")   # caller-owned output
    L = abi.load()
    prec = abi.LB_FP32 if precision == "fp32" else abi.LB_FP64
    for _ in range(2):
        out.fill_(float("nan"))
        rc = L.lb_conserved_static(lat.device_ptr(abi.LB_PTR_POPULATIONS), prec, nx, ny, LN2,
                                   C.c_void_p(out.data_ptr()), lat.stream())
        assert rc == abi.LB_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - ref[0]) <= 1e-12 * ref[0]
        assert np.abs(got[1:] - ref[1:]).max() <= 1e-12 * ref[0]
    lat.close()
