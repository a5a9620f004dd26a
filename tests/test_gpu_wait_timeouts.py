"""Failure detection of the bounded device waits: each wait is shortened from
the host so that a wait whose data does arrive gives up at its first check,
the kernel leaves cleanly (copies and MMAs it issued are waited for with the
default bound, tensor memory is freed only after that), the timeout reaches
the host as LB_ERR_TIMEOUT, and the context stays usable: with the default
bound restored, a re-initialised run reproduces a fresh one bit for bit.
No wait here is on data that never arrives."""
import ctypes as C

import numpy as np
import pytest

from pairs import LN2

pytestmark = pytest.mark.gpu


def test_staged_step_mbarrier_timeout_is_reported_and_recoverable():
    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.lattice import Lattice

    def lattice(kernel):
        g = Lattice(512, 128, -3.6, 1.0, 1e-5, stencil=4, precision="fp32")
        g.set_kernel(kernel)
        g.init(LN2, 21, 0.01)
        return g

    g = lattice(abi.LB_KERNEL_TMA)
    assert g.kernel == abi.LB_KERNEL_TMA
    abi.lb_set_wait_ns(g._h, 0)
    g.step(3)
    with pytest.raises(abi.LbError) as e:
        g.sync()
    assert e.value.code == abi.LB_ERR_TIMEOUT
    g.sync()                                   # the flag was cleared
    abi.lb_set_wait_ns(g._h, -1)               # default bound again
    g.init(LN2, 21, 0.01)
    g.step(20)
    g.sync()
    ref = lattice(abi.LB_KERNEL_PLAIN)
    ref.step(20)
    ref.sync()
    assert np.array_equal(g.download_state(), ref.download_state())


def test_persistent_ensemble_barrier_timeout_is_reported_and_recoverable():
    from paper_2212_07848_gb300 import abi
    from paper_2212_07848_gb300.ensemble import Ensemble
    reps = [(512, 512, -4.4, 1.0, 1e-6, LN2), (256, 512, -3.8, 0.9, 1e-6, 0.7),
            (128, 128, -4.6, 1.0, 1e-6, LN2)]
    a = Ensemble(reps, seed=9)
    a.set_launch(abi.LB_ENS_PERSISTENT)
    a.set_strip_height(8)
    a.init(0.01)
    abi.lb_ens_set_wait_ns(a._h, 0)
    a.step(64)                                 # two persistent windows
    with pytest.raises(abi.LbError) as e:
        a.sync()
    assert e.value.code == abi.LB_ERR_TIMEOUT
    a.sync()
    abi.lb_ens_set_wait_ns(a._h, -1)
    a.init(0.01)
    a.step(40)
    a.sync()
    b = Ensemble(reps, seed=9)                 # per-step launches, never timed out
    b.set_strip_height(8)
    b.init(0.01)
    b.step(40)
    b.sync()
    for r in range(len(reps)):
        assert np.array_equal(a.populations(r), b.populations(r)), r


@pytest.mark.parametrize("path", [2, 3])    # per-tile and persistent tcgen05 kernels
def test_tensor_core_conv_mma_wait_timeout_is_reported_and_recoverable(path):
    torch = pytest.importorskip("torch")
    from paper_2212_07848_gb300 import abi
    L = abi.load()
    P = C.c_void_p
    L.lb_nn_conv3x3.argtypes = [P, P, P, P] + [C.c_int] * 7 + [P]
    p = lambda t: C.c_void_p(t.data_ptr())
    nb, h, w, cin, cout = 2, 8, 128, 32, 128
    gen = torch.Generator(device="cpu").manual_seed(4)
    x = torch.randn((nb, h, w, cin), generator=gen).to(torch.bfloat16).cuda()
    wt = (0.1 * torch.randn((9, cout, cin), generator=gen)).to(torch.bfloat16).cuda()
    b = torch.randn(cout, generator=gen).cuda()
    y0 = torch.empty((nb, h, w, cout), dtype=torch.bfloat16, device="cuda")
    y1 = torch.zeros_like(y0)
    assert L.lb_nn_set_conv_path(path) == 0    # a tcgen05 kernel wherever it has one
    try:
        assert L.lb_nn_conv3x3(p(x), p(wt), p(b), p(y0), nb, h, w, cin, cout, 1, 0, None) == 0
        assert L.lb_nn_status() == abi.LB_OK
        abi.lb_nn_set_wait_ns(0)
        assert L.lb_nn_conv3x3(p(x), p(wt), p(b), p(y1), nb, h, w, cin, cout, 1, 0, None) == 0
        assert L.lb_nn_status() == abi.LB_ERR_TIMEOUT
        assert L.lb_nn_status() == abi.LB_OK  # cleared
    finally:
        abi.lb_nn_set_wait_ns(-1)
    # tensor memory was released: further launches allocate it and finish
    for _ in range(3):
        assert L.lb_nn_conv3x3(p(x), p(wt), p(b), p(y1), nb, h, w, cin, cout, 1, 0, None) == 0
    assert L.lb_nn_status() == abi.LB_OK
    assert torch.equal(y0, y1)
    assert L.lb_nn_set_conv_path(0) == 0


def test_tensor_core_wgrad_wait_timeout_is_reported_and_recoverable():
    """The tcgen05 weight-gradient kernel: a wait given up at its first check
    is reported, tensor memory is released, and the next calls give the
    earlier bits."""
    torch = pytest.importorskip("torch")
    from paper_2212_07848_gb300 import abi
    L = abi.load()
    P = C.c_void_p
    L.lb_nn_conv3x3_wgrad.argtypes = [P, P, P, P] + [C.c_int] * 5 + [P, C.c_size_t, P]
    L.lb_nn_wgrad_workspace.argtypes = [C.c_int] * 5
    L.lb_nn_wgrad_workspace.restype = C.c_size_t
    p = lambda t: C.c_void_p(t.data_ptr())
    nb, h, w, cin, cout = 2, 16, 256, 32, 64
    gen = torch.Generator(device="cpu").manual_seed(5)
    x = torch.randn((nb, h, w, cin), generator=gen).to(torch.bfloat16).cuda()
    dy = torch.randn((nb, h, w, cout), generator=gen).to(torch.bfloat16).cuda()
    nbytes = L.lb_nn_wgrad_workspace(nb, h, w, cin, cout)
    ws = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    dw0 = torch.zeros((9, cout, cin), device="cuda")
    dw1 = torch.zeros_like(dw0)
    call = lambda dw: L.lb_nn_conv3x3_wgrad(p(x), p(dy), p(dw), None, nb, h, w, cin, cout, p(ws),
                                            nbytes, None)
    assert L.lb_nn_set_conv_path(0) == 0
    assert call(dw0) == 0
    assert L.lb_nn_status() == abi.LB_OK
    try:
        abi.lb_nn_set_wait_ns(0)
        assert call(dw1) == 0
        assert L.lb_nn_status() == abi.LB_ERR_TIMEOUT
        assert L.lb_nn_status() == abi.LB_OK  # cleared
    finally:
        abi.lb_nn_set_wait_ns(-1)
    for _ in range(3):
        dw1.zero_()
        assert call(dw1) == 0
    assert L.lb_nn_status() == abi.LB_OK
    assert torch.equal(dw0, dw1)
