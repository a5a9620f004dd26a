"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/lbsc.h declares.  No compute call runs here (no GPU)."""
import ctypes as C
import os
import re

import pytest

from paper_2212_07848_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "lbsc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lb3?_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(abi.EXPORTED) == names


def test_strerror_and_defaults(lib):
    assert abi.lb_strerror(abi.LB_OK) == "ok"
    assert "argument" in abi.lb_strerror(abi.LB_ERR_ARG)
    assert abi.lb_strerror(12345) == "unknown status"
    p = abi.lb_params_init()
    assert (p.nx, p.ny, p.stencil, p.precision, p.device) == (128, 128, 4, abi.LB_FP32, -1)
    assert lib.lb_params_init(None) == abi.LB_ERR_ARG


@pytest.mark.parametrize("nx,ny,G,tau,kT,kind,st", [
    (130, 128, -3.6, 1.0, 0.0, 0, 4),     # nx not a multiple of 4
    (128, 2, -3.6, 1.0, 0.0, 0, 4),       # too small
    (128, 128, -3.6, 0.5, 0.0, 0, 4),     # tau <= 1/2
    (128, 128, -3.6, 1.0, -1e-6, 0, 4),   # kT < 0
    (128, 128, -3.6, 1.0, 0.0, 7, 4),     # unknown psi
    (128, 128, -3.6, 1.0, 0.0, 1, 4),     # psi kind 1 without Tc, nc
    (128, 128, -3.6, 1.0, 0.0, 0, 5),     # unknown stencil
    (128, 128, float("nan"), 1.0, 0.0, 0, 4),
])
def test_invalid_arguments_rejected_before_any_device_call(lib, nx, ny, G, tau, kT, kind, st):
    h = C.c_void_p()
    assert lib.lb_create(C.byref(h), nx, ny, G, tau, kT, kind, st) == abi.LB_ERR_ARG
    assert not h.value


def test_null_handles_are_rejected(lib):
    assert lib.lb_step(None, 1) == abi.LB_ERR_ARG
    assert lib.lb_sync(None) == abi.LB_ERR_ARG
    assert lib.lb_get_step(None) == -1
    lib.lb_destroy(None)


def test_static_conserved_rejects_before_any_device_call(lib):
    """lb_conserved_static checks its sizes and pointers before it touches the
    device: a lattice one row past its 4096 x 4096 scratch limit is
    LB_ERR_UNSUPPORTED, null pointers and bad sizes are LB_ERR_ARG.  The
    pointers are never dereferenced on these paths (no GPU here)."""
    fake = C.c_void_p(0x1000)
    f = lib.lb_conserved_static
    assert f(fake, abi.LB_FP32, 4096, 4097, 0.7, fake, None) == abi.LB_ERR_UNSUPPORTED
    assert f(fake, abi.LB_FP64, 8192, 4096, 0.7, fake, None) == abi.LB_ERR_UNSUPPORTED
    assert f(None, abi.LB_FP32, 4, 4, 0.7, fake, None) == abi.LB_ERR_ARG
    assert f(fake, abi.LB_FP32, 4, 4, 0.7, None, None) == abi.LB_ERR_ARG
    assert f(fake, abi.LB_FP32, 0, 4, 0.7, fake, None) == abi.LB_ERR_ARG
    assert f(fake, 7, 4, 4, 0.7, fake, None) == abi.LB_ERR_ARG
