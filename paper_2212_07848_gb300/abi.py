"""ctypes binding of liblbsc.so: the C ABI of include/lbsc.h under the same names.

Argument marshalling only -- every step of the method runs in the CUDA
kernels of the library.  If the library has not been built, or no CUDA
device is usable, the calls raise: there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbsc.so")

LB_OK = 0
LB_ERR_ARG = -1
LB_ERR_CUDA = -2
LB_ERR_NONFINITE = -3
LB_ERR_TIMEOUT = -4
LB_ERR_UNSUPPORTED = -5
LB_ERR_IO = -6
LB_ERR_NOMEM = -7
LB_ERR_STATE = -8

LB_PSI_EXP, LB_PSI_CRITICAL, LB_PSI_AEXP = 0, 1, 2
LB_FP32, LB_FP64 = 0, 1
LB_PTR_POPULATIONS, LB_PTR_DENSITY_SAMPLE, LB_PTR_SK_ACCUM = 0, 1, 2
LB_KERNEL_AUTO, LB_KERNEL_PLAIN, LB_KERNEL_TMA, LB_KERNEL_OVERLAP = 0, 1, 2, 3

# Every function the header declares, for export checks.
EXPORTED = [
    "lb_params_init", "lb_create", "lb_create_ex", "lb_destroy", "lb_init",
    "lb_set_replica", "lb_set_strip_height", "lb_step", "lb_sync", "lb_get_step",
    "lb_set_step", "lb_density", "lb_populations", "lb_set_populations",
    "lb_set_density", "lb_upload_state", "lb_download_state", "lb_sk_config",
    "lb_sk_reset", "lb_sk_sample_now", "lb_structure_factor",
    "lb_structure_factor_counts", "lb_conserved", "lb_save", "lb_load",
    "lb_device_ptr", "lb_stream", "lb_strerror", "lb_conserved_static",
    "lb_set_kernel", "lb_get_kernel", "lb_set_wait_ns", "lb_ens_set_wait_ns",
    "lb_ens_set_kernel", "lb_ens_get_kernel", "lb_ens_set_resident", "lb_ens_num_resident",
    "lb_ens_create", "lb_ens_destroy", "lb_ens_init", "lb_ens_sk_config",
    "lb_ens_set_strip_height", "lb_ens_autotune", "lb_ens_step", "lb_ens_sync",
    "lb_ens_get_step", "lb_ens_num_tiles", "lb_ens_populations", "lb_ens_density",
    "lb_ens_conserved", "lb_ens_structure_factor", "lb_sk_moments", "lb_ens_set_launch",
    "lb_ens_get_launch",
    "lb3_create", "lb3_destroy", "lb3_init", "lb3_set_psi", "lb3_set_replica", "lb3_set_strip", "lb3_step",
    "lb3_sync", "lb3_get_step", "lb3_density", "lb3_populations", "lb3_set_populations",
    "lb3_conserved", "lb3_sk_config", "lb3_sk_reset", "lb3_structure_factor_axes",
    "lb3_sk_full", "lb3_structure_factor", "lb3_sk_moments",
    "lb_nn_conv3x3", "lb_nn_conv3x3_wgrad", "lb_nn_relu_mask", "lb_nn_pool2", "lb_nn_up2",
    "lb_nn_add", "lb_nn_coarse_grain", "lb_nn_mse", "lb_nn_residual", "lb_nn_adam",
    "lb_nn_to_bf16", "lb_nn_flux_div", "lb_nn_coarse_momentum", "lb_nn_expand_channel",
    "lb_nn_mse_channel", "lb_nn_mse_blocks", "lb_nn_add_channel", "lb_nn_expand", "lb_nn_wgrad_workspace", "lb_nn_set_conv_path",
    "lb_nn_status", "lb_nn_set_wait_ns",
]


class LbError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {lb_strerror(code)} ({code})")


class lb_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("G", C.c_double), ("tau", C.c_double), ("kT", C.c_double),
        ("psi_kind", C.c_int), ("psi_p1", C.c_double), ("psi_p2", C.c_double),
        ("stencil", C.c_int), ("precision", C.c_int),
        ("stream", C.c_void_p), ("device", C.c_int),
        ("tau_bulk", C.c_double), ("tau_ghost", C.c_double),
    ]


class lb_replica(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("G", C.c_double), ("tau", C.c_double),
                ("kT", C.c_double), ("rho0", C.c_double)]


_lib = None
_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_LL = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def load(path=LIB_PATH):
    """Load liblbsc.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built: call "
                           "paper_2212_07848_gb300.build.build() (no CPU fallback)")
    _lib = bind(C.CDLL(path))
    return _lib


def bind(L):
    """Declare the C signatures of include/lbsc.h on a loaded library."""
    P = C.c_void_p
    sig = {
        "lb_params_init": (C.c_int, [C.POINTER(lb_params)]),
        "lb_create": (C.c_int, [C.POINTER(P), C.c_int, C.c_int, C.c_double, C.c_double,
                                C.c_double, C.c_int, C.c_int]),
        "lb_create_ex": (C.c_int, [C.POINTER(P), C.POINTER(lb_params)]),
        "lb_destroy": (None, [P]),
        "lb_init": (C.c_int, [P, C.c_double, C.c_uint64, C.c_double]),
        "lb_set_replica": (C.c_int, [P, C.c_uint32]),
        "lb_set_strip_height": (C.c_int, [P, C.c_int]),
        "lb_step": (C.c_int, [P, C.c_int]),
        "lb_sync": (C.c_int, [P]),
        "lb_get_step": (C.c_longlong, [P]),
        "lb_set_step": (C.c_int, [P, C.c_longlong]),
        "lb_density": (C.c_int, [P, _D]),
        "lb_populations": (C.c_int, [P, _D]),
        "lb_set_populations": (C.c_int, [P, _D]),
        "lb_set_density": (C.c_int, [P, _D]),
        "lb_upload_state": (C.c_int, [P, P]),
        "lb_download_state": (C.c_int, [P, P]),
        "lb_sk_config": (C.c_int, [P, C.c_int, C.c_longlong]),
        "lb_sk_reset": (C.c_int, [P]),
        "lb_sk_sample_now": (C.c_int, [P]),
        "lb_structure_factor": (C.c_int, [P, _D, C.c_int, C.POINTER(C.c_longlong)]),
        "lb_structure_factor_counts": (C.c_int, [P, _LL, C.c_int]),
        "lb_sk_moments": (C.c_int, [P, _D]),
        "lb_conserved": (C.c_int, [P, _D]),
        "lb_save": (C.c_int, [P, C.c_char_p]),
        "lb_load": (C.c_int, [P, C.c_char_p]),
        "lb_device_ptr": (C.c_void_p, [P, C.c_int]),
        "lb_stream": (C.c_void_p, [P]),
        "lb_strerror": (C.c_char_p, [C.c_int]),
        "lb_conserved_static": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_double, P, P]),
        "lb_set_kernel": (C.c_int, [P, C.c_int]),
        "lb_set_wait_ns": (C.c_int, [P, C.c_longlong]),
        "lb_ens_set_wait_ns": (C.c_int, [P, C.c_longlong]),
        "lb_ens_set_kernel": (C.c_int, [P, C.c_int]),
        "lb_ens_get_kernel": (C.c_int, [P]),
        "lb_ens_set_resident": (C.c_int, [P, C.c_int]),
        "lb_ens_num_resident": (C.c_int, [P]),
        "lb_nn_set_wait_ns": (C.c_int, [C.c_longlong]),
        "lb_get_kernel": (C.c_int, [P]),
        "lb_ens_create": (C.c_int, [C.POINTER(P), C.POINTER(lb_replica), C.c_int, C.c_int,
                                    C.c_double, C.c_double, C.c_int, C.c_uint64, P]),
        "lb_ens_destroy": (None, [P]),
        "lb_ens_init": (C.c_int, [P, C.c_double]),
        "lb_ens_sk_config": (C.c_int, [P, C.c_int, C.c_longlong]),
        "lb_ens_set_strip_height": (C.c_int, [P, C.c_int]),
        "lb_ens_autotune": (C.c_int, [P, C.c_int, C.c_char_p, C.POINTER(C.c_int)]),
        "lb_ens_step": (C.c_int, [P, C.c_int]),
        "lb_ens_set_launch": (C.c_int, [P, C.c_int]),
        "lb3_create": (C.c_int, [C.POINTER(P), C.c_int, C.c_int, C.c_int, C.c_double,
                                 C.c_double, C.c_double, C.c_int, P]),
        "lb3_destroy": (None, [P]),
        "lb3_init": (C.c_int, [P, C.c_double, C.c_uint64, C.c_double]),
        "lb3_set_psi": (C.c_int, [P, C.c_int, C.c_double, C.c_double]),
        "lb3_sk_full": (C.c_int, [P, C.c_int]),
        "lb3_structure_factor": (C.c_int, [P, _D, C.c_int, C.POINTER(C.c_longlong)]),
        "lb3_sk_moments": (C.c_int, [P, _D]),
        "lb3_set_replica": (C.c_int, [P, C.c_uint32]),
        "lb3_set_strip": (C.c_int, [P, C.c_int]),
        "lb3_step": (C.c_int, [P, C.c_int]),
        "lb3_sync": (C.c_int, [P]),
        "lb3_get_step": (C.c_longlong, [P]),
        "lb3_density": (C.c_int, [P, _D]),
        "lb3_populations": (C.c_int, [P, _D]),
        "lb3_set_populations": (C.c_int, [P, _D]),
        "lb3_conserved": (C.c_int, [P, _D]),
        "lb3_sk_config": (C.c_int, [P, C.c_int, C.c_longlong]),
        "lb3_sk_reset": (C.c_int, [P]),
        "lb3_structure_factor_axes": (C.c_int, [P, _D, C.POINTER(C.c_longlong)]),
        "lb_ens_get_launch": (C.c_int, [P]),
        "lb_ens_sync": (C.c_int, [P]),
        "lb_ens_get_step": (C.c_longlong, [P]),
        "lb_ens_num_tiles": (C.c_int, [P]),
        "lb_ens_populations": (C.c_int, [P, C.c_int, _D]),
        "lb_ens_density": (C.c_int, [P, C.c_int, _D]),
        "lb_ens_conserved": (C.c_int, [P, C.c_int, _D]),
        "lb_ens_structure_factor": (C.c_int, [P, C.c_int, _D, C.c_int, C.POINTER(C.c_longlong)]),
        # surrogate building blocks: device pointers, sizes, stream
        "lb_nn_conv3x3": (C.c_int, [P, P, P, P] + [C.c_int] * 7 + [P]),
        "lb_nn_conv3x3_wgrad": (C.c_int, [P, P, P, P] + [C.c_int] * 5 + [P, C.c_size_t, P]),
        "lb_nn_wgrad_workspace": (C.c_size_t, [C.c_int] * 5),
        "lb_nn_flux_div": (C.c_int, [P, P] + [C.c_int] * 5 + [P]),
        "lb_nn_mse_blocks": (C.c_int, [P, C.c_int, P, P] + [C.c_int] * 4 + [C.c_double, P, P, P]),
        "lb_nn_add_channel": (C.c_int, [P, C.c_int, C.c_int, P, C.c_int, C.c_int, C.c_size_t, P]),
        "lb_nn_coarse_momentum": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_double, P, P, P]),
        "lb_nn_expand_channel": (C.c_int, [P, P, P, C.c_int, C.c_int, C.c_size_t, P]),
        "lb_nn_mse_channel": (C.c_int, [P, C.c_int, C.c_int, P, P, C.c_size_t, C.c_double, P, P,
                                        P]),
        "lb_nn_set_conv_path": (C.c_int, [C.c_int]),
        "lb_nn_status": (C.c_int, []),
        "lb_nn_relu_mask": (C.c_int, [P, P, P, C.c_size_t, P]),
        "lb_nn_pool2": (C.c_int, [P, P] + [C.c_int] * 5 + [P]),
        "lb_nn_up2": (C.c_int, [P, P] + [C.c_int] * 5 + [P]),
        "lb_nn_add": (C.c_int, [P, P, P, C.c_size_t, P]),
        "lb_nn_coarse_grain": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_double, P, P]),
        "lb_nn_mse": (C.c_int, [P, C.c_int, P, P, C.c_size_t, P, P, P]),
        "lb_nn_residual": (C.c_int, [P, P, C.c_int, P, C.c_int, C.c_size_t, P, P]),
        "lb_nn_adam": (C.c_int, [P, P, P, P, P, C.c_size_t, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_longlong, P]),
        "lb_nn_to_bf16": (C.c_int, [P, P, C.c_size_t, P]),
        "lb_nn_expand": (C.c_int, [P, P, C.c_double, P, C.c_int, C.c_size_t, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


def _check(rc, where):
    if rc != LB_OK:
        raise LbError(rc, where)


def lb_strerror(code):
    return load().lb_strerror(int(code)).decode()


def lb_params_init():
    p = lb_params()
    _check(load().lb_params_init(C.byref(p)), "lb_params_init")
    return p


def lb_create(nx, ny, G, tau, kT, psi_kind=LB_PSI_EXP, stencil=4):
    h = C.c_void_p()
    _check(load().lb_create(C.byref(h), nx, ny, G, tau, kT, psi_kind, stencil), "lb_create")
    return h


def lb_create_ex(p):
    h = C.c_void_p()
    _check(load().lb_create_ex(C.byref(h), C.byref(p)), "lb_create_ex")
    return h


def lb_destroy(h):
    load().lb_destroy(h)


def lb_init(h, rho0, seed=0, init_amp=0.0):
    _check(load().lb_init(h, rho0, seed, init_amp), "lb_init")


def lb_set_replica(h, replica):
    _check(load().lb_set_replica(h, replica), "lb_set_replica")


def lb_set_strip_height(h, rows):
    _check(load().lb_set_strip_height(h, rows), "lb_set_strip_height")


def lb_set_kernel(h, mode):
    _check(load().lb_set_kernel(h, int(mode)), "lb_set_kernel")


def lb_get_kernel(h):
    return load().lb_get_kernel(h)


def lb_set_wait_ns(h, ns):
    _check(load().lb_set_wait_ns(h, int(ns)), "lb_set_wait_ns")


def lb_step(h, n=1):
    _check(load().lb_step(h, int(n)), "lb_step")


def lb_sync(h):
    _check(load().lb_sync(h), "lb_sync")


def lb_get_step(h):
    return load().lb_get_step(h)


def lb_set_step(h, t):
    _check(load().lb_set_step(h, int(t)), "lb_set_step")


def lb_density(h, out):
    _check(load().lb_density(h, out), "lb_density")
    return out


def lb_populations(h, out):
    _check(load().lb_populations(h, out), "lb_populations")
    return out


def lb_set_populations(h, f):
    _check(load().lb_set_populations(h, np.ascontiguousarray(f, np.float64).ravel()),
           "lb_set_populations")


def lb_set_density(h, rho):
    _check(load().lb_set_density(h, np.ascontiguousarray(rho, np.float64).ravel()),
           "lb_set_density")


def lb_upload_state(h, host_ptr):
    _check(load().lb_upload_state(h, host_ptr), "lb_upload_state")


def lb_download_state(h, host_ptr):
    _check(load().lb_download_state(h, host_ptr), "lb_download_state")


def lb_sk_config(h, every, start):
    _check(load().lb_sk_config(h, int(every), int(start)), "lb_sk_config")


def lb_sk_reset(h):
    _check(load().lb_sk_reset(h), "lb_sk_reset")


def lb_sk_sample_now(h):
    _check(load().lb_sk_sample_now(h), "lb_sk_sample_now")


def lb_structure_factor(h, out, nbins=0):
    n = C.c_longlong()
    _check(load().lb_structure_factor(h, out, int(nbins), C.byref(n)), "lb_structure_factor")
    return out, n.value


def lb_sk_moments(h):
    out = np.zeros(2)
    _check(load().lb_sk_moments(h, out), "lb_sk_moments")
    return out


def lb_structure_factor_counts(h, nbins):
    out = np.zeros(nbins, np.int64)
    _check(load().lb_structure_factor_counts(h, out, int(nbins)), "lb_structure_factor_counts")
    return out


def lb_conserved(h):
    out = np.zeros(3)
    _check(load().lb_conserved(h, out), "lb_conserved")
    return out


def lb_save(h, path):
    _check(load().lb_save(h, os.fsencode(path)), "lb_save")


def lb_load(h, path):
    _check(load().lb_load(h, os.fsencode(path)), "lb_load")


def lb_device_ptr(h, which):
    return load().lb_device_ptr(h, which)


def lb_stream(h):
    return load().lb_stream(h)


def lb_conserved_static(d_df, precision, nx, ny, rho0, d_out3, stream=None):
    """Allocation-free mass/momentum sums of a device population buffer into a
    caller-owned device array of 3 doubles (see include/lbsc.h)."""
    _check(load().lb_conserved_static(d_df, precision, nx, ny, rho0, d_out3, stream),
           "lb_conserved_static")


# ---- batched ensembles -------------------------------------------------------
def lb_ens_create(reps, psi_kind=LB_PSI_EXP, psi_p1=0.0, psi_p2=0.0, stencil=4, seed=0,
                  stream=None):
    """reps: sequence of (nx, ny, G, tau, kT, rho0)."""
    arr = (lb_replica * len(reps))(*[lb_replica(*r) for r in reps])
    h = C.c_void_p()
    _check(load().lb_ens_create(C.byref(h), arr, len(reps), psi_kind, psi_p1, psi_p2, stencil,
                                seed, stream), "lb_ens_create")
    return h


def lb_ens_destroy(h):
    load().lb_ens_destroy(h)


def lb_ens_init(h, init_amp=0.0):
    _check(load().lb_ens_init(h, init_amp), "lb_ens_init")


def lb_ens_sk_config(h, every, start):
    _check(load().lb_ens_sk_config(h, int(every), int(start)), "lb_ens_sk_config")


LB_ENS_PER_STEP, LB_ENS_PERSISTENT = 0, 1
LB_ENS_RESIDENT_OFF, LB_ENS_RESIDENT_ON, LB_ENS_RESIDENT_AUTO = 0, 1, 2


def lb_ens_set_launch(h, mode):
    _check(load().lb_ens_set_launch(h, int(mode)), "lb_ens_set_launch")


def lb_ens_get_launch(h):
    return load().lb_ens_get_launch(h)


def lb_ens_set_kernel(h, mode):
    _check(load().lb_ens_set_kernel(h, int(mode)), "lb_ens_set_kernel")


def lb_ens_get_kernel(h):
    return load().lb_ens_get_kernel(h)


def lb_ens_set_resident(h, mode):
    _check(load().lb_ens_set_resident(h, int(mode)), "lb_ens_set_resident")


def lb_ens_num_resident(h):
    n = load().lb_ens_num_resident(h)
    _check(min(n, 0), "lb_ens_num_resident")
    return n


def lb_ens_set_wait_ns(h, ns):
    _check(load().lb_ens_set_wait_ns(h, int(ns)), "lb_ens_set_wait_ns")


def lb_nn_set_wait_ns(ns):
    _check(load().lb_nn_set_wait_ns(int(ns)), "lb_nn_set_wait_ns")


def lb_ens_set_strip_height(h, rows):
    _check(load().lb_ens_set_strip_height(h, int(rows)), "lb_ens_set_strip_height")


def lb_ens_autotune(h, trial_steps=20, cache_path=None):
    c = C.c_int()
    _check(load().lb_ens_autotune(h, int(trial_steps),
                                  os.fsencode(cache_path) if cache_path else None, C.byref(c)),
           "lb_ens_autotune")
    return c.value


def lb_ens_step(h, n=1):
    _check(load().lb_ens_step(h, int(n)), "lb_ens_step")


def lb_ens_sync(h):
    _check(load().lb_ens_sync(h), "lb_ens_sync")


def lb_ens_get_step(h):
    return load().lb_ens_get_step(h)


def lb_ens_num_tiles(h):
    return load().lb_ens_num_tiles(h)


def lb_ens_populations(h, r, out):
    _check(load().lb_ens_populations(h, int(r), out), "lb_ens_populations")
    return out


def lb_ens_density(h, r, out):
    _check(load().lb_ens_density(h, int(r), out), "lb_ens_density")
    return out


def lb_ens_conserved(h, r):
    out = np.zeros(3)
    _check(load().lb_ens_conserved(h, int(r), out), "lb_ens_conserved")
    return out


def lb_ens_structure_factor(h, r, out, nbins=0):
    n = C.c_longlong()
    _check(load().lb_ens_structure_factor(h, int(r), out, int(nbins), C.byref(n)),
           "lb_ens_structure_factor")
    return out, n.value
