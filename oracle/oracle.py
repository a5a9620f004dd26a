"""ctypes wrapper around the FP64 CPU oracle (lbsc_oracle.c).

TEST INFRASTRUCTURE ONLY.  Callers: the test suite, the package smoke check
and the benchmark's CPU-baseline leg.  No product code imports this module.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("G", C.c_double), ("tau", C.c_double), ("kT", C.c_double),
        ("psi_kind", C.c_int), ("psi_p1", C.c_double), ("psi_p2", C.c_double),
        ("stencil", C.c_int),
        ("rho0", C.c_double),
        ("seed", C.c_uint64),
        ("replica", C.c_uint32),
        ("tau_bulk", C.c_double),
        ("tau_ghost", C.c_double),
        ("force_mrt", C.c_int),
    ]


class Or3Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("G", C.c_double), ("tau", C.c_double), ("kT", C.c_double),
        ("rho0", C.c_double),
        ("seed", C.c_uint64),
        ("replica", C.c_uint32),
        ("psi_kind", C.c_int),
        ("psi_p1", C.c_double), ("psi_p2", C.c_double),
    ]


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_U64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def lib():
    """Load (building if needed) the oracle library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_philox4x32_10.argtypes = [_U32, _U32, _U32]
        L.or_philox4x64_10.argtypes = [_U64, _U64, _U64]
        L.or_psi.argtypes = [C.POINTER(OrParams), C.c_double]
        L.or_psi.restype = C.c_double
        L.or_create.argtypes = [C.POINTER(OrParams)]
        L.or_create.restype = C.c_void_p
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_init.argtypes = [C.c_void_p, C.c_double, C.c_uint64, C.c_double]
        L.or_set_replica.argtypes = [C.c_void_p, C.c_uint32]
        L.or_set_step.argtypes = [C.c_void_p, C.c_longlong]
        L.or_get_step.argtypes = [C.c_void_p]
        L.or_get_step.restype = C.c_longlong
        L.or_set_density.argtypes = [C.c_void_p, _D]
        L.or_set_populations.argtypes = [C.c_void_p, _D]
        L.or_get_populations.argtypes = [C.c_void_p, _D]
        L.or_density.argtypes = [C.c_void_p, _D]
        L.or_conserved.argtypes = [C.c_void_p, _D]
        L.or_force_field.argtypes = [C.c_void_p, _D, _D]
        L.or_sk_config.argtypes = [C.c_void_p, C.c_int, C.c_longlong]
        L.or_sk_reset.argtypes = [C.c_void_p]
        L.or_sk_sample_now.argtypes = [C.c_void_p]
        L.or_sk_get.argtypes = [C.c_void_p, _D]
        L.or_sk_get.restype = C.c_longlong
        L.or_step.argtypes = [C.c_void_p, C.c_int]
        L.or_step.restype = C.c_int
        L.or_step_sites.argtypes = [C.POINTER(OrParams), C.c_longlong, _D, C.c_int,
                                    _I, _I, _D]
        L.or_step_sites.restype = C.c_int
        L.or_lattice_constants.argtypes = [_I, _I, _D, C.POINTER(C.c_double)]
        L.or_moment_basis.argtypes = [_D, _D]
        L.or_stencil.argtypes = [C.c_int, _I, _I, _D]
        L.or_stencil.restype = C.c_int
        L.or_normals.argtypes = [C.POINTER(OrParams), C.c_uint32, C.c_uint32, _D]
        L.or3_create.argtypes = [C.POINTER(Or3Params)]
        L.or3_create.restype = C.c_void_p
        L.or3_destroy.argtypes = [C.c_void_p]
        L.or3_init.argtypes = [C.c_void_p, C.c_double, C.c_uint64, C.c_double]
        L.or3_set_replica.argtypes = [C.c_void_p, C.c_uint32]
        L.or3_get_step.argtypes = [C.c_void_p]
        L.or3_get_step.restype = C.c_longlong
        L.or3_set_populations.argtypes = [C.c_void_p, _D]
        L.or3_get_populations.argtypes = [C.c_void_p, _D]
        L.or3_density.argtypes = [C.c_void_p, _D]
        L.or3_conserved.argtypes = [C.c_void_p, _D]
        L.or3_sk_config.argtypes = [C.c_void_p, C.c_int, C.c_longlong]
        L.or3_sk_get.argtypes = [C.c_void_p, _D]
        L.or3_sk_get.restype = C.c_longlong
        L.or3_sk_full.argtypes = [C.c_void_p, C.c_int]
        L.or3_sk_full.restype = C.c_int
        L.or3_sk_full_get.argtypes = [C.c_void_p, _D]
        L.or3_sk_full_get.restype = C.c_longlong
        L.or3_step.argtypes = [C.c_void_p, C.c_int]
        L.or3_lattice_constants.argtypes = [_I, _D]
        L.or3_force_field.argtypes = [C.c_void_p, _D]
        L.or3_moment_basis.argtypes = [_D, _D]
        L.or3_normals.argtypes = [C.POINTER(Or3Params), C.c_uint32, C.c_uint32, _D]
        L.or3_step_sites.argtypes = [C.POINTER(Or3Params), C.c_longlong, _D, C.c_int, _I, _I, _I,
                                     _D]
        L.or3_step_sites.restype = C.c_int
        L.or3_ring_pair22.argtypes = [C.c_uint32, _D]
        L.or_box_muller_ring.argtypes = [C.c_uint32, C.c_uint32, _D]
        L.or_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def threads():
    """Host threads the oracle's site loops use."""
    return int(lib().or_threads())


def set_threads(n):
    """Threads for the oracle's site loops (for timing on one core)."""
    lib().or_set_threads(int(n))


def philox4x32(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def philox4x64(ctr, key):
    out = np.zeros(4, np.uint64)
    lib().or_philox4x64_10(np.asarray(ctr, np.uint64), np.asarray(key, np.uint64), out)
    return out


def lattice_constants():
    cx = np.zeros(9, np.int32); cy = np.zeros(9, np.int32); w = np.zeros(9)
    cs2 = C.c_double()
    lib().or_lattice_constants(cx, cy, w, C.byref(cs2))
    return cx, cy, w, cs2.value


def moment_basis():
    m = np.zeros(81); b = np.zeros(9)
    lib().or_moment_basis(m, b)
    return m.reshape(9, 9), b


def stencil(order):
    ex = np.zeros(32, np.int32); ey = np.zeros(32, np.int32); w = np.zeros(32)
    n = lib().or_stencil(order, ex, ey, w)
    return ex[:n].copy(), ey[:n].copy(), w[:n].copy()


def make_params(nx, ny, G, tau, kT, psi_kind=0, psi_p1=0.0, psi_p2=0.0, stencil=4,
                rho0=0.0, seed=0, replica=0, tau_bulk=0.0, tau_ghost=0.0, force_mrt=0):
    return OrParams(nx, ny, G, tau, kT, psi_kind, psi_p1, psi_p2, stencil, rho0,
                    seed, replica, tau_bulk, tau_ghost, force_mrt)


class OracleLattice:
    """One periodic nx x ny lattice held by the FP64 oracle."""

    def __init__(self, nx, ny, G, tau, kT, psi_kind=0, stencil=4, psi_p1=0.0,
                 psi_p2=0.0, replica=0, tau_bulk=0.0, tau_ghost=0.0, force_mrt=0):
        self.p = make_params(nx, ny, G, tau, kT, psi_kind, psi_p1, psi_p2, stencil,
                             replica=replica, tau_bulk=tau_bulk, tau_ghost=tau_ghost,
                             force_mrt=force_mrt)
        self.nx, self.ny = nx, ny
        self._h = lib().or_create(C.byref(self.p))
        if not self._h:
            raise ValueError("oracle: invalid parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def init(self, rho0, seed=0, init_amp=0.0):
        self.p.rho0 = rho0
        self.p.seed = seed
        lib().or_init(self._h, rho0, seed, init_amp)

    def set_step(self, t):
        lib().or_set_step(self._h, t)

    @property
    def t(self):
        return lib().or_get_step(self._h)

    def set_density(self, rho):
        lib().or_set_density(self._h, np.ascontiguousarray(rho, np.float64).ravel())

    def set_populations(self, f):
        lib().or_set_populations(self._h, np.ascontiguousarray(f, np.float64).ravel())

    def populations(self):
        f = np.zeros(9 * self.nx * self.ny)
        lib().or_get_populations(self._h, f)
        return f.reshape(9, self.ny, self.nx)

    def density(self):
        r = np.zeros(self.nx * self.ny)
        lib().or_density(self._h, r)
        return r.reshape(self.ny, self.nx)

    def conserved(self):
        out = np.zeros(3)
        lib().or_conserved(self._h, out)
        return out

    def force(self):
        fx = np.zeros(self.nx * self.ny); fy = np.zeros(self.nx * self.ny)
        lib().or_force_field(self._h, fx, fy)
        return fx.reshape(self.ny, self.nx), fy.reshape(self.ny, self.nx)

    def step(self, n=1):
        lib().or_step(self._h, int(n))

    def sk_config(self, every, start):
        lib().or_sk_config(self._h, int(every), int(start))

    def sk_reset(self):
        lib().or_sk_reset(self._h)

    def sk_sample_now(self):
        lib().or_sk_sample_now(self._h)

    def structure_factor(self):
        """Mean S(k) over the samples on the half plane [ny][nx/2+1]."""
        out = np.zeros((self.nx // 2 + 1) * self.ny)
        n = lib().or_sk_get(self._h, out)
        return out.reshape(self.ny, self.nx // 2 + 1), n


def step_sites(params, t, f_full, xs, ys):
    """One oracle step evaluated at the sites (xs[i], ys[i]) of a full-lattice
    input state f_full ([9][ny][nx], full populations). Returns [n][9]."""
    xs = np.ascontiguousarray(xs, np.int32)
    ys = np.ascontiguousarray(ys, np.int32)
    out = np.zeros(9 * len(xs))
    rc = lib().or_step_sites(C.byref(params), int(t),
                             np.ascontiguousarray(f_full, np.float64).ravel(),
                             len(xs), xs, ys, out)
    if rc != 0:
        raise ValueError("oracle: site out of range")
    return out.reshape(len(xs), 9)


def normals(params, site, t):
    """The six thermal normals of a site and step (modes 3..8)."""
    z = np.zeros(6)
    lib().or_normals(C.byref(params), site, t, z)
    return z


def box_muller_ring(radius_word, angle_index):
    """One Box-Muller pair with the angle taken from a ring of 1024 values."""
    z = np.zeros(2)
    lib().or_box_muller_ring(radius_word, angle_index, z)
    return z


# ---------------------------------------------------------------------------
# D3Q19 (the paper's three-dimensional setting)
# ---------------------------------------------------------------------------
def lattice3_constants():
    """(c [19][3], w [19]) of the D3Q19 lattice in the oracle's order."""
    c = np.zeros(57, np.int32)
    w = np.zeros(19)
    lib().or3_lattice_constants(c, w)
    return c.reshape(19, 3), w


def moment_basis3():
    """(M [19 moments][19 velocities], b [19]) of the D3Q19 basis."""
    m = np.zeros(361)
    b = np.zeros(19)
    lib().or3_moment_basis(m, b)
    return m.reshape(19, 19), b


def normals3(nx, ny, nz, seed, replica, site, t):
    """The 15 thermal normals (modes 4..18) of a site and step."""
    p = Or3Params(nx, ny, nz, 0.0, 1.0, 0.0, 0.0, seed, replica, 0, 0.0, 0.0)
    z = np.zeros(15)
    lib().or3_normals(C.byref(p), site, t, z)
    return z


def step_sites3(nx, ny, nz, G, tau, kT, seed, t, f_full, xs, ys, zs, replica=0, psi_kind=0,
                psi_p1=0.0, psi_p2=0.0):
    """One oracle D3Q19 step evaluated at the sites (xs[i], ys[i], zs[i]) of a
    full-lattice input state f_full ([19][nz][ny][nx], full populations) at
    step t.  Returns [n][19]."""
    p = Or3Params(nx, ny, nz, G, tau, kT, 0.0, seed, replica, psi_kind, psi_p1, psi_p2)
    xs, ys, zs = (np.ascontiguousarray(a, np.int32) for a in (xs, ys, zs))
    out = np.zeros(19 * len(xs))
    rc = lib().or3_step_sites(C.byref(p), int(t), np.ascontiguousarray(f_full, np.float64).ravel(),
                              len(xs), xs, ys, zs, out)
    if rc != 0:
        raise ValueError("oracle: site out of range")
    return out.reshape(len(xs), 19)


def ring_pair22(word):
    """The 3D noise pair of one Philox word: radius from its high 22 bits,
    angle index from its low 10 bits."""
    z = np.zeros(2)
    lib().or3_ring_pair22(int(word), z)
    return z


class OracleLattice3:
    """One periodic nx x ny x nz D3Q19 lattice held by the FP64 oracle
    (psi of kind 0, 1 or 2 as in 2D, E4 force stencil, BGK + Guo, 15 noise
    modes)."""

    def __init__(self, nx, ny, nz, G, tau, kT, replica=0, psi_kind=0, psi_p1=0.0, psi_p2=0.0):
        self.p = Or3Params(nx, ny, nz, G, tau, kT, 0.0, 0, replica, psi_kind, psi_p1, psi_p2)
        self.nx, self.ny, self.nz = nx, ny, nz
        self._h = lib().or3_create(C.byref(self.p))
        if not self._h:
            raise ValueError("oracle: invalid parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or3_destroy(h)
            self._h = None

    def init(self, rho0, seed=0, init_amp=0.0):
        self.p.rho0, self.p.seed = rho0, seed
        lib().or3_init(self._h, rho0, seed, init_amp)

    def set_replica(self, r):
        lib().or3_set_replica(self._h, r)

    @property
    def t(self):
        return lib().or3_get_step(self._h)

    def set_populations(self, f):
        lib().or3_set_populations(self._h, np.ascontiguousarray(f, np.float64).ravel())

    def populations(self):
        f = np.zeros(19 * self.nx * self.ny * self.nz)
        lib().or3_get_populations(self._h, f)
        return f.reshape(19, self.nz, self.ny, self.nx)

    def density(self):
        r = np.zeros(self.nx * self.ny * self.nz)
        lib().or3_density(self._h, r)
        return r.reshape(self.nz, self.ny, self.nx)

    def conserved(self):
        out = np.zeros(4)
        lib().or3_conserved(self._h, out)
        return out

    def step(self, n=1):
        lib().or3_step(self._h, int(n))

    def force(self):
        F = np.zeros(3 * self.nx * self.ny * self.nz)
        lib().or3_force_field(self._h, F)
        return F.reshape(3, self.nz, self.ny, self.nx)

    def sk_config(self, every, start):
        lib().or3_sk_config(self._h, int(every), int(start))

    def structure_factor_axes(self):
        """(S [nx/2 + ny/2 + nz/2] on the x, y and z axes, nsamples)."""
        out = np.zeros(self.nx // 2 + self.ny // 2 + self.nz // 2)
        n = lib().or3_sk_get(self._h, out)
        return out, n

    def sk_full(self, enable=True):
        """Accumulate S(k) on every wave vector on the sampling steps."""
        if lib().or3_sk_full(self._h, 1 if enable else 0) != 0:
            raise MemoryError("oracle: full S(k)")

    def structure_factor_full(self):
        """(mean S(k) [nz][ny][nx] over every wave vector, nsamples)."""
        out = np.zeros(self.nx * self.ny * self.nz)
        n = lib().or3_sk_full_get(self._h, out)
        return out.reshape(self.nz, self.ny, self.nx), n


def radial_bins3(S):
    """Radial means of a full S(k) cube [nz][ny][nx]: shell b holds the modes
    with round(|q|) = b, q_a = m_a max(n) / n_a (m_a the folded index on axis
    a); k = 0 excluded; empty shells 0.  Returns an array over b = 0 .. the
    largest shell."""
    nz, ny, nx = S.shape
    Lm = max(nx, ny, nz)
    fold = lambda n: np.where(np.arange(n) <= n // 2, np.arange(n), np.arange(n) - n)
    qz, qy, qx = np.meshgrid(fold(nz) * (Lm / nz), fold(ny) * (Lm / ny), fold(nx) * (Lm / nx),
                             indexing="ij")
    b = np.rint(np.sqrt(qx ** 2 + qy ** 2 + qz ** 2)).astype(int)
    keep = b > 0
    keep[0, 0, 0] = False
    sums = np.bincount(b[keep], S[keep])
    cnt = np.bincount(b[keep])
    return np.where(cnt > 0, sums / np.maximum(cnt, 1), 0.0)


def full_plane(S_half, nx, ny):
    """The full spectrum [ny][nx] of a real field's S(k), rebuilt from its half
    plane [ny][nx/2+1] by S(-k) = S(k) (the density is real, so
    |dn(-k)|^2 = |dn(k)|^2)."""
    S_half = np.asarray(S_half, dtype=np.float64)
    full = np.zeros((ny, nx))
    for my in range(ny):
        for mx in range(nx):
            if mx <= nx // 2:
                full[my, mx] = S_half[my, mx]
            else:
                full[my, mx] = S_half[(-my) % ny, nx - mx]
    return full


def _folded(m, n):
    return m if m <= n // 2 else m - n


def radial_bins(S_half, nx, ny, nbins):
    """Radial read-out of a 2D S(k) (defined after Eq. (12)), binned as the
    paper bins its S(k) curves against |k| (Fig. 2): every wave vector of the
    full plane except k = 0, with q = (m_x max(n)/n_x, m_y max(n)/n_y) from
    the folded indices m, falls in bin b = round(|q|) (bin width
    dk = 2 pi / max(n_x, n_y)); bins at or above nbins are dropped.  Returns
    (mean of S over each bin, NaN where empty; number of modes per bin)."""
    full = full_plane(S_half, nx, ny)
    Lm = max(nx, ny)
    sums = np.zeros(nbins)
    counts = np.zeros(nbins, dtype=np.int64)
    for my in range(ny):
        for mx in range(nx):
            if mx == 0 and my == 0:
                continue
            qx = _folded(mx, nx) * (Lm / nx)
            qy = _folded(my, ny) * (Lm / ny)
            b = int(np.rint(np.sqrt(qx * qx + qy * qy)))
            if b < nbins:
                sums[b] += full[my, mx]
                counts[b] += 1
    with np.errstate(invalid="ignore", divide="ignore"):
        means = np.where(counts > 0, sums / np.maximum(counts, 1), np.nan)
    return means, counts


def sk_first_moments(S_half, nx, ny):
    """(sum_k S(k), sum_k |k| S(k)) over every wave vector of the full plane
    except k = 0, |k| = 2 pi sqrt((m_x/n_x)^2 + (m_y/n_y)^2) with folded
    indices.  Their ratio gives the domain size L = 2 pi sum S / sum |k| S
    (the library's definition of L(t); the paper defines none)."""
    full = full_plane(S_half, nx, ny)
    s0 = s1 = 0.0
    for my in range(ny):
        for mx in range(nx):
            if mx == 0 and my == 0:
                continue
            k = 2.0 * np.pi * np.hypot(_folded(mx, nx) / nx, _folded(my, ny) / ny)
            s0 += full[my, mx]
            s1 += k * full[my, mx]
    return s0, s1
