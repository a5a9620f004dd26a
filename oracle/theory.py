"""Closed forms of arXiv:2212.07848 used to pin the oracle (FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY (imported by the test suite and the benchmark's
CPU-baseline leg, never by the product path).

Convention (a reading of the paper, stated once here): the force is
F = -G c_s^2 psi(x) sum_a w_a psi(x+e_a) e_a with sum_a w_a e_ax^2 = 1, so the
bulk pressure is p = rho c_s^2 + (G c_s^2 / 2) psi^2 with c_s^2 = 1/3 and
G < 0 attractive.  It is the paper's Eq. (2), p = n T - (G_p / 2) psi_p^2,
with T = c_s^2 and G_p psi_p^2 = -G c_s^2 psi^2.
"""
from fractions import Fraction
from itertools import product

import numpy as np
from scipy.optimize import brentq

CS2 = 1.0 / 3.0


# --------------------------------------------------------------------------
# Pseudopotentials: kind 0 = 1 - exp(-rho); kind 1 = sqrt(Tc nc) exp(1 - nc/rho)
# (Eq. (5)); kind 2 = a exp(-b/rho) (the form introduced before Eq. (3)).
# --------------------------------------------------------------------------
def psi(rho, kind=0, p1=0.0, p2=0.0):
    rho = np.asarray(rho, dtype=np.float64)
    if kind == 0:
        return 1.0 - np.exp(-rho)
    if kind == 1:
        return np.sqrt(p1 * p2) * np.exp(1.0 - p2 / rho)
    if kind == 2:
        return p1 * np.exp(-p2 / rho)
    raise ValueError(kind)


def dpsi(rho, kind=0, p1=0.0, p2=0.0):
    rho = np.asarray(rho, dtype=np.float64)
    if kind == 0:
        return np.exp(-rho)
    if kind in (1, 2):
        b = p2
        return psi(rho, kind, p1, p2) * b / rho ** 2
    raise ValueError(kind)


def d2psi(rho, kind=0, p1=0.0, p2=0.0):
    rho = np.asarray(rho, dtype=np.float64)
    if kind == 0:
        return -np.exp(-rho)
    b = p2
    return psi(rho, kind, p1, p2) * (b * b / rho ** 4 - 2.0 * b / rho ** 3)


# --------------------------------------------------------------------------
# Equation of state, Eq. (2), and its derivatives.
# --------------------------------------------------------------------------
def pressure(rho, G, kind=0, p1=0.0, p2=0.0):
    return rho * CS2 + 0.5 * G * CS2 * psi(rho, kind, p1, p2) ** 2


def dpressure(rho, G, kind=0, p1=0.0, p2=0.0):
    """dp/drho = c_s^2 (1 + G psi psi'): the squared bulk sound speed c_s0^2."""
    return CS2 * (1.0 + G * psi(rho, kind, p1, p2) * dpsi(rho, kind, p1, p2))


def d2pressure(rho, G, kind=0, p1=0.0, p2=0.0):
    return CS2 * G * (dpsi(rho, kind, p1, p2) ** 2 + psi(rho, kind, p1, p2) * d2psi(rho, kind, p1, p2))


def critical_point_kind0():
    """Critical point of p(rho) for psi = 1 - exp(-rho): d(psi psi')/drho = 0
    fixes rho_c, then 1 + G psi psi' = 0 fixes G_c (the conditions stated
    before Eq. (4))."""
    f = lambda r: np.exp(-r) * (2.0 * np.exp(-r) - 1.0)   # d(psi psi')/drho
    rc = brentq(f, 0.1, 3.0, xtol=1e-15)
    Gc = -1.0 / (psi(rc) * dpsi(rc))
    return rc, Gc


def reduced_temperature(G, kind=0):
    """T_hat = T / T_c at fixed c_s^2: T_hat = G_c / G for kind 0."""
    _, Gc = critical_point_kind0()
    return Gc / G


def spinodal(G, kind=0, p1=0.0, p2=0.0, lo=1e-3, hi=10.0):
    """Both roots of dp/drho = 0 (gas and liquid spinodal densities)."""
    grid = np.linspace(lo, hi, 20001)
    d = dpressure(grid, G, kind, p1, p2)
    roots = []
    for a, b, da, db in zip(grid[:-1], grid[1:], d[:-1], d[1:]):
        if da == 0.0:
            roots.append(a)
        elif da * db < 0:
            roots.append(brentq(lambda r: dpressure(r, G, kind, p1, p2), a, b, xtol=1e-15))
    return roots


def kappa_T_reduced(nhat, That):
    """Isothermal compressibility of the reduced EoS, Eq. (8)."""
    return 0.5 * nhat / (nhat ** 2 * That - np.exp(2.0 - 2.0 / nhat))


def p_reduced(nhat, That):
    """General EoS in reduced variables, Eq. (7)."""
    return 2.0 * nhat * That - np.exp(2.0 - 2.0 / nhat)


def coexistence(G, eps=0.0, kind=0, p1=0.0, p2=0.0):
    """Bulk densities (rho_g, rho_l) that satisfy p(rho_g) = p(rho_l) = p0 and
    int_{rho_g}^{rho_l} (p0 - p) psi' / psi^{1+eps} drho = 0.  eps is left
    to the caller: the paper states no rule (its mechanical-equilibrium
    argument is the flat-interface constancy of Eq. (14))."""
    from scipy.integrate import quad
    from scipy.optimize import fsolve
    sp = spinodal(G, kind, p1, p2)
    if len(sp) < 2:
        raise ValueError("supercritical: no coexistence")
    rs_g, rs_l = sp[0], sp[-1]
    P = lambda r: pressure(r, G, kind, p1, p2)

    def residual(v):
        rg, rl = v
        p0 = P(rg)
        integ = quad(lambda r: (p0 - P(r)) * dpsi(r, kind, p1, p2) / psi(r, kind, p1, p2) ** (1 + eps),
                     rg, rl, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
        return [P(rl) - p0, integ]

    rg, rl = fsolve(residual, [0.5 * rs_g, 1.3 * rs_l], xtol=1e-12)
    return rg, rl


# --------------------------------------------------------------------------
# Force-stencil weights derived from the isotropy conditions (Eq. (1): the
# weights "carefully chosen" for isotropy).  Solved exactly with Fractions.
# --------------------------------------------------------------------------
_SHELLS = {4: [1, 2], 6: [1, 2, 4], 8: [1, 2, 4, 5, 8]}


def _shell_vectors(e2):
    return [(x, y) for x, y in product(range(-3, 4), repeat=2) if x * x + y * y == e2]


def _moment(e2, px, py):
    return sum(Fraction(x) ** px * Fraction(y) ** py for x, y in _shell_vectors(e2))


def isotropic_weights(order):
    """Solve for w(|e|^2) on the shells of an E<order> stencil so that
    sum_a w_a e_ax^2 = 1 and the tensors sum_a w_a e^(2n) are isotropic for
    2n = 4, ..., order.  Isotropy in 2D: sum w ex^(2n-2m) ey^(2m) is
    proportional to (2n-2m-1)!! (2m-1)!!."""
    shells = _SHELLS[order]
    rows, rhs = [], []
    rows.append([_moment(s, 2, 0) for s in shells]); rhs.append(Fraction(1))
    dfact = lambda n: 1 if n <= 0 else n * dfact(n - 2)
    for n in range(2, order // 2 + 1):
        # ratios against the pure-x moment of the same order
        for m in range(1, n // 2 + 1):
            a = dfact(2 * n - 2 * m - 1) * dfact(2 * m - 1)
            b = dfact(2 * n - 1)
            # b * M(2n-2m, 2m) - a * M(2n, 0) = 0
            rows.append([b * _moment(s, 2 * n - 2 * m, 2 * m) - a * _moment(s, 2 * n, 0)
                         for s in shells])
            rhs.append(Fraction(0))
    # exact Gaussian elimination over the rationals
    A = [r[:] + [v] for r, v in zip(rows, rhs)]
    nrow, ncol = len(A), len(shells)
    piv_row = 0
    for col in range(ncol):
        p = next((r for r in range(piv_row, nrow) if A[r][col] != 0), None)
        if p is None:
            continue
        A[piv_row], A[p] = A[p], A[piv_row]
        pv = A[piv_row][col]
        A[piv_row] = [v / pv for v in A[piv_row]]
        for r in range(nrow):
            if r != piv_row and A[r][col] != 0:
                fac = A[r][col]
                A[r] = [a - fac * b for a, b in zip(A[r], A[piv_row])]
        piv_row += 1
    if piv_row != ncol:
        raise ValueError("isotropy system is singular")
    for r in range(ncol, nrow):
        if A[r][-1] != 0:
            raise ValueError("isotropy system is inconsistent")
    return {s: A[i][-1] for i, s in enumerate(shells)}


def stencil_vectors(order):
    """(ex, ey, w) of the E<order> stencil, weights from isotropic_weights."""
    w = isotropic_weights(order)
    out = []
    for s, ws in w.items():
        for x, y in _shell_vectors(s):
            out.append((x, y, float(ws)))
    return out


# --------------------------------------------------------------------------
# Static structure factor.  Eq. (15)-(16) in the paper's convention, and the
# same on lattice axes in this library's convention for any stencil.
# --------------------------------------------------------------------------
def sk_exact_paper(k, n0, T, psi0, dpsi0, kT):
    """Eq. (16) verbatim (paper convention: c_s0^2 = dp/dn with p of Eq. (2),
    G absorbed into psi): S(k) = n0 kT / {c_s0^2 - (1/2) psi0 psi0' [cos k - 1]}."""
    cs0 = T - psi0 * dpsi0           # dp/dn of p = n T - psi^2 / 2
    return n0 * kT / (cs0 - 0.5 * psi0 * dpsi0 * (np.cos(k) - 1.0))


def force_symbol_axis(k, order=4):
    """s(k) = sum_a w_a sin(k e_ax) e_ax of the stencil, for k along x."""
    k = np.asarray(k, dtype=np.float64)
    return sum(w * np.sin(k * ex) * ex for ex, ey, w in stencil_vectors(order))


def sk_axis(k, rho0, G, kT, order=4, kind=0, p1=0.0, p2=0.0):
    """S(k) for a wave vector along a lattice axis:
        S = rho0 kT / (c_s^2 [1 + G psi0 psi0' s(k) / (2 tan(k/2))]).
    For E4, s(k) = sin k and s/(2 tan(k/2)) = (1 + cos k)/2, which is Eq. (16)
    mapped to this library's convention.  For E6/E8 this is the reading used
    for the longer-range one-dimensional projection."""
    k = np.asarray(k, dtype=np.float64)
    pp = psi(rho0, kind, p1, p2) * dpsi(rho0, kind, p1, p2)
    s = force_symbol_axis(k, order)
    return rho0 * kT / (CS2 * (1.0 + G * pp * s / (2.0 * np.tan(k / 2.0))))


def pn_lattice(rho_line, G, kind=0, p1=0.0, p2=0.0):
    """Normal pressure across a flat interface, Eq. (14), in this library's
    convention (nearest-neighbour 1D projection of E4):
        P_N(x) = rho c_s^2 + (G c_s^2 / 4) psi(x) [psi(x+1) + psi(x-1)]."""
    ps = psi(rho_line, kind, p1, p2)
    return rho_line * CS2 + 0.25 * G * CS2 * ps * (np.roll(ps, -1) + np.roll(ps, 1))
