"""FP64 CPU oracle for the stochastic-heating method (Porter & Vladimirov, HEATCODE).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The CUDA library never
loads it and shares no code with it.

The arithmetic lives in ``heat_oracle.c`` (plain C, FP64); this module only
marshals numpy arrays through ctypes.  Functions and the passages they follow:

* ``range_integral``      -- log-log interpolant of Omega (Eq. interpolation) integrated in closed form
* ``heating_matrix``      -- T_ul for u > l (Eq. heating, wavelength-integral form, plus intra-bin term)
* ``heating_matrix_point`` -- T_ul by the paper's point rule (Eq. heating at lambda_ul, Eq. interpolation)
* ``b_matrix``            -- B_fj suffix sums (Eq. bmatrix via Eq. brecurrence)
* ``recursion``           -- X recursion and renormalisation (Eq. xf, Eq. renormalization)
* ``cooling``, ``emitted_power`` -- T_{f-1,f} (Eq. cooling)
* ``emissivity``          -- j_lambda (Eq. emission, Eq. emission-lambda)
* ``ledger``              -- absorbed vs emitted power of the discrete model (follows from Eq. bequation)
* ``cooling_discrete``    -- thermal-discrete downward rates T_lu (the approximation named beside Eq. adjacent;
                             read as Eq. cooling's integrand restricted to each downward photon-energy window)
* ``solve_full``          -- stationary P of the full rate matrix (Eq. steady-state, Eq. level-sum) by state
                             reduction (Grassmann-Taksar-Heyman), for any downward rates
* ``solve_batch_discrete`` -- cells x grains with thermal-discrete cooling
* ``solve_batch``         -- all of the above over cells x grains (either heating form)
* ``size_integrate``      -- Eq. convolution, discretised
"""
from __future__ import annotations

import ctypes

import numpy as np

from .build import build_oracle

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)

OK, EINVAL, ENOMEM, ENUMERIC = 0, 1, 2, 4


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = ctypes.CDLL(path)
        L.orc_planck_lambda.restype = ctypes.c_double
        L.orc_planck_lambda.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_omega_at.restype = ctypes.c_double
        L.orc_omega_at.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double]
        L.orc_range_integral.restype = ctypes.c_double
        L.orc_range_integral.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_heating_matrix.restype = ctypes.c_int
        L.orc_heating_matrix.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int, _D, _D]
        L.orc_b_matrix.restype = None
        L.orc_b_matrix.argtypes = [ctypes.c_int, _D, _D]
        L.orc_recursion.restype = ctypes.c_int
        L.orc_recursion.argtypes = [ctypes.c_int, _D, _D, _D]
        L.orc_emitted_power.restype = ctypes.c_double
        L.orc_emitted_power.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double]
        L.orc_cooling.restype = ctypes.c_int
        L.orc_cooling.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, _D]
        L.orc_emissivity.restype = None
        L.orc_emissivity.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, _D, _D]
        L.orc_ledger.restype = None
        L.orc_ledger.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D]
        L.orc_solve_spectrum.restype = ctypes.c_int
        L.orc_solve_spectrum.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, _D, _D, _D, _D, _D,
                                         ctypes.c_int]
        L.orc_solve_batch.restype = ctypes.c_int
        L.orc_solve_batch.argtypes = [ctypes.c_int, _D, ctypes.c_int, _D, _I, _D, _D, _D, ctypes.c_int, _D, _D,
                                      _D, _D, ctypes.c_int, ctypes.c_int]
        L.orc_heating_matrix_point.restype = ctypes.c_int
        L.orc_heating_matrix_point.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int, _D, _D]
        L.orc_size_integrate.restype = None
        L.orc_size_integrate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D]
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_emitted_power_window.restype = ctypes.c_double
        L.orc_emitted_power_window.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_cooling_discrete.restype = ctypes.c_int
        L.orc_cooling_discrete.argtypes = [ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, _D]
        L.orc_solve_full.restype = ctypes.c_int
        L.orc_solve_full.argtypes = [ctypes.c_int, _D, _D, _D]
        L.orc_ledger_full.restype = None
        L.orc_ledger_full.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D]
        L.orc_solve_batch_discrete.restype = ctypes.c_int
        L.orc_solve_batch_discrete.argtypes = [ctypes.c_int, _D, ctypes.c_int, _D, _I, _D, _D, _D, ctypes.c_int, _D,
                                               _D, _D, _D, ctypes.c_int]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _dnull(a):
    if a is None:
        return None, None
    return a, a.ctypes.data_as(_D)


def planck_lambda(lam, T):
    return lib().orc_planck_lambda(float(lam), float(T))


def omega_at(lam, om, x):
    lam, pl = _d(lam)
    om, po = _d(om)
    return lib().orc_omega_at(lam.size, pl, po, float(x))


def range_integral(lam, om, p, a, b):
    lam, pl = _d(lam)
    om, po = _d(om)
    return lib().orc_range_integral(lam.size, pl, po, int(p), float(a), float(b))


def heating_matrix_point(lam, om, E):
    """Explicit T of the paper's point rule (Eq. heating)."""
    lam, pl = _d(lam)
    om, po = _d(om)
    E, pe = _d(E)
    nb = E.size
    A = np.zeros((nb, nb))
    st = lib().orc_heating_matrix_point(lam.size, pl, po, nb, pe, A.ctypes.data_as(_D))
    if st != OK:
        raise RuntimeError(f"orc_heating_matrix_point status {st}")
    return A


def heating_matrix(lam, om, E):
    lam, pl = _d(lam)
    om, po = _d(om)
    E, pe = _d(E)
    nb = E.size
    A = np.zeros((nb, nb))
    st = lib().orc_heating_matrix(lam.size, pl, po, nb, pe, A.ctypes.data_as(_D))
    if st != OK:
        raise RuntimeError(f"orc_heating_matrix status {st}")
    return A


def b_matrix(A):
    A, pa = _d(A)
    nb = A.shape[0]
    B = np.zeros((nb, nb))
    lib().orc_b_matrix(nb, pa, B.ctypes.data_as(_D))
    return B


def recursion(B, Cf, return_status=False):
    B, pb = _d(B)
    Cf, pc = _d(Cf)
    nb = B.shape[0]
    P = np.zeros(nb)
    st = lib().orc_recursion(nb, pb, pc, P.ctypes.data_as(_D))
    if return_status:
        return P, st
    if st != OK:
        raise RuntimeError(f"orc_recursion status {st}")
    return P


def emitted_power(lam, cabs, T, Emax):
    lam, pl = _d(lam)
    cabs, pc = _d(cabs)
    return lib().orc_emitted_power(lam.size, pl, pc, float(T), float(Emax))


def cooling(lam, cabs, T, E):
    lam, pl = _d(lam)
    cabs, pc = _d(cabs)
    T, pt = _d(T)
    E, pe = _d(E)
    Cf = np.zeros(E.size)
    st = lib().orc_cooling(lam.size, pl, pc, E.size, pt, pe, Cf.ctypes.data_as(_D))
    if st != OK:
        raise RuntimeError(f"orc_cooling status {st}")
    return Cf


def emissivity(lam, cabs, T, E, P):
    lam, pl = _d(lam)
    cabs, pc = _d(cabs)
    T, pt = _d(T)
    E, pe = _d(E)
    P, pp = _d(P)
    j = np.zeros(lam.size)
    lib().orc_emissivity(lam.size, pl, pc, E.size, pt, pe, pp, j.ctypes.data_as(_D))
    return j


def ledger(A, E, Cf, P):
    A, pa = _d(A)
    E, pe = _d(E)
    Cf, pc = _d(Cf)
    P, pp = _d(P)
    out = np.zeros(2)
    lib().orc_ledger(E.size, pa, pe, pc, pp, out.ctypes.data_as(_D))
    return out


def grain_cooling(wl):
    """Cooling rates for every grain of a workload, concatenated like wl.T."""
    Cf = np.zeros(wl.total_bins)
    for g in range(wl.n_grains):
        s = wl.grain_slice(g)
        Cf[s] = cooling(wl.lam, wl.cabs[g], wl.T[s], wl.E[s])
    return Cf


HEATING_INTEGRAL, HEATING_POINT = 0, 1


def solve_batch(wl, Cf=None, want_j=True, want_ledger=False, n_threads=0, u=None, heating=HEATING_INTEGRAL):
    """P [cells, total_bins], j [cells, G, N] (or None), ledger [cells, G, 2] (or None).
    heating: HEATING_INTEGRAL (elements integrated over the bin edges) or HEATING_POINT
    (the paper's point rule, Eq. heating)."""
    if Cf is None:
        Cf = grain_cooling(wl)
    u = wl.u if u is None else u
    lam, pl = _d(wl.lam)
    cabs, pc = _d(wl.cabs)
    off = np.ascontiguousarray(wl.bin_off, dtype=np.int32)
    T, pt = _d(wl.T)
    E, pe = _d(wl.E)
    Cf, pcf = _d(Cf)
    u, pu = _d(u)
    cells = u.shape[0]
    G, N = wl.n_grains, wl.n_lambda
    P = np.zeros((cells, wl.total_bins))
    j, pj = _dnull(np.zeros((cells, G, N)) if want_j else None)
    led, pld = _dnull(np.zeros((cells, G, 2)) if want_ledger else None)
    st = lib().orc_solve_batch(N, pl, G, pc, off.ctypes.data_as(_I), pt, pe, pcf, cells, pu,
                               P.ctypes.data_as(_D), pj, pld, int(n_threads), int(heating))
    return P, j, led, st


def size_integrate(w, j):
    w, pw = _d(w)
    j, pj = _d(j)
    cells, G, N = j.shape
    J = np.zeros((cells, N))
    lib().orc_size_integrate(cells, G, N, pw, pj, J.ctypes.data_as(_D))
    return J


def max_threads():
    return lib().orc_max_threads()


def emitted_power_window(lam, cabs, T, Emin, Emax):
    lam, pl = _d(lam)
    cabs, pc = _d(cabs)
    return lib().orc_emitted_power_window(lam.size, pl, pc, float(T), float(Emin), float(Emax))


def cooling_discrete(lam, cabs, T, E):
    """Thermal-discrete downward rates D[l, u] = T_lu (l < u), one grain."""
    lam, pl = _d(lam)
    cabs, pc = _d(cabs)
    T, pt = _d(T)
    E, pe = _d(E)
    D = np.zeros((E.size, E.size))
    st = lib().orc_cooling_discrete(lam.size, pl, pc, E.size, pt, pe, D.ctypes.data_as(_D))
    if st != OK:
        raise RuntimeError(f"orc_cooling_discrete status {st}")
    return D


def solve_full(A, D, return_status=False):
    """Stationary P of the full rate matrix: upward A[u, l] = T_ul, downward D[l, u] = T_lu."""
    A, pa = _d(A)
    D, pd = _d(D)
    nb = A.shape[0]
    P = np.zeros(nb)
    st = lib().orc_solve_full(nb, pa, pd, P.ctypes.data_as(_D))
    if return_status:
        return P, st
    if st != OK:
        raise RuntimeError(f"orc_solve_full status {st}")
    return P


def ledger_full(A, D, E, P):
    A, pa = _d(A)
    D, pd = _d(D)
    E, pe = _d(E)
    P, pp = _d(P)
    out = np.zeros(2)
    lib().orc_ledger_full(E.size, pa, pd, pe, pp, out.ctypes.data_as(_D))
    return out


def grain_cooling_discrete(wl):
    """Thermal-discrete rates of every grain of a workload: a list of nb_g x nb_g arrays."""
    return [cooling_discrete(wl.lam, wl.cabs[g], wl.T[wl.grain_slice(g)], wl.E[wl.grain_slice(g)])
            for g in range(wl.n_grains)]


def solve_batch_discrete(wl, Dg=None, want_j=True, want_ledger=False, n_threads=0, u=None):
    """As solve_batch with thermal-discrete cooling (Dg: grain_cooling_discrete(wl))."""
    if Dg is None:
        Dg = grain_cooling_discrete(wl)
    u = wl.u if u is None else u
    lam, pl = _d(wl.lam)
    cabs, pc = _d(wl.cabs)
    off = np.ascontiguousarray(wl.bin_off, dtype=np.int32)
    T, pt = _d(wl.T)
    E, pe = _d(wl.E)
    Dall, pd = _d(np.concatenate([np.ascontiguousarray(d, dtype=np.float64).ravel() for d in Dg]))
    u, pu = _d(u)
    cells = u.shape[0]
    G, N = wl.n_grains, wl.n_lambda
    P = np.zeros((cells, wl.total_bins))
    j, pj = _dnull(np.zeros((cells, G, N)) if want_j else None)
    led, pld = _dnull(np.zeros((cells, G, 2)) if want_ledger else None)
    st = lib().orc_solve_batch_discrete(N, pl, G, pc, off.ctypes.data_as(_I), pt, pe, pd, cells, pu,
                                        P.ctypes.data_as(_D), pj, pld, int(n_threads))
    return P, j, led, st
