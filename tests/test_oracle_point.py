"""Pins for the oracle's point-rule heating (Eq. heating, the paper's own form).

T_ul = Omega(lambda_ul) lambda_ul^3 dE_u / (h^2 c), lambda_ul = hc / (E_u - E_l), Omega the
log-log interpolant of Eq. interpolation, dE_u the width of the upper bin (the top bin
takes E_M - E_{M-1}), no intra-bin term.  Each test ties it to something other than the
oracle: the closed-form integral of a power law (the point rule is the midpoint rule of
the integral form, with a known error), a translation invariance of uniform grids, exact
zeros off the wavelength grid, and the balance equations the solve must satisfy.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1311_4627_gb300 import workloads as W

H, C = W.H_PLANCK, W.C_LIGHT
HC = H * C
EV = 1.602176634e-12


def _edges(E):
    Elo = np.empty_like(E)
    Elo[0] = 0.0
    Elo[1:] = 0.5 * (E[1:] + E[:-1])
    Ehi = np.empty_like(E)
    Ehi[:-1] = Elo[1:]
    Ehi[-1] = math.inf
    return Elo, Ehi


def _power_law(lam, s, om0=2.0e-7):
    lam0 = lam[lam.size // 2]
    return om0 * (lam / lam0) ** s, om0, lam0


def _bin_integral(om0, lam0, s, e_lo, e_hi):
    """(1/h) int Omega lambda dlambda over the photon energies [e_lo, e_hi] for
    Omega = om0 (lambda/lam0)^s, written in photon energy: the integrand is
    om0 lam0^-s (hc)^(s+2) / h * eps^-(s+3), integrated in closed form."""
    k = s + 3.0
    pref = om0 * lam0 ** (-s) * HC ** (s + 2.0) / H
    if k == 1.0:
        return pref * math.log(e_hi / e_lo)
    return pref * (e_lo ** (1.0 - k) - e_hi ** (1.0 - k)) / (k - 1.0)


@pytest.mark.parametrize("s", [-2.0, -1.0, 0.0, 1.3])
def test_point_rule_is_the_midpoint_rule_of_the_bin_integral(s):
    """Uniform enthalpy grid, power-law Omega: the point element is d * f(eps) with f the
    integrand in photon energy, the integral form is int f over [eps - d/2, eps + d/2].
    Their ratio is 1 - k(k+1)/24 (d/eps)^2 + O((d/eps)^4), k = s + 3.  A wrong constant,
    a wrong power of lambda, or a point off the bin centre fails this."""
    lam = W.wavelength_grid(200)
    om, om0, lam0 = _power_law(lam, s)
    d = 0.02 * EV
    nb = 200
    E = 0.5 * EV + d * np.arange(nb)
    A = oracle.heating_matrix_point(lam, om, E)
    k = s + 3.0
    checked = 0
    for u in range(1, nb - 1):
        for l in range(0, u, 7):
            eps = E[u] - E[l]
            if (u - l) < 8 or HC / (eps - d / 2) > lam[-1] or HC / (eps + d / 2) < lam[0]:
                continue
            want = _bin_integral(om0, lam0, s, eps - d / 2, eps + d / 2)
            x = d / eps
            pred = 1.0 - k * (k + 1.0) / 24.0 * x * x
            assert abs(A[u, l] / want - pred) <= 0.05 * k**4 * x**4 + 1e-12, (u, l, A[u, l] / want, pred)
            checked += 1
    assert checked > 500


def test_point_rule_takes_the_upper_bin_width():
    """Bin widths jump from d to 1.5 d at bin K, so the upper and the lower bin of a
    transition differ by up to 20% there.  The point rule with the upper width stays within
    its first-order midpoint bound of the bin integral; taking the lower width would not."""
    lam = W.wavelength_grid(200)
    s = 0.5
    om, om0, lam0 = _power_law(lam, s)
    d, K, nb = 0.02 * EV, 100, 160
    steps = np.where(np.arange(1, nb) <= K, d, 1.5 * d)
    E = 0.5 * EV + np.concatenate([[0.0], np.cumsum(steps)])
    Elo, Ehi = _edges(E)
    A = oracle.heating_matrix_point(lam, om, E)
    k = s + 3.0
    checked = 0
    for u in range(K - 3, K + 4):
        w_up = Ehi[u] - Elo[u]
        w_low = Ehi[u - 1] - Elo[u - 1]
        delta = E[u] - 0.5 * (Elo[u] + Ehi[u])
        for l in range(0, u - 40):
            eps = E[u] - E[l]
            want = _bin_integral(om0, lam0, s, Elo[u] - E[l], Ehi[u] - E[l])
            bound = 1.5 * (k * abs(delta) / eps + k * (k + 1) / 2 * (delta / eps) ** 2
                           + k * (k + 1) / 24 * (w_up / eps) ** 2)
            r = A[u, l] / want
            assert abs(r - 1.0) <= bound, (u, l, r, bound)
            if abs(w_up / w_low - 1.0) > 0.1:
                assert abs(r * w_low / w_up - 1.0) > 2 * bound
            checked += 1
    assert checked > 300


def test_uniform_grid_is_translation_invariant_including_the_top_bin():
    """On a uniform grid every bin (the open top bin included, which takes E_M - E_{M-1})
    has the same width, so T_ul depends on u - l only."""
    wl = W.single_cell()
    om = wl.u[0] * wl.cabs[2]
    d = 0.05 * EV
    E = 1e-3 * EV + d * np.arange(96)
    A = oracle.heating_matrix_point(wl.lam, om, E)
    for u in range(2, E.size):
        for l in range(1, u):
            a, b = A[u, l], A[u - 1, l - 1]
            assert abs(a - b) <= 1e-13 * max(abs(a), abs(b)), (u, l, a, b)
    assert np.all(np.triu(A) == 0.0)
    assert A[E.size - 1, 0] > 0.0


def test_transitions_off_the_wavelength_grid_are_zero():
    """Omega is zero outside [lambda_0, lambda_{N-1}]: transitions whose photon would be
    harder than hc/lambda_0 or softer than hc/lambda_{N-1} get exactly zero."""
    wl = W.single_cell()
    lam = wl.lam
    om = wl.u[0] * wl.cabs[0]
    E = np.concatenate([[0.0], np.geomspace(0.5 * HC / lam[-1], 3.0 * HC / lam[0], 80)])
    A = oracle.heating_matrix_point(lam, om, E)
    eps = E[:, None] - E[None, :]
    lo = np.tril(np.ones_like(A, dtype=bool), -1)
    off = lo & ((eps > HC / lam[0]) | (eps < HC / lam[-1]))
    on = lo & ~off
    assert off.sum() > 50 and on.sum() > 50
    assert np.all(A[off] == 0.0)
    assert np.all(A[on] > 0.0)


def test_point_rule_elements_from_an_independent_interpolant():
    """Elements of a real grain against a separately written log-log interpolant times the
    photon count per unit photon energy (Omega lambda / h per unit wavelength, times
    d lambda / d E = lambda^2 / (hc))."""
    wl = W.single_cell()
    g = 1
    s = wl.grain_slice(g)
    E = wl.E[s]
    om = wl.u[0] * wl.cabs[g]
    A = oracle.heating_matrix_point(wl.lam, om, E)
    Elo, Ehi = _edges(E)
    M = E.size - 1
    lam = wl.lam

    def loglog(x):
        if x < lam[0] or x > lam[-1]:
            return 0.0
        n = min(max(int(np.searchsorted(lam, x, side="right")) - 1, 0), lam.size - 2)
        w = math.log(x / lam[n]) / math.log(lam[n + 1] / lam[n])
        return om[n] ** (1.0 - w) * om[n + 1] ** w

    for u, l in [(1, 0), (5, 2), (40, 39), (77, 12), (M - 1, 0), (M, 0), (M, M - 1), (100, 99), (120, 64)]:
        x = HC / (E[u] - E[l])
        width = (Ehi[u] - Elo[u]) if u < M else (E[M] - E[M - 1])
        want = loglog(x) * x / H * (x * x / HC) * width
        assert abs(A[u, l] - want) <= 1e-12 * abs(want) + 1e-300, (u, l, A[u, l], want)


@pytest.fixture(scope="module")
def c1_point():
    wl = W.single_cell()
    Cf = oracle.grain_cooling(wl)
    P, j, led, st = oracle.solve_batch(wl, Cf, want_ledger=True, heating=oracle.HEATING_POINT)
    assert st == oracle.OK
    Pi, ji, li, st = oracle.solve_batch(wl, Cf, want_ledger=True)
    assert st == oracle.OK
    return wl, Cf, P, j, led, Pi, ji, li


def test_point_solve_is_the_recursion_of_the_point_matrix(c1_point):
    """The batch solve in point mode equals the explicit chain T -> B (Eq. brecurrence)
    -> recursion (Eq. xf) on the point matrix, and sums to one."""
    wl, Cf, P, _, _, _, _, _ = c1_point
    for g in range(wl.n_grains):
        s = wl.grain_slice(g)
        A = oracle.heating_matrix_point(wl.lam, wl.u[0] * wl.cabs[g], wl.E[s])
        p = oracle.recursion(oracle.b_matrix(A), Cf[s])
        assert np.array_equal(p, P[0, s])
        assert abs(P[0, s].sum() - 1.0) < 1e-14 and np.all(P[0, s] >= 0)


@pytest.mark.parametrize("g", [0, 3, 6])
def test_point_solve_balances_the_master_equation(c1_point, g):
    """P solves the untransformed balance equations (Eq. steady-state) with the point T."""
    wl, Cf, P, _, _, _, _, _ = c1_point
    s = wl.grain_slice(g)
    E, p = wl.E[s], P[0, s]
    T = oracle.heating_matrix_point(wl.lam, wl.u[0] * wl.cabs[g], E)
    for f in range(1, E.size):
        T[f - 1, f] = Cf[s][f]
    inflow = T @ p
    outflow = T.sum(axis=0) * p
    scale = np.maximum(inflow, outflow)
    mask = scale > 1e-250
    assert np.all(np.abs(inflow - outflow)[mask] <= 1e-9 * scale[mask])


def test_point_solve_energy_ledger(c1_point):
    """Absorbed power equals emitted power of the discrete model for any heating matrix."""
    _, _, _, _, led, _, _, _ = c1_point
    rel = np.abs(led[0, :, 0] - led[0, :, 1]) / led[0, :, 1]
    assert np.all(rel < 1e-12), rel


def test_point_versus_integral_on_the_single_cell_workload(c1_point):
    """A/B of the two heating forms on the 8-grain, 128-bin, 1024-wavelength case.  Small
    grains: bins narrow against the photon energies, the point rule is the midpoint rule
    of the integral, and the absorbed power agrees to about 1%, with the same peak
    temperature.  Large grains: bins wider than most photons; the point rule has no
    intra-bin term, so sub-bin photons are lost and the grain is underheated, the more
    so the larger it is."""
    wl, _, P, j, led, Pi, ji, li = c1_point
    ratio = led[0, :, 0] / li[0, :, 0]
    small = wl.radius < 25e-8
    large = wl.radius > 70e-8
    assert small.sum() >= 3 and large.sum() >= 2
    assert np.all(np.abs(ratio[small] - 1.0) < 0.02), ratio
    assert np.all(ratio[large] < 0.2), ratio
    order = np.argsort(wl.radius)
    r_sorted = ratio[order][wl.radius[order] > 35e-8]
    assert np.all(np.diff(r_sorted) < 0), r_sorted
    for g in np.flatnonzero(small):
        s = wl.grain_slice(g)
        assert np.argmax(P[0, s]) == np.argmax(Pi[0, s])
        pk = ji[0, g].max()
        m = ji[0, g] > 1e-3 * pk
        assert np.median(np.abs(j[0, g][m] / ji[0, g][m] - 1.0)) < 0.02
