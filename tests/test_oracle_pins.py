"""Pins for the FP64 oracle: closed forms, limits, brute force and invariants.

Each test ties one part of the oracle to something other than the oracle itself:
a closed-form integral, an exact rational solve, a dense linear solve, a
brute-force quadrature of an independently written interpolant, or an identity
of the method (Sec. 2 of the paper).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1311_4627_gb300 import workloads as W

H, C, K = W.H_PLANCK, W.C_LIGHT, W.K_BOLTZ
HC = H * C
SIGMA_SB = 2.0 * math.pi**5 * K**4 / (15.0 * H**3 * C**2)


def _bose_tail_series(x, kmax=4000):
    """int_0^x t^3/(e^t-1) dt = pi^4/15 - sum_k e^{-kx}(x^3/k + 3x^2/k^2 + 6x/k^3 + 6/k^4)."""
    s = 0.0
    for k in range(kmax, 0, -1):
        s += math.exp(-k * x) * (x**3 / k + 3 * x**2 / k**2 + 6 * x / k**3 + 6 / k**4)
    return math.pi**4 / 15.0 - s


# --------------------------------------------------------------------- cooling
def test_cooling_constant_cross_section_is_stefan_boltzmann():
    lam = W.wavelength_grid(64)
    cabs = np.full(lam.size, 3.7e-14)
    for T in (2.7, 20.0, 300.0, 2500.0):
        got = oracle.emitted_power(lam, cabs, T, 1e300)
        want = 4.0 * cabs[0] * SIGMA_SB * T**4
        assert abs(got / want - 1.0) < 1e-13, (T, got, want)


@pytest.mark.parametrize("xcut", [0.3, 1.0, 4.0, 17.0, 60.0])
def test_cooling_cutoff_is_incomplete_bose_integral(xcut):
    lam = W.wavelength_grid(128)
    cabs = np.full(lam.size, 1.0e-15)
    T = 50.0
    got = oracle.emitted_power(lam, cabs, T, xcut * K * T)
    want = 4.0 * math.pi * cabs[0] * 2.0 * K**4 * T**4 / (H**3 * C**2) * _bose_tail_series(xcut)
    assert abs(got / want - 1.0) < 1e-12


@pytest.mark.parametrize("s", [-2.0, -1.6, -1.0, 0.5])
def test_cooling_power_law_gamma_zeta(s):
    sp = pytest.importorskip("scipy.special")
    lam = W.wavelength_grid(200)
    lam0 = lam[17]
    C0 = 2.5e-12
    cabs = C0 * (lam / lam0) ** s  # exact power law: interpolant and continuation reproduce it
    for T in (5.0, 80.0, 1500.0):
        got = oracle.emitted_power(lam, cabs, T, 1e300)
        want = (4.0 * math.pi * 2.0 * K**4 * T**4 / (H**3 * C**2) * C0 * (HC / (lam0 * K * T)) ** s
                * sp.gamma(4.0 - s) * sp.zeta(4.0 - s))
        assert abs(got / want - 1.0) < 1e-12, (s, T, got, want)


def test_planck_integrates_to_sigma_t4_over_pi():
    T = 300.0
    t = np.linspace(math.log(1e-6), math.log(10.0), 200001)
    lam = np.exp(t)
    b = np.array([oracle.planck_lambda(x, T) for x in lam[::20]])
    # Simpson in ln(lambda) on the thinned grid
    f = b * lam[::20]
    h = t[20] - t[0]
    integ = h / 3.0 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
    assert abs(integ / (SIGMA_SB * T**4 / math.pi) - 1.0) < 1e-8


def test_cooling_rates_definition():
    wl = W.single_cell()
    s = wl.grain_slice(3)
    T, E, cabs = wl.T[s], wl.E[s], wl.cabs[3]
    Cf = oracle.cooling(wl.lam, cabs, T, E)
    assert Cf[0] == 0.0
    for f in (1, 40, 127):
        want = oracle.emitted_power(wl.lam, cabs, T[f], E[f]) / (E[f] - E[f - 1])
        assert Cf[f] == pytest.approx(want, rel=1e-15)
    assert np.all(Cf[1:] > 0) and np.all(np.diff(Cf[1:]) > 0)


# ------------------------------------------------------------ Omega integrals
def _loglog_python(lam, om, x):
    """Independent log-log interpolant (Eq. interpolation), zero off-grid or on zero segments."""
    if x < lam[0] or x > lam[-1]:
        return 0.0
    n = int(np.searchsorted(lam, x, side="right") - 1)
    n = min(max(n, 0), lam.size - 2)
    if om[n] <= 0 or om[n + 1] <= 0:
        return 0.0
    w = math.log(x / lam[n]) / math.log(lam[n + 1] / lam[n])
    return math.exp(math.log(om[n]) + w * math.log(om[n + 1] / om[n]))


@pytest.mark.parametrize("s,p", [(1.3, 1), (-2.0, 1), (-1.0, 0), (4.2, 0), (-0.7, 1)])
def test_range_integral_pure_power_law(s, p):
    lam = W.wavelength_grid(50)
    om0, lam0 = 3.0e-9, lam[10]
    om = om0 * (lam / lam0) ** s
    q = s + p + 1.0
    for a, b in [(lam[3] * 1.01, lam[40] * 0.97), (lam[0] * 0.5, lam[-1] * 2), (lam[7] * 1.001, lam[7] * 1.002)]:
        got = oracle.range_integral(lam, om, p, a, b)
        aa, bb = max(a, lam[0]), min(b, lam[-1])
        if q == 0.0:
            want = om0 * lam0 ** (p + 1) * math.log(bb / aa)
        else:
            want = om0 * lam0 ** (-s) * (bb**q - aa**q) / q
        assert abs(got / want - 1.0) < 1e-12, (a, b, got, want)


def test_range_integral_is_additive_across_segments():
    """int_a^c = int_a^b + int_b^c for split points inside a segment, on a node and across
    many segments (a wrong segment lookup or a dropped partial segment fails it)."""
    wl = W.single_cell()
    lam = wl.lam
    om = wl.u[0] * wl.cabs[3]
    for p in (0, 1):
        for a, b, c in [(lam[3] * 1.1, lam[3] * 1.2, lam[3] * 1.3), (lam[10] * 1.01, lam[40], lam[200] * 0.97),
                        (lam[0], lam[100] * 1.5, lam[-1]), (lam[50] * 0.999, lam[50] * 1.0005, lam[51] * 1.0001)]:
            whole = oracle.range_integral(lam, om, p, a, c)
            parts = oracle.range_integral(lam, om, p, a, b) + oracle.range_integral(lam, om, p, b, c)
            assert abs(parts / whole - 1.0) < 1e-13, (p, a, b, c)


def test_range_integral_bruteforce_quad():
    integrate = pytest.importorskip("scipy.integrate")
    rng = np.random.default_rng(7)
    lam = W.wavelength_grid(24)
    om = np.exp(rng.normal(0, 3, lam.size)) * 1e-10
    om[9] = 0.0  # kills segments 8 and 9
    for p in (0, 1):
        for a, b in [(lam[2] * 1.3, lam[20] * 0.8), (lam[0], lam[-1]), (lam[5] * 1.1, lam[12] * 1.05)]:
            got = oracle.range_integral(lam, om, p, a, b)
            pts = [x for x in lam if a < x < b]
            tot = 0.0
            edges = [a] + pts + [b]
            for x0, x1 in zip(edges[:-1], edges[1:]):
                v, _ = integrate.quad(lambda x: _loglog_python(lam, om, x) * x**p, x0, x1, epsabs=0, epsrel=1e-13,
                                      limit=200)
                tot += v
            assert abs(got / tot - 1.0) < 1e-11, (p, a, b, got, tot)
    assert oracle.omega_at(lam, om, 0.5 * (lam[8] + lam[9])) == 0.0
    assert oracle.omega_at(lam, om, lam[0] * 0.99) == 0.0


# ------------------------------------------------------------- heating matrix
def _edges(E):
    Elo = np.empty_like(E)
    Elo[0] = 0.0
    Elo[1:] = 0.5 * (E[1:] + E[:-1])
    return Elo


def test_heating_matrix_telescopes_to_closed_form_b():
    """Suffix sums of the explicit T_ul (Eq. brecurrence) equal one integral from
    0 to hc/(Elo_f - E_j): the bins' wavelength ranges tile the axis."""
    wl = W.single_cell()
    g = 1
    s = wl.grain_slice(g)
    E = wl.E[s][:48].copy()
    om = wl.u[0] * wl.cabs[g]
    A = oracle.heating_matrix(wl.lam, om, E)
    B = oracle.b_matrix(A)
    Elo = _edges(E)
    nb = E.size
    for f in range(1, nb):
        for j in range(f):
            want = oracle.range_integral(wl.lam, om, 1, 0.0, HC / (Elo[f] - E[j])) / H
            if f == j + 1:
                lsoft = HC / (Elo[j + 1] - E[j])
                want += C * oracle.range_integral(wl.lam, om, 0, lsoft, wl.lam[-1]) / (E[j + 1] - E[j])
            assert abs(B[f, j] - want) <= 1e-13 * abs(want) + 1e-300, (f, j, B[f, j], want)
    assert np.all(np.triu(A) == 0.0)
    assert np.all(A >= 0.0)


def test_heating_elements_bruteforce_quad():
    integrate = pytest.importorskip("scipy.integrate")
    wl = W.single_cell()
    g = 0
    s = wl.grain_slice(g)
    E = wl.E[s].copy()
    om = wl.u[0] * wl.cabs[g]
    A = oracle.heating_matrix(wl.lam, om, E)
    Elo = _edges(E)
    M = E.size - 1
    lam = wl.lam

    def quad(fun, a, b):
        a, b = max(a, lam[0]), min(b, lam[-1])
        if b <= a:
            return 0.0
        edges = [a] + [x for x in lam if a < x < b] + [b]
        return sum(integrate.quad(fun, x0, x1, epsabs=0, epsrel=1e-13, limit=200)[0]
                   for x0, x1 in zip(edges[:-1], edges[1:]))

    checked = 0
    for u, l in [(M, 0), (M, 100), (100, 3), (M, M - 1), (60, 59), (90, 10), (110, 50), (1, 0), (70, 69),
                 (120, 119), (126, 90)]:
        lb = HC / (Elo[u] - E[l])
        la = 0.0 if u == M else HC / (Elo[u + 1] - E[l])
        want = quad(lambda x: _loglog_python(lam, om, x) * x / H, la, lb)
        if u == l + 1:
            want += C * quad(lambda x: _loglog_python(lam, om, x), HC / (Elo[l + 1] - E[l]), lam[-1]) / (E[u] - E[l])
        if want == 0.0:
            assert A[u, l] == 0.0
        else:
            checked += 1
            assert abs(A[u, l] / want - 1.0) < 1e-10, (u, l, A[u, l], want)
    assert checked >= 5


# ------------------------------------------------------------------ recursion
def _dense_steady_state(A, Cf):
    """Solve Eq. steady-state with Eq. level-sum by dense LU (numpy)."""
    nb = A.shape[0]
    T = A.copy()
    for f in range(1, nb):
        T[f - 1, f] = Cf[f]
    G = T - np.diag(T.sum(axis=0))
    G[-1, :] = 1.0
    rhs = np.zeros(nb)
    rhs[-1] = 1.0
    return np.linalg.solve(G, rhs)


@pytest.mark.parametrize("nb", [2, 3, 5, 8, 12, 16])
def test_recursion_matches_dense_solve(nb):
    rng = np.random.default_rng(100 + nb)
    A = np.tril(np.exp(rng.normal(0, 1, (nb, nb))), -1)
    Cf = np.concatenate([[0.0], np.exp(rng.normal(0, 1, nb - 1))])
    P = oracle.recursion(oracle.b_matrix(A), Cf)
    Pd = _dense_steady_state(A, Cf)
    assert np.allclose(P, Pd, rtol=1e-11, atol=0)
    assert abs(P.sum() - 1.0) < 1e-14


def test_recursion_exact_rational():
    """Gaussian elimination in exact rationals of the original balance equations."""
    rng = np.random.default_rng(5)
    nb = 6
    A = [[Fraction(0)] * nb for _ in range(nb)]
    Af = np.zeros((nb, nb))
    for u in range(nb):
        for l in range(u):
            v = Fraction(int(rng.integers(1, 1000)), int(rng.integers(1, 50)))
            A[u][l] = v
            Af[u, l] = float(v)
    Cq = [Fraction(0)] + [Fraction(int(rng.integers(1, 1000)), int(rng.integers(1, 50))) for _ in range(nb - 1)]
    Cfl = np.array([float(x) for x in Cq])
    T = [row[:] for row in A]
    for f in range(1, nb):
        T[f - 1][f] = Cq[f]
    G = [[T[i][j] if i != j else -sum(T[k][i] for k in range(nb) if k != i) for j in range(nb)] for i in range(nb)]
    G[-1] = [Fraction(1)] * nb
    rhs = [Fraction(0)] * (nb - 1) + [Fraction(1)]
    for col in range(nb):  # Gauss-Jordan, exact
        piv = next(r for r in range(col, nb) if G[r][col] != 0)
        G[col], G[piv] = G[piv], G[col]
        rhs[col], rhs[piv] = rhs[piv], rhs[col]
        for r in range(nb):
            if r != col and G[r][col] != 0:
                fac = G[r][col] / G[col][col]
                G[r] = [a - fac * b for a, b in zip(G[r], G[col])]
                rhs[r] -= fac * rhs[col]
    exact = [rhs[i] / G[i][i] for i in range(nb)]
    P = oracle.recursion(oracle.b_matrix(Af), Cfl)
    for i in range(nb):
        assert abs(P[i] / float(exact[i]) - 1.0) < 1e-14


def test_recursion_manufactured_solution():
    rng = np.random.default_rng(11)
    nb = 200
    B = np.tril(np.exp(rng.normal(0, 2, (nb, nb))), -1)
    x = np.exp(-0.5 * ((np.arange(nb) - 80.0) / 20.0) ** 2)  # Boltzmann-like bump
    Pstar = x / x.sum()
    Cf = np.zeros(nb)
    for f in range(1, nb):
        Cf[f] = np.dot(B[f, :f], Pstar[:f]) / Pstar[f]
    P = oracle.recursion(B, Cf)
    assert np.allclose(P, Pstar, rtol=1e-12, atol=0)


def test_two_bins_closed_form():
    A = np.array([[0.0, 0.0], [3.25, 0.0]])
    Cf = np.array([0.0, 0.5])
    P = oracle.recursion(oracle.b_matrix(A), Cf)
    assert P[1] / P[0] == pytest.approx(3.25 / 0.5, rel=1e-15)
    assert P[0] == pytest.approx(1.0 / (1.0 + 6.5), rel=1e-15)


def test_recursion_power_of_two_rescale_geometric_chain():
    """B_{f,f-1} = r, C_f = 1: P_f = r^(f-M)(1-1/r)/(1-r^-nb); X overflows FP64 without rescaling."""
    nb, r = 400, 1.0e3
    B = np.zeros((nb, nb))
    for f in range(1, nb):
        B[f, f - 1] = r
    Cf = np.concatenate([[0.0], np.ones(nb - 1)])
    P = oracle.recursion(B, Cf)
    M = nb - 1
    logr = math.log(r)
    for f in range(nb):
        lw = (f - M) * logr + math.log1p(-1.0 / r) - math.log1p(-(r ** -nb) if nb * logr < 700 else 0.0)
        want = math.exp(lw) if lw > -690 else 0.0
        if want > 1e-280:
            assert abs(P[f] / want - 1.0) < 1e-12, (f, P[f], want)


def test_recursion_zero_cooling_status():
    A = np.array([[0, 0, 0], [1.0, 0, 0], [0.5, 2.0, 0]])
    _, st = oracle.recursion(oracle.b_matrix(A), np.array([0.0, 1.0, 0.0]), return_status=True)
    assert st == oracle.ENUMERIC
    A0 = np.zeros((3, 3))
    P, st = oracle.recursion(oracle.b_matrix(A0), np.array([0.0, 1.0, 0.0]), return_status=True)
    assert st == oracle.OK and P[0] == 1.0 and P[1] == 0.0 and P[2] == 0.0


# ------------------------------------------------------------- whole method
@pytest.fixture(scope="module")
def c1():
    wl = W.single_cell()
    Cf = oracle.grain_cooling(wl)
    P, j, led, st = oracle.solve_batch(wl, Cf, want_ledger=True)
    assert st == oracle.OK
    return wl, Cf, P, j, led


def test_probability_sums_to_one(c1):
    wl, _, P, _, _ = c1
    for g in range(wl.n_grains):
        p = P[0, wl.grain_slice(g)]
        assert abs(p.sum() - 1.0) < 1e-14
        assert np.all(p >= 0)


def test_energy_ledger_identity(c1):
    """Eq. bequation times (E_f - E_{f-1}), summed over f: absorbed == emitted."""
    _, _, _, _, led = c1
    rel = np.abs(led[0, :, 0] - led[0, :, 1]) / led[0, :, 1]
    assert np.all(rel < 1e-12), rel


def test_steady_state_balance_residual(c1):
    """P solves the untransformed balance equations (Eq. steady-state)."""
    wl, Cf, P, _, _ = c1
    g = 2
    s = wl.grain_slice(g)
    E, p = wl.E[s], P[0, s]
    A = oracle.heating_matrix(wl.lam, wl.u[0] * wl.cabs[g], E)
    T = A.copy()
    for f in range(1, E.size):
        T[f - 1, f] = Cf[s][f]
    inflow = T @ p
    outflow = T.sum(axis=0) * p
    scale = np.maximum(inflow, outflow)
    mask = scale > 1e-250
    assert np.all(np.abs(inflow - outflow)[mask] <= 1e-9 * scale[mask])


def test_zero_field_gives_ground_state(c1):
    wl, Cf, _, _, _ = c1
    u0 = np.zeros((1, wl.n_lambda))
    P, j, _, st = oracle.solve_batch(wl, Cf, u=u0)
    assert st == oracle.OK
    for g in range(wl.n_grains):
        s = wl.grain_slice(g)
        p = P[0, s]
        assert p[0] == 1.0 and np.all(p[1:] == 0.0)
        T0, E0 = wl.T[s][0], wl.E[s][0]
        want = np.array([wl.cabs[g][n] * oracle.planck_lambda(x, T0) if E0 >= HC / x else 0.0
                         for n, x in enumerate(wl.lam)])
        assert np.array_equal(j[0, g], want)


def test_emissivity_integrates_to_cooling_power():
    """4 pi int j dlambda for P = delta_i equals P_emit(T_i; E_i) of Eq. cooling."""
    lam = np.geomspace(1e-7, 50.0, 40001)
    cabs = np.full(lam.size, 2.0e-13)
    T = np.array([30.0, 60.0])
    E = np.array([1.0e-13, 5.0e-12])  # cut-offs at hc/E = 2.0 and 0.04 cm
    for i in range(2):
        P = np.zeros(2)
        P[i] = 1.0
        j = oracle.emissivity(lam, cabs, T, E, P)
        integ = 4.0 * math.pi * np.trapezoid(j, lam)
        want = oracle.emitted_power(lam, cabs, T[i], E[i])
        assert abs(integ / want - 1.0) < 2e-4, (i, integ, want)


@pytest.mark.parametrize("radius", [0.25e-4, 1.0e-4])
def test_large_grain_reaches_thermal_equilibrium(radius):
    """Undiluted blackbody at T_rad heats a large grain to T_rad (Kirchhoff):
    mode of P within one bin of T_rad, and j near the peak ~ C B_lambda(T_rad)."""
    lam = W.wavelength_grid(512)
    T_rad = 120.0
    wl = W.custom(lam, [radius], ["carbonaceous"], [512], W.blackbody_field(lam, T_rad)[None, :])
    Cf = oracle.grain_cooling(wl)
    P, j, led, st = oracle.solve_batch(wl, Cf, want_ledger=True)
    assert st == oracle.OK
    p = P[0]
    Tg = wl.T
    imode = int(np.argmax(p))
    dlnT = math.log(Tg[1] / Tg[0])
    assert abs(math.log(Tg[imode] / T_rad)) <= 1.01 * dlnT
    Tmean = math.exp(float(np.sum(p * np.log(Tg))))
    assert abs(math.log(Tmean / T_rad)) < 2 * dlnT
    bb = np.array([oracle.planck_lambda(x, T_rad) for x in lam]) * wl.cabs[0]
    npk = int(np.argmax(bb))
    assert abs(j[0, 0, npk] / bb[npk] - 1.0) < 0.02
    assert abs(led[0, 0, 0] / led[0, 0, 1] - 1.0) < 1e-10


@pytest.mark.parametrize("T_rad", [60.0, 300.0])
def test_undiluted_blackbody_gives_the_canonical_mean_energy(T_rad):
    """Inside an undiluted blackbody a grain of any size is in equilibrium with the field, so
    the mean enthalpy of P is the canonical one, H(T_rad) (Kirchhoff; H from the Debye model of
    the inputs, interpolated on the bin grid).  The thermal-continuous cooling of Eq. adjacent
    is not exact detailed balance, so for the smallest grains the mean is only close (within
    10 %) and the variance of H falls short of the canonical k T^2 C: for 5 A it is
    0.4-0.7 of it, the narrowing a drift-only cooling term gives (an exact Boltzmann P needs
    exact-statistical cooling).  From 20 A up the mean agrees to 2 %."""
    k = W.K_BOLTZ
    lam = W.wavelength_grid(512)
    for a in (5e-8, 10e-8, 20e-8, 50e-8, 250e-8):
        wl = W.custom(lam, [a], ["carbonaceous"], [512], W.blackbody_field(lam, T_rad)[None, :])
        P, _, _, st = oracle.solve_batch(wl, oracle.grain_cooling(wl), want_j=False)
        assert st == oracle.OK
        p, E, T = P[0], wl.E, wl.T
        H = lambda t: math.exp(float(np.interp(math.log(t), np.log(T), np.log(E))))
        Em = float(np.sum(p * E))
        tol = 0.10 if a < 20e-8 else 0.02
        assert abs(Em / H(T_rad) - 1.0) < tol, (a, Em / H(T_rad))
        if a == 5e-8:
            Cv = (H(1.001 * T_rad) - H(0.999 * T_rad)) / (0.002 * T_rad)
            ratio = float(np.sum(p * (E - Em) ** 2)) / (k * T_rad**2 * Cv)
            assert 0.3 < ratio < 0.8, ratio


@pytest.mark.parametrize("radius", [0.25e-4, 1.0e-4])
def test_large_grain_in_a_diluted_field_sits_at_the_balance_temperature(radius):
    """A large grain in a diluted 5000 K blackbody: T_eq from c int u C dlambda =
    4 pi int C B_lambda(T_eq) dlambda (trapezoid sums on the grid, root by brentq, written
    here independently of the oracle); the distribution's mean log T lies within one bin of
    T_eq and j at its peak is C B_lambda(T_eq) within 2 %."""
    from scipy import optimize

    lam = W.wavelength_grid(512)
    u = 1e-13 * W.blackbody_field(lam, 5000.0)
    wl = W.custom(lam, [radius], ["carbonaceous"], [512], u[None, :])
    C = wl.cabs[0]
    c, h, k = 2.99792458e10, 6.62607015e-27, 1.380649e-16

    def bl(T):
        with np.errstate(over="ignore"):
            return 2 * h * c * c / lam**5 / np.expm1(h * c / (lam * k * T))

    absorbed = c * np.trapezoid(u * C, lam)
    T_eq = optimize.brentq(lambda T: 4 * math.pi * np.trapezoid(C * bl(T), lam) - absorbed, 3.0, 2000.0, xtol=1e-10)
    P, j, _, st = oracle.solve_batch(wl, oracle.grain_cooling(wl))
    assert st == oracle.OK
    Tg = wl.T
    dlnT = math.log(Tg[1] / Tg[0])
    Tmean = math.exp(float(np.sum(P[0] * np.log(Tg))))
    assert abs(math.log(Tmean / T_eq)) <= dlnT, (Tmean, T_eq)
    bb = C * bl(T_eq)
    npk = int(np.argmax(bb))
    assert abs(j[0, 0, npk] / bb[npk] - 1.0) < 0.02, (j[0, 0, npk], bb[npk])


def test_size_integration_is_weighted_sum(c1):
    wl, _, _, j, _ = c1
    J = oracle.size_integrate(wl.size_weight, j)
    want = np.einsum("g,cgn->cn", wl.size_weight, j)
    assert np.allclose(J, want, rtol=1e-14, atol=0)


def test_size_integration_selects_and_adds(c1):
    """Eq. convolution discretised: a unit weight on one grain returns that grain's j exactly
    (a wrong axis or index fails it), and the sum is linear in the weights."""
    wl, _, _, j, _ = c1
    G = wl.n_grains
    for g in (0, G // 2, G - 1):
        w = np.zeros(G)
        w[g] = 1.0
        assert np.array_equal(oracle.size_integrate(w, j)[0], j[0, g])
    rng = np.random.default_rng(4)
    w1, w2 = rng.random(G), rng.random(G)
    lhs = oracle.size_integrate(w1 + w2, j)
    rhs = oracle.size_integrate(w1, j) + oracle.size_integrate(w2, j)
    assert np.allclose(lhs, rhs, rtol=1e-13, atol=0)


# ------------------------------------------------------- grain thermal model
def test_debye_enthalpy_limits():
    theta, n = 420.0, 1.0e4
    T = theta / 100.0
    low = 3.0 * math.pi**4 / 5.0 * n * K * T**4 / theta**3
    assert W.debye_enthalpy(theta, n, T)[0] == pytest.approx(low, rel=1e-12)
    T = theta * 100.0
    y = theta / T
    high = 3 * n * K * T - 9.0 / 8.0 * n * K * theta + 3.0 / 20.0 * n * K * theta * y
    assert W.debye_enthalpy(theta, n, T)[0] == pytest.approx(high, rel=1e-11)
