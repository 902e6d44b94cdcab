"""Pins of the oracle's thermal-discrete cooling (the approximation named beside Eq. adjacent)
and of its full stationary solve (Eq. steady-state with Eq. level-sum), on the CPU.

The rates are read as Eq. cooling's integrand restricted to each downward photon-energy
window, divided by the transition energy.  What fixes them independently of that code:
  * the windows tile [0, E_u]: the power the rates carry out of bin u equals Eq. cooling's
    total (an independent quadrature of the whole range), bin by bin;
  * with all emission softer than half a bin gap, every window but the adjacent one is
    empty and the treatment is the thermal-continuous one: rates equal Eq. cooling's and the
    full solve equals the Guhathakurta-Draine recursion (pinned elsewhere);
  * the solver against a dense LU solve of the balance equations, a two-state closed form,
    the energy ledger (absorbed = emitted for any stationary state) and the residual;
  * an undiluted blackbody: the discrete emission widens the small grain's distribution
    towards the canonical width that the continuous one underestimates."""
import numpy as np
import pytest

import oracle
from paper_1311_4627_gb300 import workloads as W


@pytest.fixture(scope="module")
def grain():
    wl = W.single_cell()
    g = 0  # 3.5 A: its photons span many bins
    s = wl.grain_slice(g)
    return wl.lam, wl.cabs[g], wl.T[s], wl.E[s], wl.u[0] * wl.cabs[g]


def test_windows_carry_the_cooling_power(grain):
    lam, cabs, T, E, _ = grain
    D = oracle.cooling_discrete(lam, cabs, T, E)
    for u in range(1, E.size):
        carried = sum(D[l, u] * (E[u] - E[l]) for l in range(u))
        total = oracle.emitted_power(lam, cabs, T[u], E[u])
        assert abs(carried / total - 1.0) < 1e-12, u
    assert np.all(D[np.tril_indices(E.size)] == 0.0)
    # most of a 3.5 A grain's emitted power skips levels (photons much larger than the gaps)
    share = [D[u - 1, u] * (E[u] - E[u - 1]) / oracle.emitted_power(lam, cabs, T[u], E[u]) for u in range(2, E.size)]
    assert np.median(share) < 0.1


def test_soft_emission_reduces_to_thermal_continuous():
    """Uniform bins of width dE and a cross-section that is zero shortward of hc/(1.2 dE):
    every emitted photon is softer than 1.5 dE, so only the adjacent window holds power."""
    lam = W.wavelength_grid(256)
    dE = W.H_PLANCK * W.C_LIGHT / (10.0 * W.UM)  # a 10 um photon
    nb = 40
    E = 0.5 * dE + dE * np.arange(nb)
    T = np.geomspace(20.0, 400.0, nb)
    cabs = W.cabs_model(3e-7, lam, "carbonaceous")
    cabs[lam < W.H_PLANCK * W.C_LIGHT / (1.2 * dE)] = 0.0
    D = oracle.cooling_discrete(lam, cabs, T, E)
    Cf = oracle.cooling(lam, cabs, T, E)
    off = D.copy()
    for u in range(1, nb):
        off[u - 1, u] = 0.0
    assert np.all(off == 0.0)
    np.testing.assert_allclose(np.array([D[u - 1, u] for u in range(1, nb)]), Cf[1:], rtol=1e-13)
    # a field that reaches the bins: the full solve is the recursion's
    u_field = W.three_bb_fields(lam, np.array([30.0]), np.array([0.2]), np.array([[0.3, 0.5, 0.2]]))[0]
    A = oracle.heating_matrix(lam, u_field * cabs, E)
    P_rec = oracle.recursion(oracle.b_matrix(A), Cf)
    P_full = oracle.solve_full(A, D)
    big = P_rec > 1e-280
    assert np.max(np.abs(P_full[big] / P_rec[big] - 1.0)) < 1e-12


def test_solver_against_dense_lu():
    """Random positive rates on 7 and 12 states: the state reduction against a dense LU solve
    of the balance equations with the last one replaced by the normalisation."""
    rng = np.random.default_rng(17)
    for nb in (7, 12):
        R = rng.uniform(0.1, 2.0, (nb, nb)) * (rng.random((nb, nb)) < 0.7)
        np.fill_diagonal(R, 0.0)
        for u in range(1, nb):  # every state must be able to decay
            R[u, u - 1] += 0.5
        A = np.zeros((nb, nb))
        D = np.zeros((nb, nb))
        for i in range(nb):
            for j in range(nb):
                if j > i:
                    A[j, i] = R[i, j]  # up from i to j
                elif j < i:
                    D[j, i] = R[i, j]  # down from i to j
        G = R.T - np.diag(R.sum(axis=1))  # dP/dt = G P
        Gs = G.copy()
        Gs[-1, :] = 1.0
        rhs = np.zeros(nb)
        rhs[-1] = 1.0
        P_lu = np.linalg.solve(Gs, rhs)
        P = oracle.solve_full(A, D)
        np.testing.assert_allclose(P, P_lu, rtol=1e-12, atol=0.0)
        assert abs(P.sum() - 1.0) < 1e-14


def test_two_states():
    A = np.array([[0.0, 0.0], [3.0, 0.0]])  # 0 -> 1 at rate 3
    D = np.array([[0.0, 5.0], [0.0, 0.0]])  # 1 -> 0 at rate 5
    P = oracle.solve_full(A, D)
    assert abs(P[1] / P[0] - 3.0 / 5.0) < 1e-15


def test_ledger_and_residual_of_a_discrete_spectrum(grain):
    lam, cabs, T, E, om = grain
    A = oracle.heating_matrix(lam, om, E)
    D = oracle.cooling_discrete(lam, cabs, T, E)
    P = oracle.solve_full(A, D)
    absorbed, emitted = oracle.ledger_full(A, D, E, P)
    assert abs(emitted / absorbed - 1.0) < 1e-12
    # residual of every balance equation relative to its largest term
    R = np.zeros((E.size, E.size))
    R[np.triu_indices(E.size, 1)] = A.T[np.triu_indices(E.size, 1)]  # up i -> j at A[j, i]
    R += D.T  # down i -> j at D[j, i]
    inflow = R.T @ P
    outflow = R.sum(axis=1) * P
    scale = np.maximum(inflow, outflow)
    ok = scale > 1e-250
    assert np.max(np.abs(inflow[ok] - outflow[ok]) / scale[ok]) < 1e-10


def test_blackbody_width_moves_towards_canonical():
    """A 5 A carbonaceous grain in an undiluted 60 K blackbody: the thermal-continuous P is
    about half as wide as the canonical distribution (k T^2 C); the discrete emission brings
    the width within 15 % of it, the mean energy within 10 %."""
    lam = W.wavelength_grid(256)
    a = 5e-8
    nat = W.n_atoms(a, "carbonaceous")
    T = np.geomspace(2.7, 2500.0, 128)
    E = W.debye_enthalpy(420.0, nat, T)
    cabs = W.cabs_model(a, lam, "carbonaceous")
    A = oracle.heating_matrix(lam, W.blackbody_field(lam, 60.0) * cabs, E)
    P_c = oracle.recursion(oracle.b_matrix(A), oracle.cooling(lam, cabs, T, E))
    P_d = oracle.solve_full(A, oracle.cooling_discrete(lam, cabs, T, E))
    H = W.debye_enthalpy(420.0, nat, np.array([60.0]))[0]
    Cv = (W.debye_enthalpy(420.0, nat, np.array([60.06]))[0] - W.debye_enthalpy(420.0, nat, np.array([59.94]))[0]) / 0.12
    canon = W.K_BOLTZ * 60.0**2 * Cv

    def width(P):
        m = np.sum(P * E)
        return m, np.sum(P * (E - m) ** 2) / canon

    m_c, v_c = width(P_c)
    m_d, v_d = width(P_d)
    assert v_c < 0.7 and abs(v_d - 1.0) < 0.15 and abs(v_d - 1.0) < abs(v_c - 1.0)
    assert abs(m_d / H - 1.0) < 0.1


def test_narrow_windows_against_extended_precision(grain):
    """A hot bin's photon that leaves the grain near the bottom: its photon-energy window is
    ~1e-9 of the photon energy wide.  The rates against a 40-digit quadrature of the same
    integral written in the grain's final energy (the window's limits are bin edges)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    lam, cabs, T, E, _ = grain
    D = oracle.cooling_discrete(lam, cabs, T, E)
    h, c, k = mp.mpf(W.H_PLANCK), mp.mpf(W.C_LIGHT), mp.mpf(W.K_BOLTZ)

    def c_at(x):
        x = float(x)
        n = 0 if x < lam[0] else min(max(int(np.searchsorted(lam, x, side="right")) - 1, 0), lam.size - 2)
        s = mp.log(mp.mpf(cabs[n + 1]) / cabs[n]) / mp.log(mp.mpf(lam[n + 1]) / lam[n])
        return mp.mpf(cabs[n]) * (mp.mpf(x) / lam[n]) ** s

    for u, l in ((127, 0), (127, 5), (113, 5), (99, 5)):
        Eu, Tu = mp.mpf(E[u]), mp.mpf(T[u])
        elo = mp.mpf(0) if l == 0 else (mp.mpf(E[l - 1]) + mp.mpf(E[l])) / 2
        ehi = (mp.mpf(E[l]) + mp.mpf(E[l + 1])) / 2
        f = lambda e: c_at(h * c / (Eu - e)) * (Eu - e) ** 3 / mp.expm1((Eu - e) / (k * Tu))  # noqa: E731
        ref = 8 * mp.pi / (h**3 * c**2) * mp.quad(f, [elo, ehi]) / (Eu - mp.mpf(E[l]))
        assert abs(float(mp.mpf(D[l, u]) / ref - 1)) < 1e-12, (u, l)
