"""Seeded synthetic workloads: wavelength grids, grain models and radiation fields.

This module produces *inputs* only.  It contains none of the stochastic-heating
arithmetic (no heating or cooling rates, no recursion, no emissivity); the
library and the oracle both take what it makes as plain arrays.  All draws use
numpy's PCG64 with seed ``1000 + workload number``.

Stand-ins for the paper's data (Sec. 2 benchmarks use Draine/Li & Draine optics,
WD01 size distributions and the Mathis ISRF, none of which ship with the paper):

* grain enthalpy: Debye model with 3 N_atoms modes (theta_D 420 K carbonaceous,
  500 K silicate), zero-point energy excluded;
* C_abs = pi a^2 min(1, (2 pi a / lambda) k(lambda)), k = k0 (lambda/1 um)^(1-beta)
  plus a Drude bump at 0.2175 um of width 1 um^-1, so that Q ~ lambda^-beta
  (beta = 2.0 carbonaceous, 1.6 silicate: the emissivity index);
* u_lambda = chi * norm * sum_m w_m (4 pi / c) B_lambda(T_m) (lambda / 0.55 um)^-h,
  T_m = 3000, 4000, 7500 K, w_m = 10^U(-2, 0), norm fixing the grid integral of
  u_lambda (without chi) at 0.46 eV cm^-3 (the paper's ISRF energy density);
* size-distribution weights w_g = Q(a_g) da_g with Q = A a^-3.5 (MRN).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# CODATA 2018 exact values (CGS)
H_PLANCK = 6.62607015e-27
C_LIGHT = 2.99792458e10
K_BOLTZ = 1.380649e-16
EV = 1.602176634e-12
AMU = 1.66053906660e-24
UM = 1e-4  # cm

ISRF_ENERGY_DENSITY = 0.46 * EV  # erg cm^-3
FIELD_TEMPS = (3000.0, 4000.0, 7500.0)

COMPOSITIONS = {
    # name: (theta_D [K], rho [g cm^-3], mean atomic mass [g], k0, k_drude, beta)
    "carbonaceous": (420.0, 2.2, 12.011 * AMU, 1.0, 2.0, 2.0),
    "silicate": (500.0, 3.5, 172.24 / 7.0 * AMU, 1.0, 0.0, 1.6),
}


# ----------------------------------------------------------------------------
# grain thermal model
def _bose_integral(y: np.ndarray) -> np.ndarray:
    """D(y) = int_0^y x^3/(e^x - 1) dx by composite 32-point Gauss-Legendre."""
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    xg, wg = np.polynomial.legendre.leggauss(32)
    out = np.empty_like(y)
    for idx, yy in enumerate(y):
        top = min(yy, 60.0)  # x^3 e^-x < 1e-20 of the total beyond
        npan = max(1, int(math.ceil(top / 2.0)))
        edges = np.linspace(0.0, top, npan + 1)
        a, b = edges[:-1, None], edges[1:, None]
        x = 0.5 * (a + b) + 0.5 * (b - a) * xg[None, :]
        f = x**3 / np.expm1(x)
        out[idx] = float(np.sum(0.5 * (b - a) * wg[None, :] * f))
    return out


def n_atoms(radius_cm: float, composition: str) -> float:
    _, rho, mbar, *_ = COMPOSITIONS[composition]
    return 4.0 / 3.0 * math.pi * radius_cm**3 * rho / mbar


def debye_enthalpy(theta_d: float, natoms: float, T) -> np.ndarray:
    """H(T) = 9 N k T (T/theta)^3 int_0^{theta/T} x^3/(e^x-1) dx (erg)."""
    T = np.atleast_1d(np.asarray(T, dtype=np.float64))
    return 9.0 * natoms * K_BOLTZ * T * (T / theta_d) ** 3 * _bose_integral(theta_d / T)


def cabs_model(radius_cm: float, lam_cm: np.ndarray, composition: str) -> np.ndarray:
    """Synthetic absorption cross-section (cm^2) on the wavelength grid."""
    _, _, _, k0, kd, beta = COMPOSITIONS[composition]
    lam_um = lam_cm / UM
    x = 1.0 / lam_um
    x0, gam = 1.0 / 0.2175, 1.0
    k = k0 * lam_um ** (1.0 - beta) + kd * x**2 * gam**2 / ((x**2 - x0**2) ** 2 + x**2 * gam**2)
    q = np.minimum(1.0, 2.0 * math.pi * radius_cm / lam_cm * k)
    return math.pi * radius_cm**2 * q


# ----------------------------------------------------------------------------
# radiation fields
def _bb_energy_density(lam_cm: np.ndarray, T: float) -> np.ndarray:
    """(4 pi / c) B_lambda(T) in erg cm^-3 cm^-1 (undiluted blackbody)."""
    x = H_PLANCK * C_LIGHT / (lam_cm * K_BOLTZ * T)
    with np.errstate(over="ignore"):
        b = 2.0 * H_PLANCK * C_LIGHT**2 / lam_cm**5 / np.expm1(x)
    return 4.0 * math.pi / C_LIGHT * b


def blackbody_field(lam_cm: np.ndarray, T: float) -> np.ndarray:
    """Undiluted blackbody energy density; used by the thermal-limit checks."""
    return _bb_energy_density(lam_cm, T)


def three_bb_fields(lam_cm: np.ndarray, chi: np.ndarray, hardness: np.ndarray, wts: np.ndarray) -> np.ndarray:
    """u[c, n] for per-cell chi, hardness h and blackbody weights wts[c, 3].  Every operation
    is per cell (no cross-cell reductions or blocked library products), so a cell's field
    does not depend on which other cells are generated with it."""
    basis = np.stack([_bb_energy_density(lam_cm, T) for T in FIELD_TEMPS])  # [3, N]
    u = np.multiply.outer(-hardness, np.log(lam_cm / (0.55 * UM)))  # tilt (lambda / 0.55 um)^-h
    np.exp(u, out=u)
    mix = wts[:, 0:1] * basis[0][None, :]
    mix += wts[:, 1:2] * basis[1][None, :]
    mix += wts[:, 2:3] * basis[2][None, :]
    u *= mix
    del mix
    dl = np.diff(lam_cm)
    integral = np.sum(0.5 * (u[:, 1:] + u[:, :-1]) * dl[None, :], axis=1)
    u *= (chi * ISRF_ENERGY_DENSITY / integral)[:, None]
    return u


# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    lam: np.ndarray  # [N] cm, ascending
    radius: np.ndarray  # [G] cm
    composition: list  # [G] names
    cabs: np.ndarray  # [G, N] cm^2
    bin_off: np.ndarray  # [G+1] int32
    T: np.ndarray  # [bin_off[G]] K
    E: np.ndarray  # [bin_off[G]] erg
    size_weight: np.ndarray  # [G] Q(a) da per H
    u: np.ndarray | None = None  # [cells, N] erg cm^-3 cm^-1
    chi: np.ndarray | None = None
    hardness: np.ndarray | None = None

    @property
    def n_lambda(self) -> int:
        return int(self.lam.size)

    @property
    def n_grains(self) -> int:
        return int(self.radius.size)

    @property
    def n_cells(self) -> int:
        return 0 if self.u is None else int(self.u.shape[0])

    @property
    def total_bins(self) -> int:
        return int(self.bin_off[-1])

    def bins(self, g: int) -> int:
        return int(self.bin_off[g + 1] - self.bin_off[g])

    def grain_slice(self, g: int) -> slice:
        return slice(int(self.bin_off[g]), int(self.bin_off[g + 1]))


def wavelength_grid(n: int, lo_um: float = 0.0912, hi_um: float = 1000.0) -> np.ndarray:
    return np.geomspace(lo_um * UM, hi_um * UM, n)


def make_grains(lam: np.ndarray, radii_cm, compositions, nbins, t_lo=2.7, t_hi=2500.0):
    radii = np.asarray(radii_cm, dtype=np.float64)
    nbins = np.asarray(nbins, dtype=np.int64)
    G = radii.size
    off = np.zeros(G + 1, dtype=np.int32)
    off[1:] = np.cumsum(nbins)
    T = np.empty(off[-1])
    E = np.empty(off[-1])
    cabs = np.empty((G, lam.size))
    for g in range(G):
        comp = compositions[g]
        tg = np.geomspace(t_lo, t_hi, int(nbins[g]))
        T[off[g]:off[g + 1]] = tg
        E[off[g]:off[g + 1]] = debye_enthalpy(COMPOSITIONS[comp][0], n_atoms(radii[g], comp), tg)
        cabs[g] = cabs_model(radii[g], lam, comp)
    dln = np.gradient(np.log(radii)) if G > 1 else np.ones(1)
    a_mrn = 10 ** (-25.16)
    size_weight = a_mrn * radii ** (-3.5) * radii * np.abs(dln)
    return radii, list(compositions), cabs, off, T, E, size_weight


def _workload(name, lam, radii, comps, nbins, cells, seed, chi_lo, chi_hi, hard_lo, hard_hi, fields=True):
    radii, comps, cabs, off, T, E, sw = make_grains(lam, radii, comps, nbins)
    wl = Workload(name, lam, radii, comps, cabs, off, T, E, sw)
    if fields and cells > 0:
        rng = np.random.Generator(np.random.PCG64(seed))
        chi = np.exp(rng.uniform(math.log(chi_lo), math.log(chi_hi), cells))
        hard = rng.uniform(hard_lo, hard_hi, cells) if hard_hi > hard_lo else np.zeros(cells)
        wts = 10.0 ** rng.uniform(-2.0, 0.0, (cells, 3))
        wl.u = three_bb_fields(lam, chi, hard, wts)
        wl.chi, wl.hardness = chi, hard
    return wl


def single_cell(seed_offset: int = 0) -> Workload:
    """1 cell x 8 carbonaceous radii (3.5-250 A), 128 bins, 256 wavelengths, FP64."""
    lam = wavelength_grid(256)
    radii = np.geomspace(3.5e-8, 250e-8, 8)
    return _workload("single-cell 1x8 grains, 128 bins, 256 wavelengths", lam, radii, ["carbonaceous"] * 8,
                     [128] * 8, 1, 1001 + seed_offset, 0.1, 100.0, 0.0, 0.0)


def batched_bins(g: int, G: int = 64) -> int:
    """Bins per grain for the batched workload: 32 * round(4 + 28 g / 63)."""
    return 32 * int(round(4 + 28 * g / (G - 1)))


def batched(cells: int = 4096, n_lambda: int = 1024, grains: int = 64, seed: int = 1002) -> Workload:
    """cells x 64 radii (3.5 A - 1 um), alternating carbonaceous / silicate,
    128-1024 bins growing with radius, 1024 wavelengths, chi in [1e-2, 1e4]."""
    lam = wavelength_grid(n_lambda)
    radii = np.geomspace(3.5e-8, 1e-4, grains)
    comps = ["carbonaceous" if g % 2 == 0 else "silicate" for g in range(grains)]
    nb = [batched_bins(g, grains) for g in range(grains)]
    return _workload(f"batched {cells} cells x {grains} grains, 128-1024 bins, {n_lambda} wavelengths", lam,
                     radii, comps, nb, cells, seed, 1e-2, 1e4, -1.0, 1.0)


def composition_flags(wl: Workload) -> np.ndarray:
    """1 for silicate grains, 0 for carbonaceous (the surrogate's composition input)."""
    return np.array([1.0 if c == "silicate" else 0.0 for c in wl.composition], dtype=np.float32)


def emissivity_heavy(cells: int = 65536, n_lambda: int = 2048, grains: int = 32, nbins: int = 512) -> Workload:
    """cells x 32 carbonaceous radii x 512 bins x 2048 wavelengths."""
    lam = wavelength_grid(n_lambda)
    radii = np.geomspace(3.5e-8, 1e-4, grains)
    return _workload(f"emissivity {cells} cells x {grains} grains x {nbins} bins x {n_lambda} wavelengths", lam,
                     radii, ["carbonaceous"] * grains, [nbins] * grains, cells, 1003, 1e-2, 1e4, -1.0, 1.0)


def field_subset(wl: Workload, cells) -> Workload:
    """Same grid and grains, a subset of the cells."""
    cells = np.asarray(cells)
    out = dataclasses.replace(wl)
    out.u = wl.u[cells]
    out.chi = None if wl.chi is None else wl.chi[cells]
    out.hardness = None if wl.hardness is None else wl.hardness[cells]
    return out


def custom(lam, radii, comps, nbins, u) -> Workload:
    radii, comps, cabs, off, T, E, sw = make_grains(lam, radii, comps, nbins)
    return Workload("custom", lam, radii, comps, cabs, off, T, E, sw, u=np.atleast_2d(np.asarray(u, np.float64)))


def grain_subset(wl: Workload, grains) -> Workload:
    """Same grid and fields, only the listed grains (in the given order)."""
    grains = [int(g) for g in grains]
    nb = [wl.bins(g) for g in grains]
    off = np.zeros(len(grains) + 1, dtype=np.int32)
    off[1:] = np.cumsum(nb)
    T = np.concatenate([wl.T[wl.grain_slice(g)] for g in grains])
    E = np.concatenate([wl.E[wl.grain_slice(g)] for g in grains])
    return Workload(wl.name + f" [grains {grains}]", wl.lam, wl.radius[grains], [wl.composition[g] for g in grains],
                    wl.cabs[grains], off, T, E, wl.size_weight[grains], u=wl.u, chi=wl.chi, hardness=wl.hardness)


# ---------------------------------------------------------------------------- volume
def gaussian_random_field(shape, corr_cells: float, rng: np.random.Generator) -> np.ndarray:
    """Periodic Gaussian random field on a grid: white noise smoothed by a Gaussian kernel of
    standard deviation corr_cells (in cells), through the FFT; normalised to zero mean and
    unit variance.  Its autocorrelation at separation r is exp(-r^2 / (4 corr_cells^2))."""
    noise = rng.standard_normal(shape)
    k2 = np.zeros(shape)
    for ax, n in enumerate(shape):
        k = 2.0 * math.pi * np.fft.fftfreq(n)
        sh = [1] * len(shape)
        sh[ax] = n
        k2 = k2 + (k**2).reshape(sh)
    f = np.fft.ifftn(np.fft.fftn(noise) * np.exp(-0.5 * k2 * corr_cells**2)).real
    return (f - f.mean()) / f.std()


@dataclasses.dataclass
class Volume:
    """A radiative-transfer volume: grains, and per cell the field parameters (chi, hardness,
    blackbody weights) from which u is made chunk by chunk (u of the whole volume is
    n_cells x n_lambda FP64, too large to keep)."""
    grains: Workload  # grid and grains (no fields)
    shape: tuple
    chi: np.ndarray  # [cells]
    hardness: np.ndarray  # [cells]
    wts: np.ndarray  # [cells, 3]
    seed: int

    @property
    def n_cells(self) -> int:
        return int(self.chi.size)

    def fields(self, begin: int, end: int, threads: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
        """u of cells [begin, end) (x-fastest order of the grid), generated in blocks of 4096
        cells on host threads (numpy releases the GIL; the cells are independent; default one
        thread per core, at most 16); into `out` ([end - begin][n_lambda] FP64) if given."""
        import os
        from concurrent.futures import ThreadPoolExecutor

        if threads is None:
            threads = min(16, os.cpu_count() or 1)

        lam = self.grains.lam
        if out is None:
            out = np.empty((end - begin, lam.size))

        def block(b):
            e = min(end, b + 4096)
            out[b - begin:e - begin] = three_bb_fields(lam, self.chi[b:e], self.hardness[b:e], self.wts[b:e])

        starts = range(begin, end, 4096)
        if threads > 1 and len(starts) > 1:
            with ThreadPoolExecutor(min(threads, len(starts))) as pool:
                list(pool.map(block, starts))
        else:
            for b in starts:
                block(b)
        return out


def rt_volume(shape=(128, 128, 64), corr_cells: float = 8.0, radii_per_composition: int = 40, nbins: int = 512,
              n_lambda: int = 1024, seed: int = 1005) -> Volume:
    """Gaussian-random-field volume: log10 chi a GRF of mean 0 and standard deviation 1.5,
    hardness a GRF of standard deviation 0.5 clipped to [-1, 1] (correlation length
    corr_cells), blackbody weights 10^U(-2, 0); grains: carbonaceous and silicate at
    radii_per_composition radii (3.5 A - 1 um), nbins bins each, n_lambda wavelengths."""
    lam = wavelength_grid(n_lambda)
    radii = np.geomspace(3.5e-8, 1e-4, radii_per_composition)
    rs = np.concatenate([radii, radii])
    comps = ["carbonaceous"] * radii_per_composition + ["silicate"] * radii_per_composition
    grains = _workload(f"volume {shape} x {2 * radii_per_composition} grains x {nbins} bins x {n_lambda} wavelengths",
                       lam, rs, comps, [nbins] * rs.size, 0, seed, 1.0, 1.0, 0.0, 0.0, fields=False)
    rng = np.random.Generator(np.random.PCG64(seed))
    g1 = gaussian_random_field(shape, corr_cells, rng)
    g2 = gaussian_random_field(shape, corr_cells, rng)
    cells = int(np.prod(shape))
    # x-fastest cell order: cell index = x + nx (y + ny z)
    chi = 10.0 ** (1.5 * g1.transpose().reshape(cells))
    hard = np.clip(0.5 * g2.transpose().reshape(cells), -1.0, 1.0)
    wts = 10.0 ** rng.uniform(-2.0, 0.0, (cells, 3))
    return Volume(grains, tuple(shape), chi, hard, wts, seed)
