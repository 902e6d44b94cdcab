"""Writes the stored expected values of tests/golden/ from the FP64 oracle (and nothing else).

The paper prints no numeric results (its one figure is elided), so the fixtures here are the
oracle's outputs on the seeded single-cell workload (1 cell x 8 carbonaceous grains of
3.5-250 A, 128 bins each, 256 wavelengths):

  single_cell_exact.txt     P of every grain (Guhathakurta-Draine recursion, Eq. xf, and
                            renormalisation), j at every 8th wavelength (Eq. emission), and the
                            energy ledger [absorbed, emitted] per grain
  single_cell_discrete.txt  P of grains 0 and 7 with thermal-discrete cooling (the treatment
                            named beside Eq. adjacent; full stationary solve, Eq. steady-state)

Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1311_4627_gb300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
J_STRIDE = 8
DISCRETE_GRAINS = (0, 7)


def exact_values():
    wl = W.single_cell()
    P, j, led, st = oracle.solve_batch(wl, oracle.grain_cooling(wl), want_ledger=True, n_threads=1)
    assert st == oracle.OK
    return P[0], j[0][:, ::J_STRIDE], led[0]


def discrete_values():
    wl = W.grain_subset(W.single_cell(), list(DISCRETE_GRAINS))
    P, _, _, st = oracle.solve_batch_discrete(wl, want_j=False, n_threads=1)
    assert st == oracle.OK
    return P[0]


def _write(path, header, blocks):
    with open(path, "w") as f:
        for line in header.strip().splitlines():
            f.write("# " + line + "\n")
        for name, arr in blocks:
            arr = np.asarray(arr, dtype=np.float64).ravel()
            f.write(f"{name} {arr.size}\n")
            for v in arr:
                f.write(f"{v:.17e}\n")


def read(path):
    """{name: array} of a fixture file."""
    out, name, vals, n = {}, None, [], 0
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                continue
            parts = line.split()
            if len(parts) == 2:
                name, n, vals = parts[0], int(parts[1]), []
                out[name] = vals
            else:
                vals.append(float(parts[0]))
    return {k: np.array(v) for k, v in out.items()}


def main():
    P, j, led = exact_values()
    _write(os.path.join(HERE, "single_cell_exact.txt"),
           "FP64 oracle, single-cell workload (seeded): 1 cell x 8 carbonaceous grains (3.5-250 A), 128 bins,\n"
           "256 wavelengths.  P: all grains back to back (Eq. xf, renormalised); j: each grain at every 8th\n"
           "wavelength, erg s^-1 sr^-1 cm^-1 per grain (Eq. emission); ledger: [absorbed, emitted] per grain.\n"
           "Written by tests/golden/make_golden.py, which calls only oracle/.",
           [("P", P), ("j_every8", j), ("ledger", led)])
    Pd = discrete_values()
    _write(os.path.join(HERE, "single_cell_discrete.txt"),
           "FP64 oracle, single-cell workload, grains 0 and 7 (3.5 and 250 A), thermal-discrete cooling:\n"
           "P of the full stationary solve (Eq. steady-state, Eq. level-sum), both grains back to back.\n"
           "Written by tests/golden/make_golden.py, which calls only oracle/.",
           [("P", Pd)])


if __name__ == "__main__":
    main()
