"""The stored expected values of tests/golden/ against the oracle that wrote them: the
fixtures are the oracle's outputs (the paper prints none), so a change of the oracle's
arithmetic shows here and the fixtures are rewritten deliberately (tests/golden/make_golden.py).
Compared to 1e-12 where the value is above 1e-280 (the C compilers of the two machines that
run these tests may contract the FMAs differently); the fixtures' own invariants as well."""
import os
import sys

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)
import make_golden  # noqa: E402


def _close(got, ref, rtol=1e-12):
    big = np.abs(ref) > 1e-280
    assert np.all(np.abs(got[~big]) <= 1e-270)
    r = np.max(np.abs(got[big] - ref[big]) / np.abs(ref[big]))
    assert r <= rtol, r


def test_exact_fixture_matches_the_oracle():
    d = make_golden.read(os.path.join(HERE, "single_cell_exact.txt"))
    P, j, led = make_golden.exact_values()
    _close(P.ravel(), d["P"])
    _close(j.ravel(), d["j_every8"])
    _close(led.ravel(), d["ledger"])
    Ps = d["P"].reshape(8, 128)
    np.testing.assert_allclose(Ps.sum(axis=1), 1.0, rtol=1e-13)
    lg = d["ledger"].reshape(8, 2)
    np.testing.assert_allclose(lg[:, 1] / lg[:, 0], 1.0, rtol=1e-6)


def test_discrete_fixture_matches_the_oracle():
    d = make_golden.read(os.path.join(HERE, "single_cell_discrete.txt"))
    _close(make_golden.discrete_values().ravel(), d["P"])
    np.testing.assert_allclose(d["P"].reshape(2, 128).sum(axis=1), 1.0, rtol=1e-13)
