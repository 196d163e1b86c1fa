"""The stored oracle SVD of the complex 4096 x 2048 workload
(tests/golden/c3_oracle_4096x2048.npz) against what the workload's
construction fixes, A = Q1 diag(s) Q2^H with s prescribed: the oracle's
singular values within 64 n eps of s, unit-norm sampled singular vectors;
and the helper that measures another SVD against it."""
import numpy as np
import pytest

from paper_2202_08361_gb300 import workloads
from tests.golden import c3_fixture

EPS = np.finfo(np.float64).eps


def test_stored_oracle_result_against_the_prescribed_spectrum():
    fx = c3_fixture.load()
    if fx is None:
        pytest.skip("c3_oracle_4096x2048.npz not written yet")
    n = 2048
    s = workloads.geometric_sigma(n, 1e6)
    assert fx["sigma"].shape == (n,) and np.all(np.diff(fx["sigma"]) <= 0)
    assert np.abs(fx["sigma"] - s).max() <= 64 * n * EPS * s[0]
    assert np.allclose(np.ldexp(fx["sigma_f"], fx["sigma_e"].astype(int)), fx["sigma"], rtol=0,
                       atol=0)
    for X in (fx["U_cols"], fx["V_cols"]):
        assert np.abs(np.linalg.norm(X, axis=0) - 1).max() <= 64 * n * EPS
    assert int(fx["sweeps"]) > 0


def test_error_helper_ignores_the_free_phase_and_sees_a_change():
    g = np.random.default_rng(2)
    m, n = 12, 6
    so = np.sort(g.uniform(1, 2, n))[::-1]
    cols = np.array([0, 3, 5])
    Uo = g.standard_normal((m, 3)) + 1j * g.standard_normal((m, 3))
    Vo = g.standard_normal((n, 3)) + 1j * g.standard_normal((n, 3))
    fx = {"sigma": so, "cols": cols, "U_cols": Uo, "V_cols": Vo}
    ph = np.exp(1j * np.array([0.3, -2.0, 1.1]))
    e = c3_fixture.errors(so, Uo * ph, Vo * ph, fx)
    assert e["sigma_max_err_normwise"] == 0
    assert e["U_cols_max_err"] < 1e-14 and e["V_cols_max_err"] < 1e-14
    V2 = Vo * ph
    V2[0, 1] += 1e-6
    e = c3_fixture.errors(so * (1 + 1e-9), Uo * ph, V2, fx)
    assert abs(e["V_col_err"][1] - 1e-6) < 1e-9 and e["sigma_max_err_relative"] > 0.9e-9
