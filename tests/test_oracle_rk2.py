"""Pins of the oracle's time stepping (the second-order TVD Runge-Kutta
scheme of Section 4 around the FP64 operator): second-order convergence to
an independent high-order integrator (scipy's DOP853), exact mass
conservation for any data, and stationarity of a uniform field."""
import numpy as np
import pytest

import oracle


def _field(N, seed):
    return np.random.default_rng(seed).uniform(0.2, 1.0, (N, N))


def test_second_order_against_dop853():
    """Halving dt divides the error against a converged DOP853 solution by
    about 4 (a first-order slip, e.g. reusing Q(f) in the second stage,
    gives 2)."""
    scipy_integrate = pytest.importorskip("scipy.integrate")
    N, L, Nbar, T = 8, 4.0, 1, 0.06
    f0 = _field(N, 3)
    rhs = lambda t, y: oracle.q(y.reshape(N, N), L, Nbar)["Q"].ravel()
    ref = scipy_integrate.solve_ivp(rhs, (0.0, T), f0.ravel(), method="DOP853", rtol=1e-13, atol=1e-15).y[:, -1]
    errs = []
    for n in (8, 16, 32):
        errs.append(np.max(np.abs(oracle.rk2(f0, L, Nbar, T / n, n).ravel() - ref)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.4 < r1 < 4.6 and 3.4 < r2 < 4.6, (errs, r1, r2)
    assert errs[-1] < 1e-4 * np.max(np.abs(f0))


@pytest.mark.parametrize("d,N,Nbar", [(2, 16, 3), (2, 12, 8), (3, 8, 1)])
def test_mass_conserved(d, N, Nbar):
    """Sum Q = 0 for any data on the torus (Section 2.3), so each stage keeps
    the discrete mass."""
    f0 = np.random.default_rng(N + d).uniform(0.0, 1.0, (N,) * d)
    f = oracle.rk2(f0, 4.0, Nbar, 0.01, 4, kernel="hp")
    assert abs(f.sum() - f0.sum()) <= 1e-13 * f0.sum()
    assert not np.allclose(f, f0)


def test_uniform_field_is_stationary():
    """Every term f_{i+k} f_{i+l} - f_i f_{i+k+l} vanishes for a constant f."""
    f0 = np.full((12, 12), 0.37)
    assert np.array_equal(oracle.rk2(f0, 4.0, 8, 0.1, 3), f0)


def test_zero_steps_is_identity_and_one_step_by_hand():
    rng = np.random.default_rng(5)
    f0 = rng.uniform(0.1, 1.0, (10, 10))
    assert np.array_equal(oracle.rk2(f0, 4.0, 2, 0.05, 0), f0)
    dt = 0.02
    q0 = oracle.q(f0, 4.0, 2)["Q"]
    f1 = f0 + dt * q0
    heun = f0 + 0.5 * dt * (q0 + oracle.q(f1, 4.0, 2)["Q"])
    assert np.allclose(oracle.rk2(f0, 4.0, 2, dt, 1), heun, rtol=0, atol=1e-14)
