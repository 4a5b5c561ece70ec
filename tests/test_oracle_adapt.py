"""Pins of the oracle's equilibrium indicator (the distance of a cell to the
Maxwellian with its own moments), used to choose a per-cell Nbar: a
resolved Maxwellian gives 0, the indicator is scale invariant, and for a
two-Maxwellian mixture it converges to the continuous integral computed by
scipy quadrature (which fixes rho, u and the 1/d in T independently)."""
import numpy as np
import pytest

import oracle


def _maxwellian(d, N, L, rho, u, T):
    h = 2.0 * L / N
    axes = np.meshgrid(*([-L + h * np.arange(N)] * d), indexing="ij")
    w2 = sum((v - x) ** 2 for v, x in zip(axes, u))
    return rho * (2 * np.pi * T) ** (-d / 2) * np.exp(-w2 / (2 * T))


@pytest.mark.parametrize("d,N,L", [(2, 64, 8.0), (3, 32, 7.0)])
def test_resolved_maxwellian_is_at_equilibrium(d, N, L):
    u = (0.4, -0.2, 0.1)[:d]
    f = _maxwellian(d, N, L, 1.3, u, 0.8)
    assert oracle.equilibrium_distance(f, L) < 1e-10
    assert oracle.equilibrium_distance(3.7 * f, L) < 1e-10


def test_scale_invariance_and_undefined_cases():
    f = np.random.default_rng(1).uniform(0.0, 1.0, (24, 24))
    e = oracle.equilibrium_distance(f, 6.0)
    assert 0.1 < e < 2.0
    assert abs(oracle.equilibrium_distance(2.5 * f, 6.0) - e) <= 1e-14 * e
    assert oracle.equilibrium_distance(np.zeros((8, 8)), 4.0) == float("inf")
    assert oracle.equilibrium_distance(-f, 6.0) == float("inf")


def test_two_maxwellians_match_continuous_integral():
    """f = (M(+a e1, T0) + M(-a e1, T0)) / 2: rho = 1, u = 0, T = T0 + a^2/2
    in 2D; the continuous L1 distance to M(0, T) by 2D quadrature."""
    integrate = pytest.importorskip("scipy.integrate")
    a, T0 = 1.2, 0.7
    T = T0 + a * a / 2

    def g(x, y):
        m1 = np.exp(-((x - a) ** 2 + y * y) / (2 * T0)) / (2 * np.pi * T0)
        m2 = np.exp(-((x + a) ** 2 + y * y) / (2 * T0)) / (2 * np.pi * T0)
        return abs(0.5 * (m1 + m2) - np.exp(-(x * x + y * y) / (2 * T)) / (2 * np.pi * T))

    # symmetric in x and y: integrate one quadrant, the mixture integrates to 1
    cont = 4 * integrate.dblquad(g, 0, 12, 0, 12, epsabs=1e-11, epsrel=1e-11)[0]
    N, L = 160, 10.0
    f = 0.5 * (_maxwellian(2, N, L, 1.0, (a, 0.0), T0) + _maxwellian(2, N, L, 1.0, (-a, 0.0), T0))
    disc = oracle.equilibrium_distance(f, L)
    assert abs(disc - cont) <= 2e-3 * cont
    assert cont > 0.05
