"""Pins of the oracle's box-truncated operator D^tr (Section 2.3): exact
conservation of mass, momentum and energy for any data (the property the
paper states for it), and equality with the periodised operator on data
whose collisions never reach the box edge."""
import numpy as np
import pytest

import oracle
import synth


def _axes(d, N, L):
    h = 2.0 * L / N
    return np.meshgrid(*([-L + h * np.arange(N)] * d), indexing="ij")


@pytest.mark.parametrize("d,N,L,Nbar,kernel,Nt", [(2, 16, 8.0, 16, "unit", None), (2, 20, 5.0, 2, "hp", None),
                                                  (2, 24, 6.0, 3, "hp", 5), (3, 10, 4.0, 1, "hp", None),
                                                  (3, 12, 4.0, 2, "unit", 3)])
def test_conserves_mass_momentum_energy_for_any_data(d, N, L, Nbar, kernel, Nt):
    f = np.random.default_rng(N + d).uniform(0.0, 1.0, (N,) * d)
    r = oracle.dtr(f, L, Nbar, kernel=kernel, Ntilde=Nt)
    ax = _axes(d, N, L)
    v2 = sum(v * v for v in ax)
    tot = r["scale"].sum()
    assert abs(r["Q"].sum()) <= 1e-13 * tot
    for v in ax:
        assert abs((r["Q"] * v).sum()) <= 1e-13 * tot * L
    assert abs((r["Q"] * v2).sum()) <= 1e-13 * tot * d * L * L
    # the periodised operator does not conserve momentum or energy for such data
    q = oracle.q(f, L, Nbar, kernel=kernel, Ntilde=Nt)["Q"]
    assert abs((q * v2).sum()) > 1e-6 * tot


@pytest.mark.parametrize("d,N,S", [(2, 32, 1), (2, 48, 2), (3, 20, 1)])
def test_equals_periodised_operator_inside_the_box(d, N, S):
    """Support within S of the centre and S + 2 Ntilde <= N/2 - 1: no
    collision reaches the edge, so both operators take the same terms."""
    Nt = oracle.default_ntilde(N)
    assert S + 2 * Nt <= N // 2 - 1
    f = synth.compact_support(d, N, S, seed=N)
    a = oracle.dtr(f, 5.0, 8, kernel="hp")["Q"]
    b = oracle.q(f, 5.0, 8, kernel="hp")["Q"]
    assert np.allclose(a, b, rtol=0, atol=1e-15 * np.max(np.abs(b)))
    assert np.max(np.abs(b)) > 0
