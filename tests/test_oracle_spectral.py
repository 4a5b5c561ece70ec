"""Pins for the oracle's pseudo-spectral form (Section 3.1), CPU only.

``oracle.spectral_beta`` sums the kernel modes beta(K, L) of eq. (betaKL)
pair by pair, and ``oracle.q_spectral`` evaluates eq. (sysDiff) with numpy's
FFT.  They are tied to things other than themselves:

* Q through eq. (sysDiff) equals the C oracle's direct sum of eq. (DR)
  (a different route: physical space, term by term, compensated);
* beta~(K, -K) = 0 for every K: beta is even in each argument, so the mode
  K = 0 of Q vanishes for every f (conservation of mass, Proposition 3.2);
* beta(0, 0) is the total weight of the terms, for the unit kernel the
  number of (k, l) pairs, counted independently by the C oracle;
* the rank of beta is at most the number of lines of A_m (eq. (decDVM)
  writes it as a sum of one outer product per line).
"""
import numpy as np
import pytest

import oracle


def rng_f(shape, seed):
    return np.random.default_rng(seed).uniform(0.1, 1.0, size=shape)


@pytest.mark.parametrize("d,N,Nt,Nbar,kernel", [
    (2, 8, 2, 2, "unit"), (2, 9, 2, 1, "hp"), (2, 12, 3, 3, "hp"), (2, 12, 3, 2, "unit"),
    (3, 5, 1, 1, "unit"), (3, 6, 2, 2, "hp"),
])
def test_spectral_route_equals_direct_sum(d, N, Nt, Nbar, kernel):
    f = rng_f((N,) * d, seed=N + Nt + Nbar)
    L = 3.0
    ref = oracle.q(f, L, Nbar, kernel=kernel, Ntilde=Nt)
    Q = oracle.q_spectral(f, L, Nbar, kernel=kernel, Ntilde=Nt)
    assert oracle.rel_linf(Q, ref["Q"], ref["scale"]) < 1e-12


@pytest.mark.parametrize("d,N,Nt,Nbar,kernel", [(2, 10, 3, 3, "unit"), (2, 16, 3, 2, "hp"), (3, 6, 2, 2, "unit")])
def test_beta_tilde_vanishes_on_the_antidiagonal(d, N, Nt, Nbar, kernel):
    bt = oracle.spectral_beta(d, N, 2.0, Nbar, kernel, Nt)
    M = N ** d
    modes = np.array(np.meshgrid(*([np.arange(N)] * d), indexing="ij")).reshape(d, -1).T
    neg = np.ravel_multi_index(((-modes) % N).T, (N,) * d)
    assert np.max(np.abs(bt[np.arange(M), neg])) <= 1e-12 * np.max(np.abs(bt))


@pytest.mark.parametrize("d,N,Nt,Nbar", [(2, 10, 3, 3), (2, 12, 3, 1), (3, 6, 2, 2)])
def test_beta_at_zero_counts_the_terms_and_rank_is_the_line_count(d, N, Nt, Nbar):
    """sum_K beta~(K, 0) = sum_K beta(K, 0) - N^d beta(0, 0).  The first sum
    is N^d times the weight of the pairs with k = 0 mod N, none since
    0 < |k|_inf <= Ntilde < N/2; beta(0, 0) is the total weight, for the
    unit kernel the number of pairs.  And beta is a sum of one outer product
    per line (eq. (decDVM)), so rank(beta~) <= #lines + 1."""
    bt = oracle.spectral_beta(d, N, 2.0, Nbar, "unit", Nt)
    n_terms = oracle.terms_count(d, Nt, min(Nbar, Nt))
    M = N ** d
    assert abs(bt[:, 0].sum() + M * n_terms) <= 1e-9 * M * n_terms
    assert np.linalg.matrix_rank(bt) <= len(oracle.lines(d, min(Nbar, Nt))) + 1
