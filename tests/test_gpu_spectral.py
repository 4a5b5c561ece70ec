"""The pseudo-spectral route of Section 3.1 on the GPU (qdvm_spectral_table,
qdvm_eval_spectral) against the oracle.

* The table beta~(K, L) against ``oracle.spectral_beta``, which sums the
  pairs of eq. (betaKL) one by one (the GPU groups them by line).
* Q through eq. (sysDiff) against the oracle's direct sum of eq. (DR).  The
  Fourier route sums N^d products per mode whose magnitudes exceed the
  result, so its rounding error is bounded by a multiple of
  eps * max_I sum_K |beta~(K, I - K)| |fhat_K| |fhat_{I-K}| (times N^d for
  the inverse transform), computed here from the oracle's table and numpy's
  FFT.  The bars are 64 times that bound, relative to the term scale.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

EPS = {"f64": 2.0 ** -52, "f32": 2.0 ** -23, "f32_kahan": 2.0 ** -23}


@pytest.fixture(scope="module")
def q():
    import paper_1201_3986_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _dt(torch, prec):
    return torch.float64 if prec == "f64" else torch.float32


def _modes(d, N):
    return np.array(np.meshgrid(*([np.arange(N)] * d), indexing="ij")).reshape(d, -1).T


def rounding_bound(bt, f, prec):
    """eps * N^d * max_I sum_K |beta~(K, I-K) fhat_K fhat_{I-K}| (plus the
    rounding of the table itself in FP32), the scale of the Fourier route's
    error in Q."""
    d, N = f.ndim, f.shape[0]
    M = N ** d
    modes = _modes(d, N)
    fh = np.abs(np.fft.fftn(f).ravel() / M)
    tot = 0.0
    for I in range(M):
        Li = np.ravel_multi_index(((modes[I][None, :] - modes) % N).T, (N,) * d)
        tot = max(tot, float(np.sum(np.abs(bt[np.arange(M), Li]) * fh * fh[Li])))
    return EPS[prec] * M * tot


CASES = [  # d, N, Ntilde (None = default), Nbar, kernel
    (2, 16, None, 16, "unit"), (2, 16, None, 2, "hp"), (2, 20, 4, 3, "hp"), (2, 32, None, 8, "unit"),
    (3, 8, 2, 2, "hp"), (3, 10, None, 2, "unit"), (3, 16, None, 3, "hp"),  # 16^3: the largest 3D table
]


@pytest.mark.parametrize("d,N,Nt,Nbar,kernel", CASES)
def test_table_matches_pairwise_sum(q, torch, d, N, Nt, Nbar, kernel):
    L = 8.0 if d == 2 else 6.0
    plan = q.Plan(d, N, Nbar, L, kernel=kernel, Ntilde=Nt)
    ref = oracle.spectral_beta(d, N, L, Nbar, kernel, Nt)
    for prec in ("f64", "f32"):
        tb = q.spectral_table(plan, prec).cpu().numpy().astype(np.float64)
        err = np.max(np.abs(tb - ref)) / np.max(np.abs(ref))
        assert err <= (1e-13 if prec == "f64" else 1e-6), (prec, err)


@pytest.mark.parametrize("d,N,Nt,Nbar,kernel", CASES)
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
def test_spectral_q_matches_direct_sum(q, torch, d, N, Nt, Nbar, kernel, prec):
    L = 8.0 if d == 2 else 6.0
    rng = np.random.default_rng(N + Nbar)
    cells = [synth.mixture(d, N, L, rng) for _ in range(3)]
    if prec != "f64":
        cells = [c.astype(np.float32).astype(np.float64) for c in cells]
    plan = q.Plan(d, N, Nbar, L, kernel=kernel, Ntilde=Nt)
    table = q.spectral_table(plan, prec)
    f = torch.tensor(np.stack(cells), dtype=_dt(torch, prec), device="cuda")
    Q = q.qdvm_eval_spectral(plan, table, f, prec).cpu().numpy().astype(np.float64)
    bt = oracle.spectral_beta(d, N, L, Nbar, kernel, Nt)
    for c, fc in enumerate(cells):
        r = oracle.q(fc, L, Nbar, kernel=kernel, Ntilde=Nt)
        bound = rounding_bound(bt, fc, prec) / np.max(r["scale"])
        assert oracle.rel_linf(Q[c], r["Q"], r["scale"]) <= max(64 * bound, 1e-14)
        assert abs(Q[c].sum()) <= 64 * rounding_bound(bt, fc, prec) * N ** d  # mode 0: mass


@pytest.mark.parametrize("N,Nbar", [(48, 8), (64, 8)])
def test_spectral_q_large_cells_fp64(q, torch, N, Nbar):
    """The batched configuration's largest cells through the Fourier route in
    FP64, against the direct sum with the same rounding bar."""
    L = 8.0
    f = synth.mixture(2, N, L, np.random.default_rng(7))
    plan = q.Plan(2, N, Nbar, L)
    table = q.spectral_table(plan, "f64")
    Q = q.qdvm_eval_spectral(plan, table, torch.tensor(f, device="cuda"), "f64").cpu().numpy()
    r = oracle.q(f, L, Nbar)
    bound = rounding_bound(oracle.spectral_beta(2, N, L, Nbar, "unit", None), f, "f64") / np.max(r["scale"])
    assert oracle.rel_linf(Q, r["Q"], r["scale"]) <= 64 * bound


def test_spectral_rejects_bad_arguments(q, torch):
    with pytest.raises(q.QdvmError):
        q.spectral_table(q.Plan(2, 80, 4, 8.0), "f64")  # N > 64
    with pytest.raises(q.QdvmError):
        q.spectral_table(q.Plan(3, 20, 2, 6.0), "f64")  # 3D N > 16
    plan = q.Plan(2, 16, 3, 8.0)
    table = q.spectral_table(plan, "f64")
    f = torch.zeros((2, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(q.QdvmError):
        q.qdvm_eval_spectral(plan, table, f, "f64", workspace=torch.empty(16, dtype=torch.uint8, device="cuda"))
    assert float(q.qdvm_eval_spectral(plan, table, f, "f64").abs().max()) == 0.0
    empty = torch.zeros((0, 16, 16), dtype=torch.float64, device="cuda")
    assert q.qdvm_eval_spectral(plan, table, empty, "f64").shape == (0, 16, 16)
