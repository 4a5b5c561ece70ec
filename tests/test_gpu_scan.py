"""The running-sum (SCAN) line-sum engine of the on-chip 2D evaluator.

With the loss as one FFT convolution per cell (tuning loss_fft >= 1), each
pair {e, e^perp} with window half-length J >= scan_j sums its windows
W_e, W_{e^perp} (the alpha_p factors of eq. (decDVM)) as running sums along
strips of the lattice lines instead of gathering 2J values per point; the
horizontal window (0,1) is gathered, or with loss_fft = 2 taken from the
loss transform.  The set of terms is the same, so:
  - against the FP64 oracle the bars are those of every other evaluator;
  - on integer data (loss_fft = 1) every window is an exact integer in both
    engines, so SCAN and DIRECT give bit-identical Q (same FFT loss, same
    accumulation order of the same values).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32_kahan": 1e-5}
NS = (16, 32, 48, 64)  # the cell sizes of the on-chip FFT body (default truncation)


@pytest.fixture(scope="module")
def q():
    import paper_1201_3986_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _dtype(torch, prec):
    return torch.float64 if prec == "f64" else torch.float32


def _batch(torch, b, Ns, prec):
    cp = torch.tensor([Ns.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=_dtype(torch, prec), device="cuda")
    return cp, co, f


@pytest.mark.parametrize("scan_j,loss_fft", [(1, 1), (2, 1), (3, 1), (5, 1), (1, 2), (5, 2), (7, 2), (10, 2)])
@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
@pytest.mark.parametrize("kernel", ["unit", "hp"])
def test_batched_scan_matches_oracle(q, torch, scan_j, loss_fft, threads, prec, kernel):
    b = synth.batch_2d(12, Ns=NS, L=8.0, seed=71 + scan_j)
    plans = [q.Plan(2, n, 8, 8.0, kernel=kernel) for n in NS]
    for p in plans:
        p.set_tuning(threads=threads, loss_fft=loss_fft, scan_j=scan_j)
    cp, co, f = _batch(torch, b, NS, prec)
    Q, M = q.qdvm_eval_batched(plans, cp, co, f, prec)
    Qn = Q.cpu().numpy().astype(np.float64)
    Mn = M.cpu().numpy()
    fin = f.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        r = oracle.q(b.cell(c, fin), 8.0, 8, kernel=kernel)
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= TOL[prec]
        h2 = (16.0 / b.Ns[c]) ** 2
        assert abs(Mn[c, 0]) <= (1e-13 if prec == "f64" else 1e-6) * h2 * r["scale"].sum()


@pytest.mark.parametrize("N,Nbar", [(16, 16), (32, 32), (48, 8), (64, 4), (64, 16)])
@pytest.mark.parametrize("prec", ["f64", "f32_kahan"])
def test_single_cell_scan_matches_oracle(q, torch, N, Nbar, prec):
    """One cell through qdvm_eval (FP64: pairs split over CTAs and summed)."""
    f = synth.bkw_2d(N, 8.0) if N == 64 else synth.mixture(2, N, 8.0, np.random.default_rng(N + 5))
    f = f if prec == "f64" else f.astype(np.float32).astype(np.float64)
    plan = q.Plan(2, N, Nbar, 8.0, kernel="hp", engine="scan")
    plan.set_tuning(loss_fft=1)
    Q = q.qdvm_eval(plan, torch.tensor(f, dtype=_dtype(torch, prec), device="cuda"), prec)
    r = oracle.q(f, 8.0, Nbar, kernel="hp")
    assert oracle.rel_linf(Q.cpu().numpy().astype(np.float64), r["Q"], r["scale"]) <= TOL[prec]


@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_scan_bit_identical_to_direct_on_integer_data(q, torch, threads, prec):
    b = synth.batch_2d(8, Ns=NS, L=4.0, seed=3)
    rng = np.random.default_rng(9)
    fi = rng.integers(0, 4, size=b.f.shape).astype(np.float64)
    plans = [q.Plan(2, n, 64, 4.0, kernel="unit") for n in NS]
    cp = torch.tensor([NS.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(fi, dtype=_dtype(torch, prec), device="cuda")
    out = {}
    for sj in (0, 1, 3):
        for p in plans:
            p.set_tuning(threads=threads, loss_fft=1, scan_j=sj)
        Q, _ = q.qdvm_eval_batched(plans, cp, co, f, prec)
        out[sj] = Q.cpu().numpy()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[3])


@pytest.mark.parametrize("scan_j,loss_fft", [(1, 1), (7, 2)])
def test_batched_scan_full_workload_sampled(q, torch, scan_j, loss_fft):
    """The 4096-cell mixed-size batch with N̄ = 8 in FP32 with compensation,
    every pair on the SCAN engine, or the long windows (J >= 7) with the
    axis window from the loss transform; sampled cells against the oracle."""
    b = synth.batch_2d(4096, Ns=NS, L=8.0, seed=0)
    plans = [q.Plan(2, n, 8, 8.0) for n in NS]
    for p in plans:
        p.set_tuning(loss_fft=loss_fft, scan_j=scan_j)
    cp, co, f = _batch(torch, b, NS, "f32_kahan")
    Q, M = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan")
    Qn = Q.cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    for c in (0, 1, 2, 3, 1234, 4095) + tuple(int(i) for i in np.nonzero(np.array(b.Ns) == 64)[0][:3]):
        r = oracle.q(b.cell(c, fin), 8.0, 8)
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= 1e-5


def test_engine_sets_initial_scan_threshold(q):
    assert q.Plan(2, 32, 8, 8.0, engine="direct").tuning()["scan_j"] == 0
    assert q.Plan(2, 32, 8, 8.0, engine="scan").tuning()["scan_j"] == 1
    assert q.Plan(2, 32, 8, 8.0).tuning()["scan_j"] == q.QDVM_SCAN_J_DEFAULT
    p = q.Plan(2, 32, 8, 8.0)
    for bad in (-1, 65):
        with pytest.raises(q.QdvmError):
            p.set_tuning(scan_j=bad)
