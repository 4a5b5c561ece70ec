"""The FFT window engine of the on-chip 2D evaluator (tuning loss_fft = 3).

The cell's spectrum fhat stays on chip; each pair {e, e^perp} with window
half-length J >= scan_j takes one inverse transform of
fhat (D_J(e.xi) + i D_J(e^perp.xi)), whose real and imaginary parts are the
windows W_e and W_{e^perp} (the alpha_p and alpha'_p factors of eq. (decDVM),
each a convolution of f with the line's window, Section 3.2); the loss takes
one inverse transform of fhat Ktilde, and the other pairs gather directly.
The set of terms is unchanged, so the bars are those of every evaluator:
1e-12 of the largest sum of absolute terms in FP64, 1e-5 in FP32.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32_kahan": 1e-5}
NS = (16, 32, 48, 64)


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


@pytest.mark.parametrize("fft_j", [1, 3, 7, 10, 14])
@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
@pytest.mark.parametrize("kernel", ["unit", "hp"])
def test_batched_fft_windows_match_oracle(q, torch, fft_j, threads, prec, kernel):
    b = synth.batch_2d(12, Ns=NS, L=8.0, seed=91 + fft_j)
    plans = [q.Plan(2, n, 8, 8.0, kernel=kernel) for n in NS]
    for p in plans:
        p.set_tuning(threads=threads, loss_fft=3, scan_j=fft_j)
    cp = torch.tensor([NS.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=_dtype(torch, prec), device="cuda")
    Q, M = q.qdvm_eval_batched(plans, cp, co, f, prec)
    Qn = Q.cpu().numpy().astype(np.float64)
    Mn = M.cpu().numpy()
    fin = f.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        r = oracle.q(b.cell(c, fin), 8.0, 8, kernel=kernel)
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= TOL[prec], f"cell {c} (N={b.Ns[c]})"
        h2 = (16.0 / b.Ns[c]) ** 2
        assert abs(Mn[c, 0]) <= (1e-13 if prec == "f64" else 1e-6) * h2 * r["scale"].sum()


@pytest.mark.parametrize("N,Nbar,fft_j", [(16, 16, 1), (32, 32, 2), (48, 8, 5), (64, 4, 7), (64, 16, 1)])
@pytest.mark.parametrize("prec", ["f64", "f32_kahan"])
def test_single_cell_fft_windows(q, torch, N, Nbar, fft_j, prec):
    """One cell through qdvm_eval: in FP64 the pairs are split over CTAs, each
    CTA transforming the cell for its own FFT pairs, and summed."""
    f = synth.bkw_2d(N, 8.0) if N == 64 else synth.mixture(2, N, 8.0, np.random.default_rng(N + 9))
    f = f if prec == "f64" else f.astype(np.float32).astype(np.float64)
    plan = q.Plan(2, N, Nbar, 8.0, kernel="hp")
    plan.set_tuning(loss_fft=3, scan_j=fft_j)
    Q = q.qdvm_eval(plan, torch.tensor(f, dtype=_dtype(torch, prec), device="cuda"), prec)
    r = oracle.q(f, 8.0, Nbar, kernel="hp")
    assert oracle.rel_linf(Q.cpu().numpy().astype(np.float64), r["Q"], r["scale"]) <= TOL[prec]


@pytest.mark.parametrize("fft_j", [7, 14])
def test_batched_fft_windows_full_workload_sampled(q, torch, fft_j):
    """The 4096-cell mixed-size batch (N̄ = 8, FP32 with compensation) with
    the long windows from the FFT engine: sampled cells of every size against
    the oracle, the mass defect on every cell."""
    b = synth.batch_2d(4096, Ns=NS, L=8.0, seed=0)
    plans = [q.Plan(2, n, 8, 8.0) for n in NS]
    for p in plans:
        p.set_tuning(loss_fft=3, scan_j=fft_j)
    cp = torch.tensor([NS.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    Q, M = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan")
    Qn = Q.cpu().numpy().astype(np.float64)
    Mn = M.cpu().numpy()
    fin = f.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(fft_j)
    for n in NS:
        for c in rng.choice(np.nonzero(b.Ns == n)[0], size=2, replace=False):
            r = oracle.q(b.cell(int(c), fin), 8.0, 8)
            assert oracle.rel_linf(b.cell(int(c), Qn), r["Q"], r["scale"]) <= 1e-5
    from test_gpu_eval2d import displacement_histogram, total_scale

    hist = {n: displacement_histogram(n, 8) for n in NS}
    for c in range(b.n_cells):
        fc = b.cell(c, fin)
        h2 = (16.0 / fc.shape[0]) ** 2
        assert abs(Mn[c, 0]) <= 1e-6 * h2 * total_scale(fc, hist[fc.shape[0]])


def test_fft_windows_zero_threshold_is_direct(q, torch):
    """scan_j = 0 with loss_fft = 3 gathers every window directly (the loss
    still from the stored spectrum): both launches within the FP64 bar."""
    b = synth.batch_2d(8, Ns=NS, L=8.0, seed=5)
    plans = [q.Plan(2, n, 8, 8.0) for n in NS]
    cp = torch.tensor([NS.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float64, device="cuda")
    out = []
    for fft in (1, 3):
        for p in plans:
            p.set_tuning(loss_fft=fft, scan_j=0)
        Q, _ = q.qdvm_eval_batched(plans, cp, co, f, "f64")
        out.append(Q.cpu().numpy())
    fin = f.cpu().numpy()
    for c in range(b.n_cells):
        r = oracle.q(b.cell(c, fin), 8.0, 8)
        for o in out:
            assert oracle.rel_linf(b.cell(c, o), r["Q"], r["scale"]) <= 1e-12
