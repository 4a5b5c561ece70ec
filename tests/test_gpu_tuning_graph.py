"""Launch-parameter variants, the autotuner and CUDA-graph replay: every
variant must stay within the parity bars (and bit-exact on integer data)."""
import itertools

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32_kahan": 1e-5}
TUNINGS_2D = list(itertools.product((256, 512), (0, 1, 2)))


@pytest.fixture(scope="module")
def q():
    import paper_1201_3986_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _batch(torch, b, Ns, prec):
    cp = torch.tensor([Ns.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float64 if prec == "f64" else torch.float32, device="cuda")
    return cp, co, f


@pytest.mark.parametrize("threads,direct_j", TUNINGS_2D)
@pytest.mark.parametrize("prec", ["f64", "f32_kahan"])
def test_batched_2d_every_tuning(q, torch, threads, direct_j, prec):
    Ns = (16, 20, 32, 40, 48, 64)
    b = synth.batch_2d(18, Ns=Ns, L=8.0, seed=31)
    plans = [q.Plan(2, n, 8, 8.0, kernel="hp") for n in Ns]
    for p in plans:
        p.set_tuning(threads=threads, direct_j=direct_j)
    cp, co, f = _batch(torch, b, Ns, prec)
    Q, _ = q.qdvm_eval_batched(plans, cp, co, f, prec)
    Qn = Q.cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        r = oracle.q(b.cell(c, fin), 8.0, 8, kernel="hp")
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= TOL[prec]


@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
@pytest.mark.parametrize("kernel", ["unit", "hp"])
@pytest.mark.parametrize("fft", [1, 2])
def test_fft_loss_batched_every_cell(q, torch, threads, prec, kernel, fft):
    """Loss as one on-chip FFT convolution per cell (cells of 16/32/48/64
    points with the default truncation; other sizes keep the direct sums);
    with fft = 2 the same transform also gives the axis window W_(1,0)."""
    Ns = (16, 20, 32, 48, 64)
    b = synth.batch_2d(15, Ns=Ns, L=8.0, seed=41)
    plans = [q.Plan(2, n, 8, 8.0, kernel=kernel) for n in Ns]
    for p in plans:
        p.set_tuning(threads=threads, loss_fft=fft)
    cp, co, f = _batch(torch, b, Ns, prec)
    Q, M = q.qdvm_eval_batched(plans, cp, co, f, prec)
    Qn = Q.cpu().numpy().astype(np.float64)
    Mn = M.cpu().numpy()
    fin = f.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        r = oracle.q(b.cell(c, fin), 8.0, 8, kernel=kernel)
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= TOL[prec]
        h2 = (16.0 / b.Ns[c]) ** 2
        assert abs(Mn[c, 0]) <= (1e-13 if prec == "f64" else 1e-6) * h2 * r["scale"].sum()


@pytest.mark.parametrize("N,Nbar", [(16, 16), (32, 8), (48, 8), (64, 4), (64, 16)])
@pytest.mark.parametrize("prec", ["f64", "f32_kahan"])
@pytest.mark.parametrize("fft", [1, 2])
def test_fft_loss_single_cell(q, torch, N, Nbar, prec, fft):
    f = synth.bkw_2d(N, 8.0) if N == 64 else synth.mixture(2, N, 8.0, np.random.default_rng(N))
    f = f if prec == "f64" else f.astype(np.float32).astype(np.float64)
    plan = q.Plan(2, N, Nbar, 8.0, kernel="hp")
    plan.set_tuning(loss_fft=fft)
    Q = q.qdvm_eval(plan, torch.tensor(f, dtype=torch.float64 if prec == "f64" else torch.float32, device="cuda"),
                    prec).cpu().numpy().astype(np.float64)
    r = oracle.q(f, 8.0, Nbar, kernel="hp")
    assert oracle.rel_linf(Q, r["Q"], r["scale"]) <= TOL[prec]


@pytest.mark.parametrize("threads,direct_j", TUNINGS_2D)
def test_single_2d_every_tuning_integer_exact(q, torch, threads, direct_j):
    for N, Nbar in ((16, 3), (48, 8), (64, 8)):
        f = synth.integer_field(2, N, maxval=2, seed=N + threads + direct_j)
        plan = q.Plan(2, N, Nbar, 4.0, kernel="unit")
        plan.set_tuning(threads=threads, direct_j=direct_j)
        for prec in ("f64", "f32"):
            Q = q.qdvm_eval(plan, torch.tensor(f, dtype=torch.float64 if prec == "f64" else torch.float32,
                                               device="cuda"), prec)
            assert np.array_equal(Q.cpu().numpy().astype(np.float64), oracle.q(f, 4.0, Nbar)["Q"])


def test_tuning_rejects_bad_values(q):
    p = q.Plan(2, 16, 3, 8.0)
    with pytest.raises(q.QdvmError):
        p.set_tuning(threads=128)
    with pytest.raises(q.QdvmError):
        p.set_tuning(direct_j=3)
    with pytest.raises(q.QdvmError):
        p.set_tuning(loss_fft=4)
    with pytest.raises(q.QdvmError):
        p.set_tuning(scan_j=-1)
    assert p.tuning() == {"threads": 256, "direct_j": 2, "line_chunks": 0, "loss_fft": 0,
                          "scan_j": q.QDVM_SCAN_J_DEFAULT}


def test_autotuner_2d_then_parity(q, torch):
    Ns = (16, 32, 48, 64)
    b = synth.batch_2d(600, Ns=Ns, L=8.0, seed=5)
    plans = [q.Plan(2, n, 8, 8.0) for n in Ns]
    cp, co, f = _batch(torch, b, Ns, "f32_kahan")
    best = q.qdvm_tune_batched(plans, cp, co, f, "f32_kahan")
    assert best["threads"] in (256, 512) and best["direct_j"] in (0, 1, 2) and best["loss_fft"] in (0, 1, 2, 3)
    assert 0 <= best["scan_j"] <= 64
    assert plans[0].tuning() == best
    for p in plans:  # per-plan launch parameters, one block size
        t = p.tuning()
        assert t["threads"] == best["threads"] and t["loss_fft"] in (0, 1, 2, 3) and 0 <= t["scan_j"] <= 64
    Q, _ = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan")
    Qn = Q.cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    for c in (0, 1, 2, 3, 599):
        r = oracle.q(b.cell(c, fin), 8.0, 8)
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= 1e-5


@pytest.mark.parametrize("chunks", [1, 2, 3, 7])
def test_engine_line_chunks_3d(q, torch, chunks):
    b = synth.batch_3d(4, N=12, L=6.0, seed=8)
    plan = q.Plan(3, 12, 2, 6.0, kernel="hp")
    plan.set_tuning(line_chunks=chunks)
    cp = torch.zeros(b.n_cells, dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    Q, _ = q.qdvm_eval_batched([plan], cp, co, f, "f32_kahan")
    Qn = Q.cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        r = oracle.q(b.cell(c, fin), 6.0, 2, kernel="hp")
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= 1e-5


def test_autotuner_3d(q, torch):
    b = synth.batch_3d(6, N=16, L=6.0, seed=9)
    plan = q.Plan(3, 16, 3, 6.0, kernel="hp")
    cp = torch.zeros(b.n_cells, dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    ws = torch.empty(4 * q.batched_workspace_bytes([plan], b.n_cells, "f32"), dtype=torch.uint8, device="cuda")
    best = q.qdvm_tune_batched([plan], cp, co, f, "f32", workspace=ws)
    assert best["line_chunks"] >= 0
    Q, _ = q.qdvm_eval_batched([plan], cp, co, f, "f32", workspace=ws)
    r = oracle.q(b.cell(5, f.cpu().numpy().astype(np.float64)), 6.0, 3, kernel="hp")
    assert oracle.rel_linf(b.cell(5, Q.cpu().numpy().astype(np.float64)), r["Q"], r["scale"]) <= 1e-5


@pytest.mark.parametrize("d", [2, 3])
def test_graph_replay_matches_direct_call(q, torch, d):
    if d == 2:
        Ns = (16, 32)
        b = synth.batch_2d(10, Ns=Ns, L=8.0, seed=3)
        plans = [q.Plan(2, n, 8, 8.0) for n in Ns]
    else:
        Ns = (12,)
        b = synth.batch_3d(3, N=12, L=6.0, seed=3)
        plans = [q.Plan(3, 12, 2, 6.0)]
    cp, co, f = _batch(torch, b, Ns, "f32_kahan")
    Qd, Md = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan")
    Q = torch.full_like(f, float("nan"))
    M = torch.full((b.n_cells, d + 2), float("nan"), dtype=torch.float64, device="cuda")
    g = q.BatchedGraph(plans, cp, co, f, Q, M, "f32_kahan")
    for _ in range(3):
        Q.fill_(float("nan"))
        g.launch()
        torch.cuda.synchronize()
        assert torch.equal(Q, Qd) and torch.equal(M, Md)


def test_per_plan_launch_parameters_in_one_batch(q, torch):
    """Each cell of a batched 2D call runs with its own plan's loss_fft and
    scan_j: a batch whose plans carry four different engines (direct loss,
    FFT loss + axis window, SCAN, FFT windows) against the oracle, and each
    cell equal bit for bit to the same cell evaluated in a batch of its own
    plan alone."""
    Ns = (16, 32, 48, 64)
    b = synth.batch_2d(16, Ns=Ns, L=8.0, seed=44)
    plans = [q.Plan(2, n, 8, 8.0) for n in Ns]
    settings = [dict(loss_fft=0, scan_j=0), dict(loss_fft=2, scan_j=0), dict(loss_fft=1, scan_j=3),
                dict(loss_fft=3, scan_j=7)]
    for p, st in zip(plans, settings):
        p.set_tuning(**st)
    cp, co, f = _batch(torch, b, Ns, "f32_kahan")
    Q, _ = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan")
    Qn = Q.cpu().numpy()
    fin = f.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        r = oracle.q(b.cell(c, fin), 8.0, 8)
        assert oracle.rel_linf(b.cell(c, Qn).astype(np.float64), r["Q"], r["scale"]) <= 1e-5
        i = Ns.index(int(b.Ns[c]))
        one = torch.zeros(1, dtype=torch.int32, device="cuda")
        off = torch.zeros(1, dtype=torch.int64, device="cuda")
        fc = torch.tensor(b.cell(c, fin).ravel(), dtype=torch.float32, device="cuda")
        Qc, _ = q.qdvm_eval_batched([plans[i]], one, off, fc, "f32_kahan")
        assert np.array_equal(Qc.cpu().numpy(), b.cell(c, Qn).ravel())
