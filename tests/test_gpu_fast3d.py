"""GPU parity of the 3D evaluator that takes the loss as one FFT convolution
per cell (tuning loss_fft = 1; plans sharing N in {16, 32}) against the CPU
oracle, plus the fall-back to the line engine where it does not apply."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32_kahan": 1e-5}


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


def _sample_idx(N, n, seed):
    rng = np.random.default_rng(seed)
    idx = rng.choice(N ** 3, size=n, replace=False)
    extra = [0, N - 1, N * N - 1, N ** 3 - 1, (N // 2) * (N * N + N + 1)]
    return np.unique(np.concatenate([idx, extra])).astype(np.int64)


def _run_batch(q, torch, b, plans, prec, chunks=0):
    for p in plans:
        p.set_tuning(loss_fft=1, line_chunks=chunks)
    cp = torch.zeros(b.n_cells, dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=_dt(torch, prec), device="cuda")
    Q, mom = q.qdvm_eval_batched(plans, cp, co, f, prec)
    return Q.cpu().numpy().astype(np.float64), mom.cpu().numpy(), f.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("chunks", [0, 1, 3])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
@pytest.mark.parametrize("kernel", ["unit", "hp"])
def test_batched_N16_every_cell(q, torch, chunks, prec, kernel):
    b = synth.batch_3d(5, N=16, L=6.0, seed=12)
    Qn, mom, fin = _run_batch(q, torch, b, [q.Plan(3, 16, 3, 6.0, kernel=kernel)], prec, chunks)
    for c in range(b.n_cells):
        r = oracle.q(b.cell(c, fin), 6.0, 3, kernel=kernel)
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= TOL[prec]
        # mass: the loss convolution and the gain sums cancel to rounding
        h3 = (12.0 / 16) ** 3
        assert abs(mom[c, 0]) <= (1e-13 if prec == "f64" else 1e-6) * h3 * r["scale"].sum()


@pytest.mark.parametrize("Nt,Nbar", [(2, 2), (5, 4), (7, 7)])
def test_batched_N16_other_truncations(q, torch, Nt, Nbar):
    """The halo follows the plan's Ntilde (any 2 Ntilde < N)."""
    b = synth.batch_3d(3, N=16, L=6.0, seed=Nt)
    for prec in ("f64", "f32_kahan"):
        Qn, _, fin = _run_batch(q, torch, b, [q.Plan(3, 16, Nbar, 6.0, kernel="hp", Ntilde=Nt)], prec)
        for c in range(b.n_cells):
            r = oracle.q(b.cell(c, fin), 6.0, Nbar, kernel="hp", Ntilde=Nt)
            assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= TOL[prec]


@pytest.mark.parametrize("Nbar", [3, 5, 7])
@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_batched_N32_sampled(q, torch, Nbar, prec):
    """32^3 cells, hard spheres, Ntilde = 7: sampled points of every cell."""
    b = synth.batch_3d(4, N=32, L=6.0, seed=Nbar)
    Qn, mom, fin = _run_batch(q, torch, b, [q.Plan(3, 32, Nbar, 6.0, kernel="hp")], prec)
    assert np.all(np.isfinite(Qn))
    for c in range(b.n_cells):
        idx = _sample_idx(32, 40, 10 * Nbar + c)
        r = oracle.q_points(b.cell(c, fin), 6.0, Nbar, idx, kernel="hp")
        err = np.max(np.abs(b.cell(c, Qn).ravel()[idx] - r["Q"])) / np.max(r["scale"])
        assert err <= 1e-5, f"cell {c}: {err:.3e}"


def test_single_cell_trimaxwellian_N32(q, torch):
    f = synth.trimaxwellian_3d(32, 6.0).astype(np.float32).astype(np.float64)
    plan = q.Plan(3, 32, 5, 6.0, kernel="hp")
    plan.set_tuning(loss_fft=1)
    Q = q.qdvm_eval(plan, torch.tensor(f, dtype=torch.float32, device="cuda"), "f32_kahan").cpu().numpy()
    idx = _sample_idx(32, 120, 3)
    r = oracle.q_points(f, 6.0, 5, idx, kernel="hp")
    assert np.max(np.abs(Q.astype(np.float64).ravel()[idx] - r["Q"])) / np.max(r["scale"]) <= 1e-5


@pytest.mark.parametrize("prec", ["f64", "f32_kahan"])
def test_single_cell_N16_full(q, torch, prec):
    f = synth.mixture(3, 16, 6.0, np.random.default_rng(21))
    f = f if prec == "f64" else f.astype(np.float32).astype(np.float64)
    plan = q.Plan(3, 16, 3, 6.0, kernel="hp")
    plan.set_tuning(loss_fft=1)
    Q = q.qdvm_eval(plan, torch.tensor(f, dtype=_dt(torch, prec), device="cuda"), prec).cpu().numpy()
    r = oracle.q(f, 6.0, 3, kernel="hp")
    assert oracle.rel_linf(Q.astype(np.float64), r["Q"], r["scale"]) <= TOL[prec]


def test_fallbacks_fp64_N32_and_mixed_sizes(q, torch):
    """FP64 32^3 does not fit on chip and a batch mixing 12^3 and 16^3 has no
    common N: both run the line engine with loss_fft = 1 set."""
    b = synth.batch_3d(2, N=32, L=6.0, seed=2)
    Qn, _, fin = _run_batch(q, torch, b, [q.Plan(3, 32, 3, 6.0, kernel="hp")], "f64")
    idx = _sample_idx(32, 40, 9)
    r = oracle.q_points(b.cell(1, fin), 6.0, 3, idx, kernel="hp")
    assert np.max(np.abs(b.cell(1, Qn).ravel()[idx] - r["Q"])) / np.max(r["scale"]) <= 1e-12

    b1 = synth.batch_3d(2, N=12, L=6.0, seed=4)
    b2 = synth.batch_3d(2, N=16, L=6.0, seed=5)
    bb = synth.Batch(3, 6.0, np.concatenate([b1.Ns, b2.Ns]), np.concatenate([b1.f, b2.f]))
    plans = [q.Plan(3, 12, 2, 6.0), q.Plan(3, 16, 3, 6.0)]
    for p in plans:
        p.set_tuning(loss_fft=1)
    cp = torch.tensor([0, 0, 1, 1], dtype=torch.int32, device="cuda")
    co = torch.tensor(bb.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(bb.f, dtype=torch.float32, device="cuda")
    Q, _ = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan")
    Qn = Q.cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    for c in range(4):
        r = oracle.q(bb.cell(c, fin), 6.0, 2 if c < 2 else 3)
        assert oracle.rel_linf(bb.cell(c, Qn), r["Q"], r["scale"]) <= 1e-5


def test_autotuner_considers_fft_loss_and_graph_replay(q, torch):
    b = synth.batch_3d(40, N=16, L=6.0, seed=17)
    plan = q.Plan(3, 16, 3, 6.0, kernel="hp")
    cp = torch.zeros(b.n_cells, dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    plan.set_tuning(loss_fft=1)
    ws_fft = q.batched_workspace_bytes([plan], b.n_cells, "f32_kahan")
    plan.set_tuning(loss_fft=0)
    ws_eng = q.batched_workspace_bytes([plan], b.n_cells, "f32_kahan")
    ws = torch.empty(8 * max(ws_fft, ws_eng), dtype=torch.uint8, device="cuda")
    best = q.qdvm_tune_batched([plan], cp, co, f, "f32_kahan", workspace=ws)
    assert best["loss_fft"] in (0, 1) and plan.tuning() == best
    plan.set_tuning(loss_fft=1, line_chunks=2)
    Qd, Md = q.qdvm_eval_batched([plan], cp, co, f, "f32_kahan")
    Q = torch.full_like(f, float("nan"))
    M = torch.full((b.n_cells, 5), float("nan"), dtype=torch.float64, device="cuda")
    g = q.BatchedGraph([plan], cp, co, f, Q, M, "f32_kahan")
    for _ in range(2):
        Q.fill_(float("nan"))
        g.launch()
        torch.cuda.synchronize()
        assert torch.equal(Q, Qd) and torch.equal(M, Md)
    Qn = Qd.cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    for c in (0, 39):
        r = oracle.q(b.cell(c, fin), 6.0, 3, kernel="hp")
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= 1e-5


@pytest.mark.parametrize("N,Nbar,Nt", [(16, 3, None), (16, 7, 7), (32, 3, None), (32, 5, None), (32, 7, None)])
def test_row_tables_present(q, N, Nbar, Nt):
    """3D plans with N in {16, 32} and Ntilde <= 7 carry the row form of the
    plane polygons; the rows cover every polygon point (sum of row lengths =
    sum of plane sizes is checked through parity elsewhere)."""
    p = q.Plan(3, N, Nbar, 6.0, kernel="hp", Ntilde=Nt)
    nc, nr = p.row_info()
    assert 1 <= nc <= p.n_lines and nr >= p.n_lines
    assert q.Plan(2, 32, 8, 6.0).row_info() == (0, 0)
    assert q.Plan(3, 12, 2, 6.0).row_info() == (0, 0)
    assert q.Plan(3, 32, 3, 6.0, Ntilde=9).row_info() == (0, 0)


@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_point_sum_form_N32_wide_truncation(q, torch, prec):
    """Ntilde = 9 > 7 has no row tables: the FFT-loss evaluator sums the plane
    polygons point by point."""
    f = synth.trimaxwellian_3d(32, 6.0).astype(np.float32).astype(np.float64)
    plan = q.Plan(3, 32, 3, 6.0, kernel="hp", Ntilde=9)
    plan.set_tuning(loss_fft=1)
    Q = q.qdvm_eval(plan, torch.tensor(f, dtype=torch.float32, device="cuda"), prec).cpu().numpy()
    idx = _sample_idx(32, 64, 7)
    r = oracle.q_points(f, 6.0, 3, idx, kernel="hp", Ntilde=9)
    assert np.max(np.abs(Q.astype(np.float64).ravel()[idx] - r["Q"])) / np.max(r["scale"]) <= 1e-5


def test_integer_data_row_form_close(q, torch):
    """Integer data: the gain sums are exact integers in the row form, the FFT
    loss is within rounding of the integer loss."""
    f = synth.integer_field(3, 16, maxval=2, seed=3)
    plan = q.Plan(3, 16, 3, 4.0, kernel="unit")
    plan.set_tuning(loss_fft=1)
    Q = q.qdvm_eval(plan, torch.tensor(f, dtype=torch.float64, device="cuda"), "f64").cpu().numpy()
    r = oracle.q(f, 4.0, 3)
    assert np.max(np.abs(Q - r["Q"])) <= 1e-9 * np.max(r["scale"])


def _jvp_batch(q, torch, b, a, plan, prec, chunks):
    plan.set_tuning(loss_fft=1, line_chunks=chunks)
    cp = torch.zeros(b.n_cells, dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=_dt(torch, prec), device="cuda")
    d = torch.tensor(a, dtype=_dt(torch, prec), device="cuda")
    J = q.qdvm_jvp_batched([plan], cp, co, f, d, prec)
    return (J.cpu().numpy().astype(np.float64), f.cpu().numpy().astype(np.float64),
            d.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("chunks", [0, 1, 3])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
@pytest.mark.parametrize("kernel", ["unit", "hp"])
def test_jvp_row_form_N16_every_cell(q, torch, chunks, prec, kernel):
    """JVP with the loss -d (K * f) - f (K * d) from one complex FFT and the
    gain in two row-form passes (rows of f with windows of d, then rows of d
    with windows of f)."""
    b = synth.batch_3d(3, N=16, L=6.0, seed=30)
    a = synth.gaussian(b.f.shape, seed=31)
    J, fin, din = _jvp_batch(q, torch, b, a, q.Plan(3, 16, 3, 6.0, kernel=kernel), prec, chunks)
    for c in range(b.n_cells):
        r, sc = oracle.jvp_points(b.cell(c, fin), b.cell(c, din), 6.0, 3, kernel=kernel)
        assert np.max(np.abs(b.cell(c, J) - r)) / np.max(sc) <= TOL[prec]


@pytest.mark.parametrize("Nbar", [3, 5])
def test_jvp_row_form_N32_sampled(q, torch, Nbar):
    b = synth.batch_3d(3, N=32, L=6.0, seed=40 + Nbar)
    a = synth.gaussian(b.f.shape, seed=Nbar)
    for prec in ("f32", "f32_kahan"):
        J, fin, din = _jvp_batch(q, torch, b, a, q.Plan(3, 32, Nbar, 6.0, kernel="hp"), prec, 0)
        for c in range(b.n_cells):
            idx = _sample_idx(32, 40, c + Nbar)
            r, sc = oracle.jvp_points(b.cell(c, fin), b.cell(c, din), 6.0, Nbar, idx, kernel="hp")
            assert np.max(np.abs(b.cell(c, J).ravel()[idx] - r)) / np.max(sc) <= 1e-5


def test_jvp_row_form_single_cell_and_transpose(q, torch):
    """Single-cell JVP through the row form against the oracle, and
    <g, J d> = <J^T g, d> with the VJP (line engine)."""
    rs = np.random.default_rng(8)
    f = synth.mixture(3, 16, 6.0, rs)
    d = rs.standard_normal((16,) * 3)
    g = rs.standard_normal((16,) * 3)
    plan = q.Plan(3, 16, 3, 6.0, kernel="hp")
    plan.set_tuning(loss_fft=1)
    tf = lambda x: torch.tensor(x, dtype=torch.float64, device="cuda")
    J = q.qdvm_jvp(plan, tf(f), tf(d), "f64").cpu().numpy()
    G = q.qdvm_vjp(plan, tf(f), tf(g), "f64").cpu().numpy()
    r, sc = oracle.jvp_points(f, d, 6.0, 3, kernel="hp")
    assert np.max(np.abs(J - r)) / np.max(sc) <= 1e-12
    lhs, rhs = float(np.sum(g * J)), float(np.sum(G * d))
    assert abs(lhs - rhs) <= 1e-11 * (np.sum(np.abs(g)) * np.max(sc))


def _vjp_batch(q, torch, b, a, plan, prec, chunks):
    plan.set_tuning(loss_fft=1, line_chunks=chunks)
    cp = torch.zeros(b.n_cells, dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=_dt(torch, prec), device="cuda")
    g = torch.tensor(a, dtype=_dt(torch, prec), device="cuda")
    G = q.qdvm_vjp_batched([plan], cp, co, f, g, prec)
    return (G.cpu().numpy().astype(np.float64), f.cpu().numpy().astype(np.float64),
            g.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("chunks", [0, 1, 3])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
@pytest.mark.parametrize("kernel", ["unit", "hp"])
def test_vjp_row_form_N16_every_cell(q, torch, chunks, prec, kernel):
    """VJP: loss -[g (K * f) + K * (g f)] from one complex FFT; gain
    Omega_e(g P_e f) + Pi_e(g W_e f) with the per-line products materialised
    (windows of X = g P in global scratch, rows of Y = g W in shared memory)."""
    b = synth.batch_3d(3, N=16, L=6.0, seed=50)
    a = synth.gaussian(b.f.shape, seed=51)
    G, fin, gin = _vjp_batch(q, torch, b, a, q.Plan(3, 16, 3, 6.0, kernel=kernel), prec, chunks)
    for c in range(b.n_cells):
        r, sc = oracle.vjp(b.cell(c, fin), b.cell(c, gin), 6.0, 3, kernel=kernel, with_scale=True)
        assert np.max(np.abs(b.cell(c, G) - r)) / np.max(sc) <= TOL[prec]


@pytest.mark.parametrize("Nbar", [3, 5])
def test_vjp_row_form_N32_sampled(q, torch, Nbar):
    b = synth.batch_3d(2, N=32, L=6.0, seed=60 + Nbar)
    a = synth.gaussian(b.f.shape, seed=Nbar + 1)
    for prec in ("f32", "f32_kahan"):
        G, fin, gin = _vjp_batch(q, torch, b, a, q.Plan(3, 32, Nbar, 6.0, kernel="hp"), prec, 0)
        for c in range(b.n_cells):
            idx = _sample_idx(32, 32, c + 3 * Nbar)
            r, sc = oracle.vjp_points(b.cell(c, fin), b.cell(c, gin), 6.0, Nbar, idx, kernel="hp")
            assert np.max(np.abs(b.cell(c, G).ravel()[idx] - r)) / np.max(sc) <= 1e-5


@pytest.mark.parametrize("Nt,Nbar", [(7, 7), (5, 4)])
def test_jvp_vjp_transpose_row_form_N16(q, torch, Nt, Nbar):
    """<g, J d> = <J^T g, d> with both derivatives in row form, FP64, long
    rows (Ntilde = 7 gives rows of 15 points)."""
    rs = np.random.default_rng(Nt)
    f = synth.mixture(3, 16, 6.0, rs)
    d = rs.standard_normal((16,) * 3)
    g = rs.standard_normal((16,) * 3)
    plan = q.Plan(3, 16, Nbar, 6.0, kernel="hp", Ntilde=Nt)
    plan.set_tuning(loss_fft=1)
    tf = lambda x: torch.tensor(x, dtype=torch.float64, device="cuda")
    J = q.qdvm_jvp(plan, tf(f), tf(d), "f64").cpu().numpy()
    G = q.qdvm_vjp(plan, tf(f), tf(g), "f64").cpu().numpy()
    r, sc = oracle.vjp(f, g, 6.0, Nbar, kernel="hp", Ntilde=Nt, with_scale=True)
    assert np.max(np.abs(G - r)) / np.max(sc) <= 1e-12
    lhs, rhs = float(np.sum(g * J)), float(np.sum(G * d))
    assert abs(lhs - rhs) <= 1e-11 * np.sum(np.abs(g)) * np.max(sc)
