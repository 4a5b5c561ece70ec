"""Edge cases: 2D cells larger than the on-chip evaluator (generic engine),
the largest 3D cell, odd sizes, and argument errors of the batched entry
points."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import paper_1201_3986_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _idx(n_total, n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.choice(n_total, size=n, replace=False), [0, n_total - 1]])).astype(np.int64)


@pytest.mark.parametrize("N,Nbar", [(80, 3), (96, 4), (128, 2)])
@pytest.mark.parametrize("prec", ["f64", "f32_kahan"])
def test_2d_large_cells_generic_engine(q, torch, N, Nbar, prec):
    f = synth.mixture(2, N, 8.0, np.random.default_rng(N))
    f = f if prec == "f64" else f.astype(np.float32).astype(np.float64)
    plan = q.Plan(2, N, Nbar, 8.0, kernel="hp")
    Q = q.qdvm_eval(plan, torch.tensor(f, dtype=torch.float64 if prec == "f64" else torch.float32, device="cuda"),
                    prec).cpu().numpy().astype(np.float64)
    idx = _idx(N * N, 300, N)
    r = oracle.q_points(f, 8.0, Nbar, idx, kernel="hp")
    err = np.max(np.abs(Q.ravel()[idx] - r["Q"])) / np.max(r["scale"])
    assert err <= (1e-12 if prec == "f64" else 1e-5)


def test_2d_large_cells_derivatives(q, torch):
    N, Nbar = 80, 2
    rs = np.random.default_rng(1)
    f = rs.uniform(0.1, 1.0, (N, N))
    g = rs.standard_normal((N, N))
    plan = q.Plan(2, N, Nbar, 8.0, kernel="hp")
    ft = torch.tensor(f, device="cuda")
    gt = torch.tensor(g, device="cuda")
    G = q.qdvm_vjp(plan, ft, gt, "f64").cpu().numpy()
    J = q.qdvm_jvp(plan, ft, gt, "f64").cpu().numpy()
    idx = _idx(N * N, 100, 2)
    Gr, Gs = oracle.vjp_points(f, g, 8.0, Nbar, idx, kernel="hp")
    Jr, Js = oracle.jvp_points(f, g, 8.0, Nbar, idx, kernel="hp")
    assert np.max(np.abs(G.ravel()[idx] - Gr)) / np.max(Gs) <= 1e-12
    assert np.max(np.abs(J.ravel()[idx] - Jr)) / np.max(Js) <= 1e-12


def test_2d_mixed_batch_on_and_off_chip(q, torch):
    """One batch whose plans do not all fit on chip runs entirely on the
    generic engine."""
    Ns = (16, 80)
    b = synth.batch_2d(5, Ns=Ns, L=8.0, seed=4)
    plans = [q.Plan(2, n, 2, 8.0) for n in Ns]
    cp = torch.tensor([Ns.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float64, device="cuda")
    Q, M = q.qdvm_eval_batched(plans, cp, co, f, "f64")
    Qn = Q.cpu().numpy()
    for c in range(b.n_cells):
        fc = b.cell(c)
        idx = _idx(fc.size, 60, c)
        r = oracle.q_points(fc, 8.0, 2, idx)
        assert np.max(np.abs(b.cell(c, Qn).ravel()[idx] - r["Q"])) / np.max(r["scale"]) <= 1e-12


def test_3d_largest_cell_fp32(q, torch):
    N = 64
    f = synth.maxwellian(3, N, 8.0, 1.0, (0.3, 0.0, -0.2), 1.5)
    plan = q.Plan(3, N, 1, 8.0, kernel="hp")
    Q = q.qdvm_eval(plan, torch.tensor(f, dtype=torch.float32, device="cuda"), "f32").cpu().numpy()
    idx = _idx(N ** 3, 40, 3)
    r = oracle.q_points(f.astype(np.float32).astype(np.float64), 8.0, 1, idx, kernel="hp")
    assert np.max(np.abs(Q.ravel()[idx] - r["Q"])) / np.max(r["scale"]) <= 1e-5


@pytest.mark.parametrize("N", [9, 13])
def test_3d_odd_sizes(q, torch, N):
    f = np.random.default_rng(N).uniform(0, 1, (N,) * 3)
    plan = q.Plan(3, N, 2, 3.0, kernel="unit")
    Q = q.qdvm_eval(plan, torch.tensor(f, device="cuda"), "f64").cpu().numpy()
    r = oracle.q(f, 3.0, 2)
    assert oracle.rel_linf(Q, r["Q"], r["scale"]) <= 1e-12


def test_batched_argument_errors(q, torch):
    p2 = q.Plan(2, 16, 3, 8.0)
    p3 = q.Plan(3, 12, 2, 6.0)
    cp = torch.zeros(1, dtype=torch.int32, device="cuda")
    co = torch.zeros(1, dtype=torch.int64, device="cuda")
    f = torch.zeros(256, dtype=torch.float32, device="cuda")
    with pytest.raises(q.QdvmError) as ei:  # plans of different dimension
        q.qdvm_eval_batched([p2, p3], cp, co, f, "f32")
    assert ei.value.status == 1
    with pytest.raises(q.QdvmError) as ei:  # workspace too small
        q.qdvm_eval_batched([p2], cp, co, f, "f32", workspace=torch.zeros(8, dtype=torch.uint8, device="cuda"))
    assert ei.value.status == 1
    with pytest.raises(q.QdvmError):  # aliasing
        q.qdvm_eval_batched([p2], cp, co, f, "f32", out=f)
    with pytest.raises(q.QdvmError):  # more plans than a batch holds
        q.qdvm_eval_batched([p2] * 17, cp, co, f, "f32")
