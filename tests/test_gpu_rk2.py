"""Time stepping on the GPU (second-order TVD Runge-Kutta of Section 4 around
the batched evaluator) against the oracle's stepping, graph replay of the
loop, conservation of mass, and argument checks."""
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


def _setup(q, torch, b, plans, Ns, prec):
    cp = torch.tensor([Ns.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=_dt(torch, prec), device="cuda")
    return cp, co, f


def _bound(f0, L, Nbar, kernel, dt, n, Nt=None):
    """Error scale of n steps: the field plus n dt times the term scale."""
    r = oracle.q(f0, L, Nbar, kernel=kernel, Ntilde=Nt)
    return np.max(np.abs(f0)) + n * dt * np.max(r["scale"])


@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
@pytest.mark.parametrize("loss_fft", [0, 1])
def test_rk2_batched_2d_matches_oracle(q, torch, prec, loss_fft):
    Ns = (16, 32)
    b = synth.batch_2d(6, Ns=Ns, L=8.0, seed=71)
    plans = [q.Plan(2, n, 8, 8.0) for n in Ns]
    for p in plans:
        p.set_tuning(loss_fft=loss_fft)
    cp, co, f = _setup(q, torch, b, plans, list(Ns), prec)
    fin = f.cpu().numpy().astype(np.float64)
    dt, n = 0.004, 3
    q.qdvm_rk2_batched(plans, cp, co, f, dt, n, prec)
    fout = f.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        f0 = b.cell(c, fin)
        ref = oracle.rk2(f0, 8.0, 8, dt, n)
        assert np.max(np.abs(b.cell(c, fout) - ref)) <= TOL[prec] * _bound(f0, 8.0, 8, "unit", dt, n)


@pytest.mark.parametrize("prec", ["f64", "f32_kahan"])
def test_rk2_3d_row_form_matches_oracle(q, torch, prec):
    b = synth.batch_3d(2, N=16, L=6.0, seed=72)
    plan = q.Plan(3, 16, 3, 6.0, kernel="hp")
    plan.set_tuning(loss_fft=1)
    cp, co, f = _setup(q, torch, b, [plan], [16], prec)
    fin = f.cpu().numpy().astype(np.float64)
    dt, n = 0.05, 2  # a stable step: the field changes by about 5%
    q.qdvm_rk2_batched([plan], cp, co, f, dt, n, prec)
    fout = f.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        f0 = b.cell(c, fin)
        ref = oracle.rk2(f0, 6.0, 3, dt, n, kernel="hp")
        assert np.max(np.abs(b.cell(c, fout) - ref)) <= TOL[prec] * _bound(f0, 6.0, 3, "hp", dt, n)
        assert 1e-2 * np.max(np.abs(f0)) < np.max(np.abs(ref - f0)) < 0.2 * np.max(np.abs(f0))


def test_rk2_graph_replay_and_mass(q, torch):
    Ns = (16, 48, 64)
    b = synth.batch_2d(9, Ns=Ns, L=8.0, seed=73)
    plans = [q.Plan(2, n, 8, 8.0) for n in Ns]
    cp, co, f = _setup(q, torch, b, plans, list(Ns), "f64")
    f_direct = f.clone()
    _, m0 = q.qdvm_rk2_batched(plans, cp, co, f.clone(), 0.0, 0, "f64", moments=True)
    _, m_direct = q.qdvm_rk2_batched(plans, cp, co, f_direct, 0.003, 4, "f64", moments=True)
    g = q.RK2Graph(plans, cp, co, f, 0.003, 4, "f64", moments=True)
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(f, f_direct) and torch.equal(g.moments, m_direct)
    # mass is conserved by every stage
    m0, m1 = m0.cpu().numpy(), m_direct.cpu().numpy()
    assert np.all(np.abs(m1[:, 0] - m0[:, 0]) <= 1e-13 * np.abs(m0[:, 0]))
    assert not torch.equal(f_direct, torch.tensor(b.f, dtype=torch.float64, device="cuda"))


def test_rk2_zero_steps_and_argument_errors(q, torch):
    b = synth.batch_2d(3, Ns=(16,), L=8.0, seed=74)
    plans = [q.Plan(2, 16, 3, 8.0)]
    cp, co, f = _setup(q, torch, b, plans, [16], "f32")
    f0 = f.clone()
    q.qdvm_rk2_batched(plans, cp, co, f, 0.01, 0, "f32")
    assert torch.equal(f, f0)
    with pytest.raises(q.QdvmError):
        q.qdvm_rk2_batched(plans, cp, co, f, 0.01, -1, "f32")
    with pytest.raises(q.QdvmError):
        q.qdvm_rk2_batched(plans, cp, co, f, float("nan"), 1, "f32")
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(q.QdvmError):
        q.qdvm_rk2_batched(plans, cp, co, f, 0.01, 1, "f32", workspace=small)
    assert torch.equal(f, f0)


@pytest.mark.parametrize("d,N,Nbar,kernel,dt,loss_fft", [(2, 32, 7, "unit", 0.002, 0), (2, 32, 7, "unit", 0.002, 1),
                                                          (2, 80, 4, "unit", 0.002, 0), (3, 16, 3, "hp", 0.05, 1)])
def test_rk2_single_cell_matches_oracle(q, torch, d, N, Nbar, kernel, dt, loss_fft):
    """One cell through qdvm_rk2 (the single-cell evaluator, lines spread
    over the GPU; N = 80 takes the generic engine), FP64."""
    f0 = synth.bkw_2d(N, 8.0) if d == 2 else synth.mixture(3, N, 6.0, np.random.default_rng(2))
    L = 8.0 if d == 2 else 6.0
    plan = q.Plan(d, N, Nbar, L, kernel=kernel)
    plan.set_tuning(loss_fft=loss_fft)
    f = torch.tensor(f0, dtype=torch.float64, device="cuda")
    q.qdvm_rk2(plan, f, dt, 2, "f64")
    ref = oracle.rk2(f0, L, Nbar, dt, 2, kernel=kernel)
    assert np.max(np.abs(f.cpu().numpy() - ref)) <= 1e-12 * _bound(f0, L, Nbar, kernel, dt, 2)
    assert np.max(np.abs(ref - f0)) > 1e-4 * np.max(np.abs(f0))
