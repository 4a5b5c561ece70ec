"""Term-by-term GPU evaluation: the box-truncated operator D^tr of Section 2.3
against the oracle's (and its exact conservation of mass, momentum and
energy on the device), and the periodised operator computed without the
fast decomposition, against the oracle and against the fast evaluator."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32_kahan": 1e-5}
CASES = [(2, 16, 8.0, 16, "unit", None), (2, 20, 5.0, 3, "hp", None), (2, 32, 8.0, 8, "hp", None),
         (3, 8, 3.0, 1, "unit", None), (3, 12, 4.0, 2, "hp", None)]


@pytest.fixture(scope="module")
def q():
    import paper_1201_3986_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _f(d, N, L, seed):
    return synth.mixture(d, N, L, np.random.default_rng(seed))


@pytest.mark.parametrize("case", CASES, ids=[f"d{c[0]}N{c[1]}Nb{c[3]}{c[4]}" for c in CASES])
@pytest.mark.parametrize("prec", ["f64", "f32_kahan"])
@pytest.mark.parametrize("boundary", ["box", "periodic"])
def test_direct_matches_oracle(q, torch, case, prec, boundary):
    d, N, L, Nbar, kernel, Nt = case
    f0 = _f(d, N, L, N + d)
    f0 = f0 if prec == "f64" else f0.astype(np.float32).astype(np.float64)
    plan = q.Plan(d, N, Nbar, L, kernel=kernel, Ntilde=Nt)
    ft = torch.tensor(f0, dtype=torch.float64 if prec == "f64" else torch.float32, device="cuda")
    Q = q.qdvm_eval_direct(plan, ft, prec, boundary).cpu().numpy().astype(np.float64)
    r = oracle.dtr(f0, L, Nbar, kernel=kernel, Ntilde=Nt) if boundary == "box" else \
        oracle.q(f0, L, Nbar, kernel=kernel, Ntilde=Nt)
    assert oracle.rel_linf(Q, r["Q"], r["scale"]) <= TOL[prec]
    if boundary == "periodic":  # a second, independent GPU evaluation of Q
        Qf = q.qdvm_eval(plan, ft, prec).cpu().numpy().astype(np.float64)
        assert np.max(np.abs(Q - Qf)) <= 2 * TOL[prec] * np.max(r["scale"])


def test_box_operator_conserves_on_device(q, torch):
    """Moments of D^tr vanish for random positive data (FP64), unlike those
    of the periodised operator."""
    Ns = (16, 24, 32)
    b = synth.batch_2d(6, Ns=Ns, L=5.0, seed=81)
    rng = np.random.default_rng(82)
    fr = rng.uniform(0.0, 1.0, b.f.shape)
    plans = [q.Plan(2, n, 4, 5.0, kernel="hp") for n in Ns]
    cp = torch.tensor([Ns.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(fr, dtype=torch.float64, device="cuda")
    Qb, mb = q.qdvm_eval_direct_batched(plans, cp, co, f, "f64", "box")
    Qp, mp = q.qdvm_eval_direct_batched(plans, cp, co, f, "f64", "periodic")
    mb, mp = mb.cpu().numpy(), mp.cpu().numpy()
    Qbn = Qb.cpu().numpy()
    for c in range(b.n_cells):
        n = int(b.Ns[c])
        r = oracle.dtr(b.cell(c, fr), 5.0, 4, kernel="hp")
        assert oracle.rel_linf(b.cell(c, Qbn), r["Q"], r["scale"]) <= 1e-12
        h2 = (10.0 / n) ** 2
        bound = 1e-12 * h2 * r["scale"].sum() * 50.0  # |v|^2 <= 2 L^2 = 50
        assert np.all(np.abs(mb[c]) <= bound), (c, mb[c], bound)
        assert abs(mp[c, 3]) > 1e3 * bound  # the periodised operator moves energy


def test_direct_argument_errors(q, torch):
    plan = q.Plan(2, 16, 3, 8.0)
    f = torch.zeros(16 * 16, dtype=torch.float64, device="cuda")
    with pytest.raises(KeyError):
        q.qdvm_eval_direct(plan, f, "f64", "reflecting")
    cp = torch.zeros(1, dtype=torch.int32, device="cuda")
    co = torch.zeros(1, dtype=torch.int64, device="cuda")
    import ctypes
    lib = q._lib
    st = lib.qdvm_eval_direct_batched((ctypes.c_void_p * 1)(plan.handle), 1, 1, ctypes.c_void_p(cp.data_ptr()),
                                      ctypes.c_void_p(co.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                      ctypes.c_void_p(f.data_ptr()), None, 0, 1, None)
    assert st != 0  # f aliases Q
    st = lib.qdvm_eval_direct_batched((ctypes.c_void_p * 1)(plan.handle), 1, 1, ctypes.c_void_p(cp.data_ptr()),
                                      ctypes.c_void_p(co.data_ptr()), ctypes.c_void_p(f.data_ptr()), None, None, 0, 2,
                                      None)
    assert st != 0  # unknown boundary
