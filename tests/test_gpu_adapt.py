"""Space-dependent Nbar on the GPU: the equilibrium indicator against the
oracle's (the kernel sums in FP32 with compensation: agreement to about
1e-7), the level selection (unique for cells farther than the indicator's
accuracy from a threshold; either adjacent level is valid within it), and an
adaptive batched evaluation against the oracle at each cell's selected Nbar."""

EPS_TOL = 2e-6  # |indicator - oracle| <= EPS_TOL * (1 + oracle)
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

NS = (16, 32, 48, 64)
NBARS = (2, 4, 8)
THR = (0.02, 0.1)


@pytest.fixture(scope="module")
def q():
    import paper_1201_3986_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _batch(torch, b, prec):
    cb = torch.tensor([NS.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float64 if prec == "f64" else torch.float32, device="cuda")
    return cb, co, f


def _level(e):
    return int(sum(not (e < t) for t in THR))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_indicator_matches_oracle_2d(q, torch, prec):
    b = synth.batch_2d_relaxing(40, Ns=NS, L=8.0, seed=11)
    plans = [q.Plan(2, n, 8, 8.0) for n in NS]
    cb, co, f = _batch(torch, b, prec)
    eps = q.equilibrium_distance(plans, cb, co, f, prec).cpu().numpy()
    fin = f.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        ref = oracle.equilibrium_distance(b.cell(c, fin), 8.0)
        assert abs(eps[c] - ref) <= EPS_TOL * (1.0 + ref), (c, eps[c], ref)


def test_indicator_3d_and_undefined_cells(q, torch):
    b = synth.batch_3d(3, N=16, L=6.0, seed=12)
    f_np = b.f.copy()
    f_np[b.offsets[1]:b.offsets[1] + 16 ** 3] = 0.0          # empty cell
    f_np[b.offsets[2]:b.offsets[2] + 16 ** 3] *= -1.0        # negative mass
    plan = q.Plan(3, 16, 3, 6.0)
    cp = torch.zeros(3, dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(f_np, dtype=torch.float64, device="cuda")
    eps = q.equilibrium_distance([plan], cp, co, f, "f64").cpu().numpy()
    ref = oracle.equilibrium_distance(f_np[:16 ** 3].reshape(16, 16, 16), 6.0)
    assert abs(eps[0] - ref) <= EPS_TOL * (1.0 + ref)
    assert np.isinf(eps[1]) and np.isinf(eps[2])
    sel = q.select_levels(torch.tensor(eps, device="cuda"), cp, THR, [[5, 6, 7]]).cpu().numpy()
    assert sel[1] == 7 and sel[2] == 7


def test_adaptive_batched_evaluation(q, torch):
    b = synth.batch_2d_relaxing(48, Ns=NS, L=8.0, seed=13)
    plans = [q.Plan(2, n, nb, 8.0) for n in NS for nb in NBARS]  # plan index = 3 * base + level
    level_plan = np.arange(len(plans)).reshape(len(NS), len(NBARS))
    cb, co, f = _batch(torch, b, "f32_kahan")
    # the indicator needs each cell's N and L: the first plan of each size
    eps = q.equilibrium_distance(plans[::len(NBARS)], cb, co, f, "f32_kahan")
    cp = q.select_levels(eps, cb, THR, level_plan)
    Q, _ = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan")
    eps_n, cp_n = eps.cpu().numpy(), cp.cpu().numpy()
    fin = f.cpu().numpy().astype(np.float64)
    Qn = Q.cpu().numpy().astype(np.float64)
    seen = set()
    for c in range(b.n_cells):
        e_ref = oracle.equilibrium_distance(b.cell(c, fin), 8.0)
        lo, hi = _level(e_ref - EPS_TOL * (1 + e_ref)), _level(e_ref + EPS_TOL * (1 + e_ref))
        assert lo <= cp_n[c] - 3 * NS.index(int(b.Ns[c])) <= hi
        # the selection itself is exact on the indicator values it is given
        assert cp_n[c] == 3 * NS.index(int(b.Ns[c])) + _level(eps_n[c])
        lev = int(cp_n[c]) % 3
        seen.add(lev)
        r = oracle.q(b.cell(c, fin), 8.0, NBARS[lev])
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= 1e-5
    assert seen == {0, 1, 2}


def test_select_levels_argument_errors(q, torch):
    eps = torch.zeros(4, dtype=torch.float64, device="cuda")
    cb = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(q.QdvmError):
        q.select_levels(eps, cb, (0.1, 0.05), [[0, 1, 2]])      # not increasing
    with pytest.raises(q.QdvmError):
        q.select_levels(eps, cb, (0.1,), [[0, 99]])             # plan index out of range
    with pytest.raises(q.QdvmError):
        q.select_levels(eps, cb, tuple(np.linspace(0.1, 0.9, 8)), [list(range(9))])  # 9 levels
    out = q.select_levels(eps, torch.tensor([0, 1, -1, 5], dtype=torch.int32, device="cuda"), (0.5,),
                          [[3, 4], [5, 6]]).cpu().numpy()
    assert list(out) == [3, 5, -1, -1]
