"""GPU parity of the 3D path (plane sums over e^perp) against the CPU oracle.

Small grids are compared at every point; the 32^3 workloads (hard spheres,
Nbar in {3, 5, 7}) on sampled points the oracle evaluates one by one.
"""
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


def _as_prec(f, prec):
    return f if prec == "f64" else f.astype(np.float32).astype(np.float64)


def _eval(q, torch, f, L, Nbar, kernel, prec, Ntilde=None):
    plan = q.Plan(3, f.shape[0], Nbar, L, kernel=kernel, Ntilde=Ntilde)
    Q = q.qdvm_eval(plan, torch.tensor(f, dtype=_dt(torch, prec), device="cuda"), prec)
    torch.cuda.synchronize()
    return Q.cpu().numpy().astype(np.float64), plan


CASES = [
    ("random_N8", 8, 2.0, 1, None, 1),
    ("random_N10", 10, 3.0, 2, None, 2),
    ("random_N12_Nt3", 12, 3.0, 2, 3, 3),
    ("random_N16", 16, 4.0, 3, None, 4),
    ("random_N15_odd", 15, 4.0, 2, None, 5),
    ("mixture_N16", 16, 6.0, 2, None, 6),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
@pytest.mark.parametrize("kernel", ["unit", "hp"])
def test_single_cell_parity_small(q, torch, case, prec, kernel):
    name, N, L, Nbar, Nt, seed = case
    rng = np.random.default_rng(seed)
    f = synth.mixture(3, N, L, rng) if name.startswith("mixture") else rng.uniform(0, 1, (N,) * 3)
    f = _as_prec(f, prec)
    Q, _ = _eval(q, torch, f, L, Nbar, kernel, prec, Ntilde=Nt)
    ref = oracle.q(f, L, Nbar, kernel=kernel, Ntilde=Nt)
    err = oracle.rel_linf(Q, ref["Q"], ref["scale"])
    assert err <= TOL[prec], f"{name} {prec} {kernel}: {err:.3e}"


@pytest.mark.parametrize("N,Nbar", [(12, 2), (16, 3)])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
def test_integer_data_bit_exact(q, torch, N, Nbar, prec):
    f = synth.integer_field(3, N, maxval=2, seed=N)
    Q, _ = _eval(q, torch, f, 3.0, Nbar, "unit", prec)
    ref = oracle.q(f, 3.0, Nbar, kernel="unit")["Q"]
    assert np.array_equal(Q, ref)


def _sample_idx(N, n, seed):
    rng = np.random.default_rng(seed)
    idx = rng.choice(N ** 3, size=n, replace=False)
    # always include corners / faces (periodic wrap in every direction)
    extra = [0, N - 1, N * N - 1, N ** 3 - 1, (N // 2) * (N * N + N + 1)]
    return np.unique(np.concatenate([idx, extra])).astype(np.int64)


@pytest.mark.parametrize("Nbar", [3, 5, 7])
@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_trimaxwellian_N32_hard_spheres_sampled(q, torch, Nbar, prec):
    """3D, N = 32 on [-6,6]^3, anisotropic Gaussian T = (0.5, 1, 2), drift
    (0.5, 0, 0), hard-sphere weights, FP32 line sums."""
    f = _as_prec(synth.trimaxwellian_3d(32, 6.0), prec)
    Q, plan = _eval(q, torch, f, 6.0, Nbar, "hp", prec)
    assert plan.n_lines == {3: 145, 5: 577, 7: 1441}[Nbar]
    idx = _sample_idx(32, 160, Nbar)
    r = oracle.q_points(f, 6.0, Nbar, idx, kernel="hp")
    err = np.max(np.abs(Q.ravel()[idx] - r["Q"])) / np.max(r["scale"])
    assert err <= 1e-5, f"Nbar={Nbar} {prec}: {err:.3e}"


def test_fp64_N32_global_memory_path(q, torch):
    """FP64 32^3 does not fit on chip; the cell is read from a global copy."""
    f = synth.trimaxwellian_3d(32, 6.0)
    Q, _ = _eval(q, torch, f, 6.0, 3, "hp", "f64")
    idx = _sample_idx(32, 96, 11)
    r = oracle.q_points(f, 6.0, 3, idx, kernel="hp")
    assert np.max(np.abs(Q.ravel()[idx] - r["Q"])) / np.max(r["scale"]) <= 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32_kahan"])
def test_batched_3d_every_cell(q, torch, prec):
    b1 = synth.batch_3d(3, N=12, L=6.0, seed=4)
    b2 = synth.batch_3d(3, N=16, L=6.0, seed=5)
    Ns = np.concatenate([b1.Ns, b2.Ns])
    order = np.array([0, 3, 1, 4, 2, 5])
    parts = [b1.cell(i).ravel() for i in range(3)] + [b2.cell(i).ravel() for i in range(3)]
    b = synth.Batch(3, 6.0, Ns[order], np.concatenate([parts[i] for i in order]))
    plans = [q.Plan(3, 12, 2, 6.0, kernel="hp"), q.Plan(3, 16, 3, 6.0, kernel="hp")]
    cp = torch.tensor([0 if n == 12 else 1 for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=_dt(torch, prec), device="cuda")
    Q, mom = q.qdvm_eval_batched(plans, cp, co, f, prec)
    Qn = Q.cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    mom = mom.cpu().numpy()
    for c in range(b.n_cells):
        n = int(b.Ns[c])
        r = oracle.q(b.cell(c, fin), 6.0, 2 if n == 12 else 3, kernel="hp")
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= TOL[prec]
        mref = oracle.moments(b.cell(c, Qn), 6.0)
        h3 = (12.0 / n) ** 3
        assert np.allclose(mom[c], mref, rtol=0, atol=1e-12 * h3 * r["scale"].sum())
        assert abs(mom[c, 0]) <= (1e-13 if prec == "f64" else 1e-6) * h3 * r["scale"].sum()


def test_batched_3d_workload_sampled(q, torch):
    """256 cells of 32^3, Nbar = 5 (577 lines), hard spheres, FP32: sampled
    cells and points against the oracle."""
    b = synth.batch_3d(256, N=32, L=6.0, seed=1)
    plans = [q.Plan(3, 32, 5, 6.0, kernel="hp")]
    cp = torch.zeros(b.n_cells, dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    Q, mom = q.qdvm_eval_batched(plans, cp, co, f, "f32")
    Qn = Q.cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(Qn))
    for c in (0, 77, 255):
        idx = _sample_idx(32, 48, c)
        r = oracle.q_points(b.cell(c, fin), 6.0, 5, idx, kernel="hp")
        err = np.max(np.abs(b.cell(c, Qn).ravel()[idx] - r["Q"])) / np.max(r["scale"])
        assert err <= 1e-5
