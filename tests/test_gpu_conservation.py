"""Conservation defects of the GPU results, per result, against the FP64
oracle's own defects.

The invariants are those of Section 2.2 (the four facts after eq. (weakpe)):
sum_v Q phi = 0 for phi = 1, v, |v|^2.  Under periodisation only mass is
exact for any data; momentum and energy are exact when no term wraps around
the torus (data supported in [-S, S]^d with S + Ntilde <= N/2 - 1).  So the
FP32 path is held to the FP64 oracle's defect, per cell and per phi:

    defect_phi = |h^d sum_i Q_i phi(v_i)| / (h^d sum_i scale_i |phi(v_i)|),
    |defect_gpu - defect_oracle64| <= 1e-6,

with scale_i the oracle's sum of absolute terms at i.  The test asserts the
stronger |m_gpu - m_oracle| / denominator <= 1e-6 (the difference of the
absolute values is bounded by it).  The GPU moments are the ones the
evaluator writes (FP64 accuracy from FP32 line sums).
"""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_eval2d import displacement_histogram, total_scale

pytestmark = pytest.mark.gpu

BAR = 1e-6


@pytest.fixture(scope="module")
def q():
    import paper_1201_3986_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def phis(d, N, L):
    """phi = 1, v_0, ..., v_{d-1}, |v|^2 on the vertex grid v = -L + j h,
    as arrays of shape N^d (axis 0 first)."""
    v = -L + np.arange(N) * (2.0 * L / N)
    grids = np.meshgrid(*([v] * d), indexing="ij")
    return [np.ones((N,) * d)] + list(grids) + [sum(g * g for g in grids)]


def defects(m_gpu, Q_ref, scale, L):
    """(defect_gpu, defect_oracle, |m_gpu - m_oracle| / den) per phi."""
    d, N = Q_ref.ndim, Q_ref.shape[0]
    hd = (2.0 * L / N) ** d
    m_ref = oracle.moments(Q_ref, L)
    den = np.array([hd * np.sum(scale * np.abs(p)) for p in phis(d, N, L)])
    m_gpu = np.asarray(m_gpu, dtype=np.float64)[: d + 2]
    return np.abs(m_gpu) / den, np.abs(m_ref) / den, np.abs(m_gpu - m_ref) / den


def test_benchmark_launch_defects(q, torch):
    """The benchmark's own launch (4096 cells, N in {16, 32, 48, 64}, Nbar = 8,
    FP32 with compensation, autotuned, replayed from a CUDA graph): all four
    defects against the oracle's on 16 cells, four of each size, and the
    mass bar on every cell."""
    Ns = (16, 32, 48, 64)
    L = 8.0
    b = synth.batch_2d(4096, Ns=Ns, L=L, seed=0)
    plans = [q.Plan(2, n, 8, L, kernel="unit") for n in Ns]
    cp = torch.tensor([Ns.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    ws = torch.empty(q.batched_workspace_bytes(plans, b.n_cells, "f32_kahan"), dtype=torch.uint8, device="cuda")
    q.qdvm_tune_batched(plans, cp, co, f, "f32_kahan", workspace=ws)
    Q = torch.empty_like(f)
    M = torch.full((b.n_cells, 4), float("nan"), dtype=torch.float64, device="cuda")
    g = q.BatchedGraph(plans, cp, co, f, Q, M, "f32_kahan", workspace=ws)
    g.launch()
    torch.cuda.synchronize()
    Mn = M.cpu().numpy()
    fin = f.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(Mn))
    rng = np.random.default_rng(7)
    for n in Ns:
        for c in rng.choice(np.nonzero(b.Ns == n)[0], size=4, replace=False):
            r = oracle.q(b.cell(int(c), fin), L, 8)
            dg, dr, dm = defects(Mn[c], r["Q"], r["scale"], L)
            assert np.all(np.abs(dg - dr) <= BAR), f"cell {c} (N={n}): {dg} vs oracle {dr}"
            assert np.all(dm <= BAR), f"cell {c} (N={n}): moment differences {dm}"
    hist = {n: displacement_histogram(n, 8) for n in Ns}
    for c in range(b.n_cells):
        fc = b.cell(c, fin)
        h2 = (2.0 * L / fc.shape[0]) ** 2
        assert abs(Mn[c, 0]) <= BAR * h2 * total_scale(fc, hist[fc.shape[0]]), f"mass, cell {c}"


_REF3 = {}


def _oracle_3d(Nbar):
    """Full FP64 oracle of the 32^3 tri-axial cell (hard spheres), once per
    Nbar: the defects need every point."""
    if Nbar not in _REF3:
        f = synth.trimaxwellian_3d(32, 6.0).astype(np.float32).astype(np.float64)
        _REF3[Nbar] = (f, oracle.q(f, 6.0, Nbar, kernel="hp"))
    return _REF3[Nbar]


@pytest.mark.parametrize("Nbar", [3, 5, 7])
@pytest.mark.parametrize("prec,loss_fft", [("f32", 1), ("f32_kahan", 0)])
def test_config3_defects(q, torch, Nbar, prec, loss_fft):
    """3D, N = 32 on [-6, 6]^3, hard spheres, the tri-axial Gaussian
    (temperatures 0.5, 1, 2, drift (0.5, 0, 0)), FP32 line sums, FP64
    moments: the five defects (mass, three momentum components, energy)
    against the oracle's, with the row-form evaluator (loss_fft = 1) and
    the line engine (loss_fft = 0)."""
    f, r = _oracle_3d(Nbar)
    plan = q.Plan(3, 32, Nbar, 6.0, kernel="hp")
    plan.set_tuning(loss_fft=loss_fft)
    cp = torch.zeros(1, dtype=torch.int32, device="cuda")
    co = torch.zeros(1, dtype=torch.int64, device="cuda")
    ft = torch.tensor(f.ravel(), dtype=torch.float32, device="cuda")
    Q, M = q.qdvm_eval_batched([plan], cp, co, ft, prec)
    Qn = Q.cpu().numpy().astype(np.float64).reshape(f.shape)
    assert oracle.rel_linf(Qn, r["Q"], r["scale"]) <= 1e-5
    dg, dr, dm = defects(M.cpu().numpy()[0], r["Q"], r["scale"], 6.0)
    assert np.all(np.abs(dg - dr) <= BAR), f"{dg} vs oracle {dr}"
    assert np.all(dm <= BAR), f"moment differences {dm}"


@pytest.mark.parametrize("d,N,L,Nbar,S,loss_fft", [(2, 64, 8.0, 8, 17, 2), (2, 48, 8.0, 8, 13, 0),
                                                  (3, 32, 6.0, 5, 8, 1)])
def test_exact_conservation_without_wrap(q, torch, d, N, L, Nbar, S, loss_fft):
    """Data supported in [-S, S]^d (lattice offsets from the centre) with
    S + Ntilde = N/2 - 1: no term wraps, so momentum and energy are conserved
    exactly (Section 2.2) and the FP32 defects of all d + 2 moments are
    within 1e-6 of zero, as are the oracle's (to rounding)."""
    Nt = oracle.default_ntilde(N)
    assert S + Nt <= N // 2 - 1
    f = synth.compact_support(d, N, S, seed=N + d).astype(np.float32).astype(np.float64)
    plan = q.Plan(d, N, Nbar, L, kernel="hp")
    plan.set_tuning(loss_fft=loss_fft)
    cp = torch.zeros(1, dtype=torch.int32, device="cuda")
    co = torch.zeros(1, dtype=torch.int64, device="cuda")
    ft = torch.tensor(f.ravel(), dtype=torch.float32, device="cuda")
    _, M = q.qdvm_eval_batched([plan], cp, co, ft, "f32_kahan")
    r = oracle.q(f, L, Nbar, kernel="hp")
    dg, dr, dm = defects(M.cpu().numpy()[0], r["Q"], r["scale"], L)
    assert np.all(dr <= 1e-13), f"oracle defects {dr}"
    assert np.all(dg <= BAR), f"GPU defects {dg}"
