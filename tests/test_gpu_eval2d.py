"""GPU parity of the 2D path against the CPU oracle (through the C ABI).

Bars: FP64 rel L_inf <= 1e-12 and FP32 / FP32+compensation <= 1e-5, the error
taken relative to max_i sum_{(k,l)} |terms| (the oracle's ``scale``; Q itself
vanishes near equilibrium).  Integer data with the unit kernel must match
bit for bit.
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


def _gpu_eval(q, torch, f, L, Nbar, kernel, prec, Ntilde=None):
    d, N = f.ndim, f.shape[0]
    plan = q.Plan(d, N, Nbar, L, kernel=kernel, Ntilde=Ntilde)
    dt = torch.float64 if prec == "f64" else torch.float32
    ft = torch.tensor(f, dtype=dt, device="cuda")
    Q = q.qdvm_eval(plan, ft, prec)
    torch.cuda.synchronize()
    return Q.cpu().numpy().astype(np.float64), plan


def _as_prec(f, prec):
    return f if prec == "f64" else f.astype(np.float32).astype(np.float64)


# ------------------------------------------------------------------ plans

@pytest.mark.parametrize("d,N,Nbar", [(2, 16, 16), (2, 64, 4), (2, 64, 8), (2, 64, 16), (2, 48, 8), (2, 7, 1),
                                      (3, 32, 3), (3, 32, 5), (3, 16, 2)])
@pytest.mark.parametrize("kernel", ["unit", "hp"])
def test_plan_lines_match_oracle_enumeration(q, d, N, Nbar, kernel):
    L = 8.0 if d == 2 else 6.0
    plan = q.Plan(d, N, Nbar, L, kernel=kernel)
    Nt = oracle.default_ntilde(N)
    m = min(Nbar, Nt)
    assert plan.Ntilde == Nt and plan.m == m
    ref = oracle.lines(d, m)
    dirs, J, c = plan.lines()
    assert np.array_equal(dirs, ref)
    linf = np.max(np.abs(ref), axis=1)
    assert np.array_equal(J, Nt // linf)
    h = 2 * L / N
    want = np.ones(len(ref)) if kernel == "unit" else h ** (2 * d - 1) * np.linalg.norm(ref, axis=1)
    assert np.allclose(c, want, rtol=1e-15, atol=0)
    assert plan.n_terms == oracle.terms_count(d, Nt, m)


def test_plan_rejects_bad_arguments(q):
    for args in [(1, 16, 3, 8.0), (2, 3, 3, 8.0), (2, 16, 0, 8.0), (2, 16, 3, 0.0), (3, 65, 3, 6.0), (2, 300, 3, 8.0)]:
        with pytest.raises(q.QdvmError):
            q.Plan(*args)
    with pytest.raises(q.QdvmError):
        q.Plan(2, 16, 3, 8.0, Ntilde=8)  # 2 Ntilde must be < N


# ------------------------------------------------------------ single cell

CASES_2D = [
    # (name, f builder, N, L, Nbar, Ntilde)
    ("two_maxwellians_N16_all", lambda: synth.two_maxwellians_2d(16, 8.0), 16, 8.0, 16, None),
    ("bkw_N64_Nbar4", lambda: synth.bkw_2d(64, 8.0), 64, 8.0, 4, None),
    ("bkw_N64_Nbar8", lambda: synth.bkw_2d(64, 8.0), 64, 8.0, 8, None),
    ("bkw_N64_Nbar16", lambda: synth.bkw_2d(64, 8.0), 64, 8.0, 16, None),
    ("bkw_literal_N64_Nbar8", lambda: synth.bkw_literal_2d(64, 8.0), 64, 8.0, 8, None),
    ("random_N20", lambda: np.random.default_rng(1).uniform(0, 1, (20, 20)), 20, 3.0, 3, None),
    ("random_N40_Nt9", lambda: np.random.default_rng(2).uniform(0, 1, (40, 40)), 40, 5.0, 5, 9),
    ("random_N50", lambda: np.random.default_rng(3).uniform(0, 1, (50, 50)), 50, 5.0, 6, None),
    ("random_N5_min", lambda: np.random.default_rng(4).uniform(0, 1, (5, 5)), 5, 2.0, 1, None),
    ("mixture_N48", lambda: synth.mixture(2, 48, 8.0, np.random.default_rng(5)), 48, 8.0, 8, None),
    ("mixture_N32", lambda: synth.mixture(2, 32, 8.0, np.random.default_rng(6)), 32, 8.0, 8, None),
]


@pytest.mark.parametrize("case", CASES_2D, ids=[c[0] for c in CASES_2D])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
@pytest.mark.parametrize("kernel", ["unit", "hp"])
def test_single_cell_parity(q, torch, case, prec, kernel):
    name, build, N, L, Nbar, Nt = case
    f = _as_prec(build(), prec)
    Q, plan = _gpu_eval(q, torch, f, L, Nbar, kernel, prec, Ntilde=Nt)
    ref = oracle.q(f, L, Nbar, kernel=kernel, Ntilde=Nt)
    err = oracle.rel_linf(Q, ref["Q"], ref["scale"])
    assert err <= TOL[prec], f"{name} {prec} {kernel}: rel err {err:.3e}"


@pytest.mark.parametrize("N,Nbar,maxval", [(16, 3, 3), (32, 5, 3), (64, 8, 2), (48, 8, 3), (21, 4, 5)])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
def test_integer_data_bit_exact(q, torch, N, Nbar, maxval, prec):
    f = synth.integer_field(2, N, maxval=maxval, seed=N)
    Q, _ = _gpu_eval(q, torch, f, 4.0, Nbar, "unit", prec)
    ref = oracle.q(f, 4.0, Nbar, kernel="unit")["Q"]
    assert np.array_equal(Q, ref)


def test_special_inputs(q, torch):
    N = 32
    for prec in ("f64", "f32"):
        Q, _ = _gpu_eval(q, torch, np.zeros((N, N)), 8.0, 8, "hp", prec)
        assert np.all(Q == 0)
        Q, _ = _gpu_eval(q, torch, np.full((N, N), 0.25), 8.0, 8, "unit", prec)
        assert np.all(Q == 0)
        d = np.zeros((N, N))
        d[3, 30] = 1.0
        Q, _ = _gpu_eval(q, torch, d, 8.0, 8, "hp", prec)
        assert np.all(Q == 0)


def test_deterministic(q, torch):
    f = synth.bkw_2d(64, 8.0)
    a, _ = _gpu_eval(q, torch, f, 8.0, 8, "hp", "f32_kahan")
    b, _ = _gpu_eval(q, torch, f, 8.0, 8, "hp", "f32_kahan")
    assert np.array_equal(a, b)


def test_moments_single(q, torch):
    f = synth.two_maxwellians_2d(16, 8.0)
    plan = q.Plan(2, 16, 16, 8.0)
    Qt = q.qdvm_eval(plan, torch.tensor(f, device="cuda"), "f64")
    m = q.qdvm_moments(plan, Qt, "f64").cpu().numpy()
    ref = oracle.moments(Qt.cpu().numpy(), 8.0)
    scale = oracle.q(f, 8.0, 16)["scale"]
    assert np.allclose(m, ref, rtol=0, atol=1e-14 * scale.sum())


def test_rejects_bad_eval_arguments(q, torch):
    plan = q.Plan(2, 16, 3, 8.0)
    f = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        q.qdvm_eval(plan, f.float(), "f64")
    with pytest.raises(q.QdvmError):
        q.qdvm_eval(plan, f, "f64", out=f)  # aliasing f and Q


# ----------------------------------------------------------------- batched

def _batch_tensors(torch, b, plans_N, prec):
    idx = {n: i for i, n in enumerate(plans_N)}
    cp = torch.tensor([idx[int(n)] for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    dt = torch.float64 if prec == "f64" else torch.float32
    f = torch.tensor(b.f, dtype=dt, device="cuda")
    return cp, co, f


@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
def test_batched_parity_every_cell(q, torch, prec):
    Ns = (16, 32, 48, 64)
    b = synth.batch_2d(24, Ns=Ns, L=8.0, seed=7)
    plans = [q.Plan(2, n, 8, 8.0, kernel="unit") for n in Ns]
    cp, co, f = _batch_tensors(torch, b, Ns, prec)
    Q, mom = q.qdvm_eval_batched(plans, cp, co, f, prec)
    Qn = Q.cpu().numpy().astype(np.float64)
    mom = mom.cpu().numpy()
    fin = f.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        fc = b.cell(c, fin)
        r = oracle.q(fc, 8.0, 8)
        Qc = b.cell(c, Qn)
        assert oracle.rel_linf(Qc, r["Q"], r["scale"]) <= TOL[prec]
        mref = oracle.moments(Qc, 8.0)
        h2 = (16.0 / fc.shape[0]) ** 2
        assert np.allclose(mom[c], mref, rtol=0, atol=1e-13 * h2 * np.sum(np.abs(Qc)) * 64 + 1e-300)


def test_batched_matches_single_bitwise(q, torch):
    Ns = (16, 48)
    b = synth.batch_2d(6, Ns=Ns, L=8.0, seed=9)
    plans = [q.Plan(2, n, 8, 8.0, kernel="hp") for n in Ns]
    cp, co, f = _batch_tensors(torch, b, Ns, "f32_kahan")
    Q, _ = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan")
    for c in range(b.n_cells):
        n = int(b.Ns[c])
        o = int(b.offsets[c])
        Qs = q.qdvm_eval(plans[Ns.index(n)], f[o:o + n * n].view(n, n).contiguous(), "f32_kahan")
        # the single-cell path may split the lines across CTAs (different
        # summation grouping), so compare at the FP32 bar, not bitwise
        ref = oracle.q(b.cell(c, f.cpu().numpy().astype(np.float64)), 8.0, 8, kernel="hp")
        assert oracle.rel_linf(Q[o:o + n * n].view(n, n).cpu().numpy(), Qs.cpu().numpy(), ref["scale"]) <= 1e-5


def test_batched_empty_and_invalid_plan_index(q, torch):
    plans = [q.Plan(2, 16, 3, 8.0)]
    cp = torch.zeros(0, dtype=torch.int32, device="cuda")
    co = torch.zeros(0, dtype=torch.int64, device="cuda")
    f = torch.zeros(0, dtype=torch.float32, device="cuda")
    Q, mom = q.qdvm_eval_batched(plans, cp, co, f, "f32")
    assert Q.numel() == 0 and mom.shape == (0, 4)
    # a cell whose plan index is out of range is skipped (its Q untouched)
    b = synth.batch_2d(3, Ns=(16,), L=8.0, seed=1)
    cp = torch.tensor([0, 5, 0], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    out = torch.full_like(f, 7.0)
    Q, _ = q.qdvm_eval_batched(plans, cp, co, f, "f32", out=out)
    Qn = Q.cpu().numpy()
    assert np.all(Qn[256:512] == 7.0)
    r = oracle.q(b.cell(2, f.cpu().numpy().astype(np.float64)), 8.0, 3)
    assert oracle.rel_linf(Qn[512:].reshape(16, 16), r["Q"], r["scale"]) <= 1e-5


@pytest.mark.parametrize("loss_fft", [0, 1, 2])
def test_batched_full_workload_sampled(q, torch, loss_fft):
    """4096 cells, N uniform in {16,32,48,64}, Nbar = 8, FP32 + compensation,
    with the loss by direct sums (0), by the FFT (1), or by the FFT that also
    gives the axis window (2).  Sampled cells against the oracle, mass
    conservation on every cell."""
    Ns = (16, 32, 48, 64)
    b = synth.batch_2d(4096, Ns=Ns, L=8.0, seed=0)
    plans = [q.Plan(2, n, 8, 8.0, kernel="unit") for n in Ns]
    for p in plans:
        p.set_tuning(loss_fft=loss_fft)
    cp, co, f = _batch_tensors(torch, b, Ns, "f32_kahan")
    Q, mom = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan")
    Qn = Q.cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    mom = mom.cpu().numpy()
    assert np.all(np.isfinite(Qn))
    rng = np.random.default_rng(0)
    picks = []
    for n in Ns:
        cells = np.nonzero(b.Ns == n)[0]
        picks += list(rng.choice(cells, size=2, replace=False))
    for c in picks:
        r = oracle.q(b.cell(c, fin), 8.0, 8)
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= 1e-5
    # mass defect |sum Q| / sum scale <= 1e-6 on every cell (FP32 bar)
    hist = {n: displacement_histogram(n, 8) for n in Ns}
    for c in range(b.n_cells):
        fc = b.cell(c, fin)
        h2 = (16.0 / fc.shape[0]) ** 2
        assert abs(mom[c, 0]) <= 1e-6 * h2 * total_scale(fc, hist[fc.shape[0]])


def test_benchmark_launch_full_workload(q, torch):
    """The benchmark's own launch on its 4096-cell batch: the autotuner picks
    the configuration, the evaluation is replayed from a captured CUDA graph.
    Sampled cells against the oracle; on every cell the mass defect (FP32
    bar) and the moments against an FP64 sum of the stored Q; the graph
    replay equal bit for bit to a direct call with the same tuning."""
    Ns = (16, 32, 48, 64)
    b = synth.batch_2d(4096, Ns=Ns, L=8.0, seed=0)
    plans = [q.Plan(2, n, 8, 8.0, kernel="unit") for n in Ns]
    cp, co, f = _batch_tensors(torch, b, Ns, "f32_kahan")
    ws = torch.empty(q.batched_workspace_bytes(plans, b.n_cells, "f32_kahan"), dtype=torch.uint8, device="cuda")
    tuning = q.qdvm_tune_batched(plans, cp, co, f, "f32_kahan", workspace=ws)
    # per-plan launch parameters: plans[0]'s is returned, the block size is shared
    assert plans[0].tuning() == tuning
    assert all(p.tuning()["threads"] == tuning["threads"] for p in plans)
    Q = torch.full_like(f, float("nan"))
    mom = torch.full((b.n_cells, 4), float("nan"), dtype=torch.float64, device="cuda")
    g = q.BatchedGraph(plans, cp, co, f, Q, mom, "f32_kahan", workspace=ws)
    g.launch()
    g.launch()
    torch.cuda.synchronize()
    Qd, momd = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan")
    assert torch.equal(Q, Qd) and torch.equal(mom, momd)
    Qn = Q.cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    mom = mom.cpu().numpy()
    rng = np.random.default_rng(3)
    for n in Ns:
        for c in rng.choice(np.nonzero(b.Ns == n)[0], size=2, replace=False):
            r = oracle.q(b.cell(int(c), fin), 8.0, 8)
            assert oracle.rel_linf(b.cell(int(c), Qn), r["Q"], r["scale"]) <= 1e-5
    hist = {n: displacement_histogram(n, 8) for n in Ns}
    for c in range(b.n_cells):
        fc, Qc = b.cell(c, fin), b.cell(c, Qn)
        h2 = (16.0 / fc.shape[0]) ** 2
        assert abs(mom[c, 0]) <= 1e-6 * h2 * total_scale(fc, hist[fc.shape[0]])
        mref = oracle.moments(Qc, 8.0)
        assert np.allclose(mom[c], mref, rtol=0, atol=1e-13 * h2 * np.sum(np.abs(Qc)) * 64)


def displacement_histogram(N, Nbar):
    """K(m) = number of unit-kernel terms (k, l) of the restricted set with
    k + l = m (mod N), from the oracle's line list."""
    Nt = oracle.default_ntilde(N)
    K = np.zeros((N, N))
    for e in oracle.lines(2, min(Nbar, Nt)):
        J = Nt // int(np.max(np.abs(e)))
        ep = np.array([-e[1], e[0]])
        js = [j for j in range(-J, J + 1) if j]
        for j in js:
            for jp in js:
                m = (j * e + jp * ep) % N
                K[m[0], m[1]] += 1
    return K


def total_scale(f, K):
    """sum_i scale_i = sum gain + sum loss = 2 sum_i loss_i
    = 2 sum_m K(m) R(m), R(m) = sum_i f_i f_{i+m} (f >= 0)."""
    F = np.fft.fft2(f)
    R = np.fft.ifft2(np.conj(F) * F).real
    return 2.0 * float(np.sum(K * R))


@pytest.mark.parametrize("n16,n12", [(1, 0), (5, 0), (7, 3), (4, 1), (9, 6)])
@pytest.mark.parametrize("loss_fft", [1, 2])
def test_quad16_tails_and_other_plans(q, torch, n16, n12, loss_fft):
    """16^2 FP32 cells go four to a CTA (64 threads each): batches whose
    count of 16^2 cells is not a multiple of four, and 12^2 cells drawn
    along with them (the schedule lists the cheaper 12^2 plan right after),
    against the oracle cell by cell, Q and moments."""
    b16 = synth.batch_2d(n16, Ns=(16,), L=8.0, seed=60 + n16)
    b12 = synth.batch_2d(max(n12, 1), Ns=(12,), L=8.0, seed=70 + n12)
    Ns = np.concatenate([b16.Ns, b12.Ns[:n12]])
    fs = np.concatenate([b16.f, b12.f[: n12 * 144]])
    order = np.random.default_rng(n16 + 10 * n12).permutation(len(Ns))
    cells = [fs[int(sum(Ns[:i] ** 2)):int(sum(Ns[:i + 1] ** 2))] for i in range(len(Ns))]
    Ns = Ns[order]
    fcat = np.concatenate([cells[i] for i in order])
    b = synth.Batch(2, 8.0, Ns, fcat)
    plans = [q.Plan(2, 16, 3, 8.0), q.Plan(2, 12, 3, 8.0)]
    for p in plans:
        p.set_tuning(threads=256, loss_fft=loss_fft, scan_j=0)
    cp = torch.tensor([0 if n == 16 else 1 for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    Q = torch.full_like(f, float("nan"))
    Q, M = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan", out=Q)
    Qn = Q.cpu().numpy().astype(np.float64)
    Mn = M.cpu().numpy()
    fin = f.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        r = oracle.q(b.cell(c, fin), 8.0, 3)
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= 1e-5, f"cell {c} (N={b.Ns[c]})"
        mref = oracle.moments(b.cell(c, Qn), 8.0)
        h2 = (16.0 / b.Ns[c]) ** 2
        assert np.allclose(Mn[c], mref, rtol=0, atol=1e-12 * h2 * np.sum(np.abs(b.cell(c, Qn))) * 64)


@pytest.mark.parametrize("n32,n24", [(1, 0), (3, 2), (4, 1)])
def test_pair32_tails_and_other_plans(q, torch, n32, n24):
    """32^2 FP32 cells go two to a CTA (128 threads each): odd counts, and
    24^2 cells drawn along, against the oracle cell by cell."""
    b32 = synth.batch_2d(n32, Ns=(32,), L=8.0, seed=80 + n32)
    b24 = synth.batch_2d(max(n24, 1), Ns=(24,), L=8.0, seed=90 + n24)
    Ns = np.concatenate([b32.Ns, b24.Ns[:n24]])
    f = np.concatenate([b32.f, b24.f[: n24 * 576]])
    b = synth.Batch(2, 8.0, Ns, f)
    plans = [q.Plan(2, 32, 8, 8.0), q.Plan(2, 24, 8, 8.0)]
    for p in plans:
        p.set_tuning(threads=256, loss_fft=2, scan_j=0)
    cp = torch.tensor([0 if n == 32 else 1 for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    ft = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    Q, M = q.qdvm_eval_batched(plans, cp, co, ft, "f32_kahan")
    Qn = Q.cpu().numpy().astype(np.float64)
    Mn = M.cpu().numpy()
    fin = ft.cpu().numpy().astype(np.float64)
    for c in range(b.n_cells):
        r = oracle.q(b.cell(c, fin), 8.0, 8)
        assert oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]) <= 1e-5, f"cell {c} (N={b.Ns[c]})"
        h2 = (16.0 / b.Ns[c]) ** 2
        mref = oracle.moments(b.cell(c, Qn), 8.0)
        assert np.allclose(Mn[c], mref, rtol=0, atol=1e-12 * h2 * np.sum(np.abs(b.cell(c, Qn))) * 64)


def test_batched_results_repeat_bit_for_bit(q, torch):
    """The 4096-cell mixed batch evaluated three times: Q and the moments are
    identical bit for bit, whichever CTA draws which cell (the persistent
    schedule is a race on an atomic counter; a cell's arithmetic must not
    depend on it)."""
    Ns = (16, 32, 48, 64)
    b = synth.batch_2d(4096, Ns=Ns, L=8.0, seed=0)
    plans = [q.Plan(2, n, 8, 8.0, kernel="unit") for n in Ns]
    for p in plans:
        p.set_tuning(threads=256, loss_fft=2, scan_j=0)
    cp, co, f = _batch_tensors(torch, b, Ns, "f32_kahan")
    runs = [q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan") for _ in range(3)]
    for Q, M in runs[1:]:
        assert torch.equal(Q, runs[0][0]) and torch.equal(M, runs[0][1])


def test_schedule_order(q, torch):
    """The order in which the persistent evaluator draws cells, read back from
    the workspace (a 256-byte counter, then one int per cell): plans by
    decreasing cost (N^2 x lines, ties by plan index), cells ascending within
    a plan, out-of-range plan indices left out, the tail -1.  5000 cells (more
    chunks of 1024 than the schedule keeps in registers), five plans, the
    indices -1 and 5 mixed in."""
    Ns = (8, 12, 16, 10, 14)
    plans = [q.Plan(2, n, 2, 8.0) for n in Ns]
    rng = np.random.default_rng(11)
    n_cells = 5000
    cpn = rng.integers(-1, len(Ns) + 1, size=n_cells).astype(np.int32)
    sizes = np.array([Ns[c] ** 2 if 0 <= c < len(Ns) else 64 for c in cpn], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    f = torch.rand(int(sizes.sum()), dtype=torch.float32, device="cuda")
    cp = torch.tensor(cpn, device="cuda")
    co = torch.tensor(offs, device="cuda")
    ws = torch.zeros(q.batched_workspace_bytes(plans, n_cells, "f32"), dtype=torch.uint8, device="cuda")
    q.qdvm_eval_batched(plans, cp, co, f, "f32", moments=False, workspace=ws)
    torch.cuda.synchronize()
    order = ws[256:256 + 4 * n_cells].view(torch.int32).cpu().numpy()
    cost = [p.N ** 2 * p.n_lines for p in plans]
    rank = sorted(range(len(plans)), key=lambda k: -cost[k])
    ref = [i for k in rank for i in range(n_cells) if cpn[i] == k]
    ref = np.array(ref + [-1] * (n_cells - len(ref)), dtype=np.int32)
    assert np.array_equal(order, ref)
