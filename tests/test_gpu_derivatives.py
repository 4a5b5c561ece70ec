"""GPU JVP / VJP of Q (through the C ABI) against the oracle's term-by-term
derivative, finite differences and the transpose identity; the
torch.autograd.Function built on them."""
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


def _t(torch, a, prec):
    return torch.tensor(a, dtype=torch.float64 if prec == "f64" else torch.float32, device="cuda")


def _r(a, prec):
    return a if prec == "f64" else a.astype(np.float32).astype(np.float64)


CASES = [
    # d, N, L, Nbar, Ntilde
    (2, 16, 8.0, 3, None),
    (2, 20, 5.0, 4, None),
    (2, 12, 3.0, 2, 3),
    (3, 8, 3.0, 1, None),
    (3, 12, 6.0, 2, None),
    (3, 16, 6.0, 3, None),
]


@pytest.mark.parametrize("case", CASES, ids=[f"d{c[0]}N{c[1]}Nb{c[3]}" for c in CASES])
@pytest.mark.parametrize("prec", ["f64", "f32", "f32_kahan"])
@pytest.mark.parametrize("kernel", ["unit", "hp"])
def test_jvp_vjp_parity(q, torch, case, prec, kernel):
    d, N, L, Nbar, Nt = case
    rs = np.random.default_rng(N + 7 * d)
    f = _r(rs.uniform(0.05, 1.0, (N,) * d), prec)
    dl = _r(rs.standard_normal((N,) * d), prec)
    g = _r(rs.standard_normal((N,) * d), prec)
    plan = q.Plan(d, N, Nbar, L, kernel=kernel, Ntilde=Nt)
    J = q.qdvm_jvp(plan, _t(torch, f, prec), _t(torch, dl, prec), prec).cpu().numpy().astype(np.float64)
    G = q.qdvm_vjp(plan, _t(torch, f, prec), _t(torch, g, prec), prec).cpu().numpy().astype(np.float64)
    Jr, Js = oracle.jvp_points(f, dl, L, Nbar, kernel=kernel, Ntilde=Nt)
    Gr, Gs = oracle.vjp(f, g, L, Nbar, kernel=kernel, Ntilde=Nt, with_scale=True)
    ej = np.max(np.abs(J - Jr)) / np.max(Js)
    eg = np.max(np.abs(G - Gr)) / np.max(Gs)
    assert ej <= TOL[prec], f"jvp {ej:.3e}"
    assert eg <= TOL[prec], f"vjp {eg:.3e}"


@pytest.mark.parametrize("d,N,Nbar", [(2, 16, 3), (3, 12, 2)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_integer_data_bit_exact(q, torch, d, N, Nbar, prec):
    rs = np.random.default_rng(3)
    f = rs.integers(0, 3, (N,) * d).astype(np.float64)
    dl = rs.integers(-2, 3, (N,) * d).astype(np.float64)
    g = rs.integers(-2, 3, (N,) * d).astype(np.float64)
    plan = q.Plan(d, N, Nbar, 3.0, kernel="unit")
    J = q.qdvm_jvp(plan, _t(torch, f, prec), _t(torch, dl, prec), prec).cpu().numpy().astype(np.float64)
    G = q.qdvm_vjp(plan, _t(torch, f, prec), _t(torch, g, prec), prec).cpu().numpy().astype(np.float64)
    assert np.array_equal(J, oracle.jvp(f, dl, 3.0, Nbar, kernel="unit"))
    assert np.array_equal(G, oracle.vjp(f, g, 3.0, Nbar, kernel="unit"))


@pytest.mark.parametrize("d,N,Nbar", [(2, 32, 5), (3, 16, 3)])
def test_central_difference_and_transpose_identity(q, torch, d, N, Nbar):
    """Q is quadratic: (Q(f+hd) - Q(f-hd)) / 2h is the JVP up to rounding
    (FP32, h = 1e-3: bar 1e-3 of the JVP scale), and <g, J d> = <J^T g, d>."""
    rs = np.random.default_rng(11)
    L = 6.0
    f = synth.mixture(d, N, L, rs).astype(np.float32).astype(np.float64)
    dl = (rs.standard_normal((N,) * d) * np.max(f)).astype(np.float32).astype(np.float64)
    g = rs.standard_normal((N,) * d).astype(np.float32).astype(np.float64)
    plan = q.Plan(d, N, Nbar, L, kernel="hp")
    h = 1e-3
    qp = q.qdvm_eval(plan, _t(torch, f + h * dl, "f32"), "f32").double()
    qm = q.qdvm_eval(plan, _t(torch, f - h * dl, "f32"), "f32").double()
    fd = ((qp - qm) / (2 * h)).cpu().numpy()
    J = q.qdvm_jvp(plan, _t(torch, f, "f32"), _t(torch, dl, "f32"), "f32").cpu().numpy().astype(np.float64)
    _, Js = oracle.jvp_points(f, dl, L, Nbar, kernel="hp")
    assert np.max(np.abs(fd - J)) / np.max(Js) <= 1e-3
    # transpose identity in FP64
    J64 = q.qdvm_jvp(plan, _t(torch, f, "f64"), _t(torch, dl, "f64"), "f64").cpu().numpy()
    G64 = q.qdvm_vjp(plan, _t(torch, f, "f64"), _t(torch, g, "f64"), "f64").cpu().numpy()
    lhs, rhs = float(np.sum(g * J64)), float(np.sum(G64 * dl))
    assert abs(lhs - rhs) <= 1e-12 * float(np.sum(np.abs(g) * Js))


def test_autograd_function(q, torch):
    N = 10
    plan = q.Plan(2, N, 2, 3.0, kernel="hp")
    rs = np.random.default_rng(5)
    f = torch.tensor(rs.uniform(0.1, 1.0, (N, N)), dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: q.collision(x, plan, "f64"), (f,), eps=1e-6, atol=1e-8, rtol=1e-6)
    g = torch.tensor(rs.standard_normal((N, N)), dtype=torch.float64, device="cuda")
    (gr,) = torch.autograd.grad((q.collision(f, plan, "f64") * g).sum(), f)
    ref = oracle.vjp(f.detach().cpu().numpy(), g.cpu().numpy(), 3.0, 2, kernel="hp")
    assert np.allclose(gr.cpu().numpy(), ref, rtol=1e-11, atol=1e-14)


def _sample_idx(N, d, n, seed):
    rng = np.random.default_rng(seed)
    idx = rng.choice(N ** d, size=n, replace=False)
    return np.unique(np.concatenate([idx, [0, N ** d - 1]])).astype(np.int64)


@pytest.mark.parametrize("op", ["jvp", "vjp"])
def test_batched_3d_N32_workload_sampled(q, torch, op):
    """256 cells of 32^3, Nbar = 5, hard spheres, FP32, Gaussian tangents /
    cotangents (seed 2): sampled cells and points against the oracle."""
    b = synth.batch_3d(256, N=32, L=6.0, seed=1)
    a = synth.gaussian(b.f.shape, seed=2)
    plans = [q.Plan(3, 32, 5, 6.0, kernel="hp")]
    cp = torch.zeros(b.n_cells, dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    at = torch.tensor(a, dtype=torch.float32, device="cuda")
    fn = q.qdvm_jvp_batched if op == "jvp" else q.qdvm_vjp_batched
    out = fn(plans, cp, co, f, at, "f32").cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    ain = at.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(out))
    for c in (0, 131, 255):
        idx = _sample_idx(32, 3, 40, c)
        ref_fn = oracle.jvp_points if op == "jvp" else oracle.vjp_points
        r, s = ref_fn(b.cell(c, fin), b.cell(c, ain), 6.0, 5, idx, kernel="hp")
        err = np.max(np.abs(b.cell(c, out).ravel()[idx] - r)) / np.max(s)
        assert err <= 1e-5, f"cell {c}: {err:.3e}"


def test_batched_2d_mixed_every_cell(q, torch):
    Ns = (16, 24)
    b = synth.batch_2d(6, Ns=Ns, L=8.0, seed=12)
    g = synth.gaussian(b.f.shape, seed=13)
    plans = [q.Plan(2, n, 3, 8.0, kernel="unit") for n in Ns]
    cp = torch.tensor([Ns.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float64, device="cuda")
    gt = torch.tensor(g, dtype=torch.float64, device="cuda")
    G = q.qdvm_vjp_batched(plans, cp, co, f, gt, "f64").cpu().numpy()
    J = q.qdvm_jvp_batched(plans, cp, co, f, gt, "f64").cpu().numpy()
    for c in range(b.n_cells):
        Gr, Gs = oracle.vjp(b.cell(c), b.cell(c, g), 8.0, 3, with_scale=True)
        assert np.max(np.abs(b.cell(c, G) - Gr)) / np.max(Gs) <= 1e-12
        Jr, Js = oracle.jvp_points(b.cell(c), b.cell(c, g), 8.0, 3)
        assert np.max(np.abs(b.cell(c, J) - Jr)) / np.max(Js) <= 1e-12


@pytest.mark.parametrize("loss_fft", [0, 1])
def test_config5_central_difference_N32(q, torch, loss_fft):
    """The adjoint workload at its own size: 256 cells of 32^3, Nbar = 5, hard
    spheres, FP32, Gaussian tangents and cotangents (seeds 2 and 3).  Q is
    quadratic (eq. (DR)), so the central difference (Q(f + h d) - Q(f - h d)) / 2h
    of the batched evaluation equals the batched JVP up to rounding
    (h = 1e-3: bar 1e-3 of the JVP's term scale) on three cells, and
    <g, J d> = <J^T g, d> holds for the batched VJP on the same cells to
    FP32 rounding.  The term scale is the oracle's at 200 sampled points
    (a lower bound of its maximum, so the bar only gets stricter)."""
    b = synth.batch_3d(256, N=32, L=6.0, seed=1)
    dl = synth.gaussian(b.f.shape, seed=2)
    g = synth.gaussian(b.f.shape, seed=3)
    plan = q.Plan(3, 32, 5, 6.0, kernel="hp")
    plan.set_tuning(loss_fft=loss_fft)
    cp = torch.zeros(b.n_cells, dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    d = torch.tensor(dl, dtype=torch.float32, device="cuda")
    gt = torch.tensor(g, dtype=torch.float32, device="cuda")
    h = 1e-3
    qp, _ = q.qdvm_eval_batched([plan], cp, co, f + h * d, "f32", moments=False)
    qm, _ = q.qdvm_eval_batched([plan], cp, co, f - h * d, "f32", moments=False)
    fd = ((qp.double() - qm.double()) / (2 * h)).cpu().numpy()
    J = q.qdvm_jvp_batched([plan], cp, co, f, d, "f32").cpu().numpy().astype(np.float64)
    G = q.qdvm_vjp_batched([plan], cp, co, f, gt, "f32").cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    din = d.cpu().numpy().astype(np.float64)
    gin = gt.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(fd)) and np.all(np.isfinite(J)) and np.all(np.isfinite(G))
    for c in (0, 97, 255):
        idx = _sample_idx(32, 3, 200, c)
        _, Js = oracle.jvp_points(b.cell(c, fin), b.cell(c, din), 6.0, 5, idx, kernel="hp")
        _, Gs = oracle.vjp_points(b.cell(c, fin), b.cell(c, gin), 6.0, 5, idx, kernel="hp")
        err = np.max(np.abs(b.cell(c, fd) - b.cell(c, J))) / np.max(Js)
        assert err <= 1e-3, f"cell {c}: FD vs JVP {err:.3e}"
        lhs = float(np.sum(b.cell(c, gin) * b.cell(c, J)))
        rhs = float(np.sum(b.cell(c, G) * b.cell(c, din)))
        bound = 1e-5 * (float(np.sum(np.abs(b.cell(c, gin)))) * np.max(Js)
                        + float(np.sum(np.abs(b.cell(c, din)))) * np.max(Gs))
        assert abs(lhs - rhs) <= bound, f"cell {c}: <g, J d> = {lhs:.6e}, <J^T g, d> = {rhs:.6e}"


def test_autograd_gradcheck_3d(q, torch):
    """torch.autograd.gradcheck of the differentiable Q in FP64 on a 3D 8^3
    cell (hard spheres, Nbar = 2): the backward (qdvm_vjp) against numerical
    Jacobian columns of the forward, and the VJP against the oracle's."""
    N = 8
    plan = q.Plan(3, N, 2, 3.0, kernel="hp")
    rs = np.random.default_rng(9)
    f = torch.tensor(rs.uniform(0.1, 1.0, (N,) * 3), dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: q.collision(x, plan, "f64"), (f,), eps=1e-6, atol=1e-8, rtol=1e-6)
    g = torch.tensor(rs.standard_normal((N,) * 3), dtype=torch.float64, device="cuda")
    (gr,) = torch.autograd.grad((q.collision(f, plan, "f64") * g).sum(), f)
    ref = oracle.vjp(f.detach().cpu().numpy(), g.cpu().numpy(), 3.0, 2, kernel="hp")
    assert np.allclose(gr.cpu().numpy(), ref, rtol=1e-11, atol=1e-14)
