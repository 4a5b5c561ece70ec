"""The allocation-free batched entry point (qdvm_eval_batched_noalloc).

It is meant for callers that cannot allocate device memory (a solver that
owns a fixed device budget, a plug-in inside another framework's time loop):
they pass f, Q, the cell layout and the moments array, and the library keeps
its small scratch (work counter and cell schedule) in a static device array.
This test calls it twice in a row through the C ABI and checks both results
against the FP64 oracle and against the entry point that takes a caller
workspace, at the FP32 parity bar the other tests use (1e-5 of the largest
sum of absolute terms); it checks that a call leaves the device's free memory
unchanged, the size limit, and the rejection of plans it does not cover.  It
lives in a file collected last and passes alone or after the other tests.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    import torch

    import paper_1201_3986_gb300 as q

    Ns = (16, 32, 48, 64)
    b = synth.batch_2d(40, Ns=Ns, L=8.0, seed=21)
    plans = [q.Plan(2, n, 8, 8.0, kernel="hp") for n in Ns]
    cp = torch.tensor([Ns.index(int(n)) for n in b.Ns], dtype=torch.int32, device="cuda")
    co = torch.tensor(b.offsets, dtype=torch.int64, device="cuda")
    f = torch.tensor(b.f, dtype=torch.float32, device="cuda")
    Q_ref, M_ref = q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan")
    Q_ref = Q_ref.cpu().numpy().astype(np.float64)
    M_ref = M_ref.cpu().numpy()
    fin = f.cpu().numpy().astype(np.float64)
    refs = [oracle.q(b.cell(c, fin), 8.0, 8, kernel="hp") for c in range(b.n_cells)]
    scales = [np.max(r["scale"]) for r in refs]
    Q = torch.full_like(f, float("nan"))
    M = torch.full((b.n_cells, 4), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        Q.fill_(float("nan"))
        M.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        q.qdvm_eval_batched_noalloc(plans, cp, co, f, Q, M, "f32_kahan")
        torch.cuda.synchronize()
        if call == 1:  # the first call may load the library's kernels; later calls must not allocate
            assert torch.cuda.mem_get_info()[0] == free0, "the call changed the device's free memory"
        Qn = Q.cpu().numpy().astype(np.float64)
        Mn = M.cpu().numpy()
        assert np.all(np.isfinite(Qn)) and np.all(np.isfinite(Mn)), f"call {call}: unwritten outputs"
        for c in range(b.n_cells):
            err = np.max(np.abs(b.cell(c, Qn) - refs[c]["Q"])) / scales[c]
            assert err <= 1e-5, f"call {call}, cell {c}: {err:.3e} against the oracle"
            err = np.max(np.abs(b.cell(c, Qn) - b.cell(c, Q_ref))) / scales[c]
            assert err <= 1e-5, f"call {call}, cell {c}: {err:.3e} against qdvm_eval_batched"
            h2 = (16.0 / b.Ns[c]) ** 2
            assert np.all(np.abs(Mn[c] - M_ref[c]) <= 1e-5 * h2 * scales[c] * b.Ns[c] ** 2)


def test_noalloc_rejects_oversized_batch_and_uncovered_plans():
    import torch

    import paper_1201_3986_gb300 as q

    plans = [q.Plan(2, 16, 3, 8.0)]
    n = q.QDVM_NOALLOC_MAX_CELLS + 1
    cp = torch.zeros(n, dtype=torch.int32, device="cuda")
    co = torch.zeros(n, dtype=torch.int64, device="cuda")
    f = torch.zeros(256, dtype=torch.float32, device="cuda")
    Q = torch.zeros_like(f)
    with pytest.raises(q.QdvmError) as ei:
        q.qdvm_eval_batched_noalloc(plans, cp, co, f, Q, None, "f32")
    assert ei.value.status == 1 and "QDVM_NOALLOC_MAX_CELLS" in str(ei.value)
    plans3 = [q.Plan(3, 16, 2, 6.0)]
    cp1, co1 = cp[:1].contiguous(), co[:1].contiguous()
    f3 = torch.zeros(16 ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(q.QdvmError) as ei:
        q.qdvm_eval_batched_noalloc(plans3, cp1, co1, f3, torch.zeros_like(f3), None, "f32")
    assert ei.value.status == 2
