"""Benchmark of the batched fast-summation collision operator.

Workload (one step): evaluate Q(f) on 4096 independent 2D cells with N drawn
uniformly from {16, 32, 48, 64} (seed 0), L = 8, Nbar = 8, unit kernel,
each cell a two-Maxwellian mixture (random drifts in [-1,1]^2, temperatures
in [0.5, 2]), FP32 arithmetic with compensated direction sums, plus the FP64
moments (mass, momentum, energy) of every cell -- one persistent launch.

Metric: Q evaluations per second counted in grid points, sum_cells N^d per
second (whole job over all ranks).  Device time of exactly K steps between
CUDA events, after W warm-up steps; 6 rotating copies of the batch (inputs +
outputs 377 MB > 129 MB L2) so no step reads its inputs from L2.

Also reported: an end-to-end figure through the public API with host
buffers (pinned host -> device copy of f, evaluation, device -> host copy of
Q and moments inside the timed region), the roofline of the dominant kernel,
the plain single-cell FP64 GPU evaluation, the accuracy against the FP64
oracle on sampled cells, the CPU oracle timed on the host cores, and the SM
clocks sampled during the timed region.

``--impl reference`` times the CPU oracle (the reference implementation of
the method: direct FP64 sum) on a bounded sample of the same workload.
Multi-GPU (torchrun): independent replicas, one batch per rank, no
collective in the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Q evals/s (cells×N^d pts/s) vs plain FP64 GPU; %HBM roofline; rel L∞ err vs FP64 oracle"
UNIT = "pts/s"
NS = (16, 32, 48, 64)
N_CELLS = 4096
NBAR = 8
L = 8.0
ROTATE = 6
FLOPS_PER_POINT_PAIR = 10  # running windows W_e, W_e^perp, V_e (2 each) + assembly (4)
ACCURACY_CELLS_PER_N = 4  # accuracy leg: cells per size checked against the oracle in full
DEFECT_BAR = 1e-6  # |defect_gpu - defect_oracle64| per phi (FP32 path)
ORACLE_SAMPLE_CELLS = 1024  # CPU baseline: ~10-30 s of oracle work
REF_STEP_CELLS = 96  # reference arm: one step = the first 96 cells (~1 s)


def workload_config(extra=None):
    ns = ",".join(str(n) for n in NS)
    cfg = {"workload": f"batched 2D DVM Q: {N_CELLS} cells, N~U{{{ns}}} (seed 0), L={L:g}, Nbar={NBAR}, unit kernel, "
                       "two-Maxwellian mixtures, FP32 + compensated direction sums, FP64 moments",
           "n_cells": N_CELLS, "Ns": list(NS), "Nbar": NBAR, "L": L, "prec": "f32_kahan",
           "l2": f"{ROTATE} rotating input/output batch copies (> 129 MB L2)"}
    if extra:
        cfg.update(extra)
    return cfg


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


PROFILE = os.path.join(ROOT, "profiles", "k_fused2d_batched__batch2d_4096cells.md")
KERNEL_SOURCES = ["paper_1201_3986_gb300/csrc/fused2d.cuh", "paper_1201_3986_gb300/csrc/fused2d_f32k.cu",
                  "paper_1201_3986_gb300/csrc/fft.cuh", "paper_1201_3986_gb300/csrc/qdvm_internal.cuh"]


def kernel_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


PROFILE_KEYS = ("source_sha256:", "dram_bytes_per_launch:", "smem_wavefronts_per_launch:", "launch_tuning:")


def profiled_fields() -> dict:
    """The key: value lines of the committed ncu summary of the evaluator, or
    {} when the kernel sources changed since it was captured."""
    if not os.path.exists(PROFILE):
        return {}
    vals = {}
    for line in open(PROFILE):
        t = line.strip().lstrip("-").strip().strip("`")
        if t.startswith(PROFILE_KEYS):
            k, v = t.split(":", 1)
            vals[k.strip()] = v.split("`")[0].split("(")[0].strip()
    return vals if vals.get("source_sha256") == kernel_source_hash() else {}


def profiled_value(key: str):
    """A per-launch count of the evaluator from the committed ncu summary
    (dram_bytes_per_launch, smem_wavefronts_per_launch), or None when the
    kernel sources changed since it was captured."""
    try:
        return int(profiled_fields()[key])
    except (KeyError, ValueError):
        return None


def effective_tuning(t: dict, ntilde: int) -> tuple:
    """(threads, direct_j, loss_fft, scan_j) with the parameters that select
    no different code for this plan set to their neutral values: direct_j
    only matters with the direct loss (loss_fft 0), scan_j only when it
    reaches a pair of the cell (1 <= scan_j <= Ntilde) and the loss is an FFT."""
    fft = t["loss_fft"]
    dj = t["direct_j"] if fft == 0 else 2
    sj = t["scan_j"] if fft > 0 and 1 <= t["scan_j"] <= ntilde else 0
    return t["threads"], dj, fft, sj


def tuning_key(tunings: dict, ntildes: dict | None = None) -> str:
    """The launch configuration of a batched 2D call as one string: per cell
    size N, the plan's threads,direct_j,loss_fft,scan_j (each cell runs with
    its own plan's parameters), normalised by effective_tuning when the
    plans' Ntilde are given."""
    out = []
    for n, t in sorted(tunings.items()):
        v = effective_tuning(t, ntildes[n]) if ntildes else (t["threads"], t["direct_j"], t["loss_fft"], t["scan_j"])
        out.append(f"{n}=" + ",".join(str(x) for x in v))
    return " ".join(out)


def profiled_tuning():
    """The launch configuration (tuning_key) of the profiled launch, or None."""
    return profiled_fields().get("launch_tuning")


def profiled_traffic(key=None):
    """DRAM bytes per launch of the profiled launch configuration (None for
    another configuration or changed sources)."""
    pt = profiled_tuning()
    if pt is None or key != pt:
        return None
    return profiled_value("dram_bytes_per_launch")


def smem_roofline(kernel_ms: float, clocks: dict, key, n_sm: int = 152):
    """The evaluator's binding resource: shared-memory wavefronts (the LSU
    pipe serves one per SM and cycle).  Wavefronts per launch from the ncu
    summary (they depend on the code, the workload and the launch
    configuration, not on timing) over the live kernel time, the device's
    SMs and the SM clock sampled in the timed region; None when the
    configuration is not the profiled one."""
    wf = profiled_value("smem_wavefronts_per_launch")
    mhz = clocks.get("sm_mhz") or 2070.0
    pt = profiled_tuning()
    if wf is None or pt is None or key != pt or NS != (16, 32, 48, 64) or NBAR != 8:
        return None
    per_cycle = wf / (kernel_ms / 1e3 * n_sm * mhz * 1e6)
    return {"bound": "smem", "achieved": per_cycle, "peak": 1.0, "unit": "wavefronts/cycle/SM",
            "frac": per_cycle, "wavefronts_per_launch": wf, "sm_mhz": mhz}


def set_tunings(plans, spec: str) -> None:
    """Pin the launch configuration from the command line: one
    threads,direct_j,loss_fft[,scan_j] for every plan, or per cell size
    N=threads,direct_j,loss_fft,scan_j entries separated by spaces or ';'."""
    entries = spec.replace(";", " ").split()
    per = {}
    for ent in entries:
        if "=" in ent:
            n, v = ent.split("=", 1)
            per[int(n)] = v
    for p in plans:
        v = per.get(p.N, entries[0] if not per else None)
        if v is None:
            continue
        vals = [int(x) for x in v.split(",")]
        p.set_tuning(threads=vals[0], direct_j=vals[1], loss_fft=vals[2], scan_j=vals[3] if len(vals) > 3 else None)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def combine_ranks(ms_local: float, pts_per_rank: int, steps: int, dist=None, device=None):
    """Whole-job figure of independent replicas: the step time is the max over
    ranks (the slowest replica bounds the job) and the value counts the
    points all ranks processed.  ``dist`` is torch.distributed (or None for a
    single process); ``device`` holds the reduction tensor (cuda for NCCL,
    cpu for gloo)."""
    import torch

    ws = 1
    ms = float(ms_local)
    if dist is not None and dist.is_initialized():
        ws = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = ws * pts_per_rank * steps / (ms / 1e3)
    return ms, value, ws


def fp32_peak_tflops(n_sm: int, clocks: dict):
    """FP32 FMA peak of the device: SMs x 128 FP32 lanes x 2 flops x the SM
    clock sampled under load in the timed region (the maximum clock when no
    sample is available)."""
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    peak = n_sm * 128 * 2 * mhz * 1e6 / 1e12
    return peak, f"FP32 peak = {n_sm} SMs x 128 lanes x 2 x {mhz:.0f} MHz (sampled SM clock)"


def phi_arrays(d: int, N: int, L: float):
    """phi = 1, v_0..v_{d-1}, |v|^2 on the vertex grid v = -L + j h."""
    v = -L + np.arange(N) * (2.0 * L / N)
    g = np.meshgrid(*([v] * d), indexing="ij")
    return [np.ones((N,) * d)] + list(g) + [sum(x * x for x in g)]


def accuracy_leg(b, Qn: np.ndarray, Mn: np.ndarray) -> dict:
    """Accuracy of one evaluated batch (host copies of Q and the moments)
    against the FP64 oracle.

    On ACCURACY_CELLS_PER_N cells of every size: the relative L-inf error
    max|Q - Q_ref| / max scale_ref, and the conservation defects per phi
    (mass, momentum, energy), defect = |h^d sum Q phi| / (h^d sum scale |phi|),
    for the GPU moments and for the oracle's Q, with the largest
    |defect_gpu - defect_oracle| (bar DEFECT_BAR).  On every cell: the mass
    defect |m_0| / (h^d sum scale), with sum scale = 2 sum_m K(m) R(m) from
    the displacement histogram K of the terms and the autocorrelation R of f
    (f >= 0)."""
    import oracle

    f32 = b.f.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(1)
    picks = []
    for n in NS:
        picks += [int(c) for c in rng.choice(np.nonzero(b.Ns == n)[0], size=ACCURACY_CELLS_PER_N, replace=False)]
    names = ("mass", "momentum", "energy")
    errs, dg_max, dr_max, dd_max = [], dict.fromkeys(names, 0.0), dict.fromkeys(names, 0.0), dict.fromkeys(names, 0.0)
    for c in picks:
        fc = b.cell(c, f32)
        N = fc.shape[0]
        r = oracle.q(fc, L, NBAR)
        errs.append(oracle.rel_linf(b.cell(c, Qn), r["Q"], r["scale"]))
        h2 = (2 * L / N) ** 2
        den = np.array([h2 * np.sum(r["scale"] * np.abs(p)) for p in phi_arrays(2, N, L)])
        dg = np.abs(Mn[c]) / den
        dr = np.abs(oracle.moments(r["Q"], L)) / den
        dd = np.abs(dg - dr)
        for k, nm in ((0, "mass"), (1, "momentum"), (2, "momentum"), (3, "energy")):
            dg_max[nm] = max(dg_max[nm], float(dg[k]))
            dr_max[nm] = max(dr_max[nm], float(dr[k]))
            dd_max[nm] = max(dd_max[nm], float(dd[k]))
    hist = {}
    for n in NS:
        Nt = oracle.default_ntilde(n)
        K = np.zeros((n, n))
        for e in oracle.lines(2, min(NBAR, Nt)):
            J = Nt // int(np.max(np.abs(e)))
            ep = np.array([-e[1], e[0]])
            js = [j for j in range(-J, J + 1) if j]
            for j in js:
                for jp in js:
                    m = (j * e + jp * ep) % n
                    K[m[0], m[1]] += 1
        hist[n] = K
    mass_all = 0.0
    for c in range(b.n_cells):
        fc = b.cell(c, f32)
        N = fc.shape[0]
        F = np.fft.fft2(fc)
        R = np.fft.ifft2(np.conj(F) * F).real
        tot = 2.0 * float(np.sum(hist[N] * R))
        mass_all = max(mass_all, abs(Mn[c, 0]) / ((2 * L / N) ** 2 * tot))
    return {"rel_linf_vs_fp64_oracle_max": max(errs), "cells_checked": picks,
            "cells_checked_note": f"{ACCURACY_CELLS_PER_N} cells of each N, drawn with seed 1",
            "defect_gpu_max": dg_max, "defect_oracle64_max": dr_max, "defect_diff_max": dd_max,
            "defect_bar": DEFECT_BAR, "defect_ok": all(v <= DEFECT_BAR for v in dd_max.values()),
            "mass_defect_rel_max_all_cells": mass_all, "cells_all": int(b.n_cells)}


# ------------------------------------------------------------ CPU oracle

def oracle_sample(cells: int):
    import oracle

    b = synth.batch_2d(N_CELLS, Ns=NS, L=L, seed=0)
    n = min(cells, b.n_cells)
    f32 = b.f.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    pts = 0
    for c in range(n):
        oracle.q(b.cell(c, f32), L, NBAR)
        pts += int(b.Ns[c]) ** 2
    dt = time.perf_counter() - t0
    return pts / dt, pts, dt, oracle.max_threads(), n


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        oracle_sample(args.ref_cells)
    t_all = 0.0
    pts_all = 0
    cores = 1
    for _ in range(args.steps):
        v, pts, dt, cores, n = oracle_sample(args.ref_cells)
        vals.append(v)
        t_all += dt
        pts_all += pts
    value = pts_all / t_all
    sample = f"first {args.ref_cells} cells of the 4096-cell batch per step (same N mix), FP64 direct sum"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_all / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config({"sample_cells": args.ref_cells}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ clocks

class ClockSampler:
    def __init__(self, index: int):
        self.proc = None
        self.path = None
        self.index = index

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------ GPU arm

def run_gpu(args):
    import torch

    import paper_1201_3986_gb300 as q

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    b = synth.batch_2d(N_CELLS, Ns=NS, L=L, seed=0)
    plans = [q.Plan(2, n, NBAR, L, kernel="unit") for n in NS]
    idx = {n: i for i, n in enumerate(NS)}
    cp = torch.tensor([idx[int(n)] for n in b.Ns], dtype=torch.int32, device=dev)
    co = torch.tensor(b.offsets, dtype=torch.int64, device=dev)
    f_host = torch.from_numpy(b.f.astype(np.float32))
    fs = [f_host.to(dev) for _ in range(ROTATE)]
    Qs = [torch.empty_like(fs[0]) for _ in range(ROTATE)]
    Ms = [torch.empty((N_CELLS, 4), dtype=torch.float64, device=dev) for _ in range(ROTATE)]
    wsb = q.batched_workspace_bytes(plans, N_CELLS, "f32_kahan")
    wss = torch.empty(wsb, dtype=torch.uint8, device=dev)
    total_pts = int((b.Ns ** 2).sum())
    point_pairs = sum(int(n) ** 2 * (p.n_lines // 2) for n, p in zip(b.Ns, [plans[idx[int(n)]] for n in b.Ns]))

    # the library's autotuner picks the launch configuration on this batch;
    # each rotating buffer set is then captured once into a CUDA graph
    if args.tuning:
        set_tunings(plans, args.tuning)
    else:
        q.qdvm_tune_batched(plans, cp, co, fs[0], "f32_kahan", workspace=wss)
    tunings = {int(n): p.tuning() for n, p in zip(NS, plans)}
    key = tuning_key(tunings, {int(n): p.Ntilde for n, p in zip(NS, plans)})
    graphs = [q.BatchedGraph(plans, cp, co, fs[k], Qs[k], Ms[k], "f32_kahan", workspace=wss) for k in range(ROTATE)]

    for g in graphs:  # first replay of a graph uploads it; keep that out of the timed region
        g.launch()
    torch.cuda.synchronize(dev)

    def step(k):
        graphs[k % ROTATE].launch()

    stream = torch.cuda.current_stream(dev)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for k in range(args.steps):
            step(k)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms, value, _ = combine_ranks(e0.elapsed_time(e1), total_pts, args.steps, dist, dev)
    if dist:
        dist.barrier()
    ms_per_step = ms / args.steps
    launches = 2 * args.steps  # schedule + persistent evaluator per step

    # time of one step (schedule, 13 us, + persistent evaluator), events on the launching stream
    kt = []
    for k in range(max(3, min(args.steps, 10))):
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(k)
        z.record(stream)
        torch.cuda.synchronize(dev)
        kt.append(a.elapsed_time(z))
    kernel_ms = float(np.median(kt))

    # end to end through the public API with host buffers: every step copies
    # its input from pinned host memory and reads its Q and moments back.
    # Serial: copy in, evaluate, copy out on one stream.  Pipelined: two
    # device buffer sets; the copy-in of step k+1 and the copy-out of step
    # k-1 run on their own streams while step k evaluates.
    f_pin = f_host.pin_memory()
    Q_pin = torch.empty_like(f_pin).pin_memory()
    M_pin = torch.empty((N_CELLS, 4), dtype=torch.float64).pin_memory()
    n_e2e = max(3, min(args.steps, 20))

    def e2e_serial_step():
        fs[0].copy_(f_pin, non_blocking=True)
        q.qdvm_eval_batched(plans, cp, co, fs[0], "f32_kahan", out=Qs[0], moments=Ms[0], workspace=wss)
        Q_pin.copy_(Qs[0], non_blocking=True)
        M_pin.copy_(Ms[0], non_blocking=True)

    for _ in range(2):
        e2e_serial_step()
    torch.cuda.synchronize(dev)
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n_e2e):
        e2e_serial_step()
    z.record(stream)
    torch.cuda.synchronize(dev)
    e2e_serial_ms = a.elapsed_time(z) / n_e2e

    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def e2e_pipelined(n):
        used = [False, False]
        for k in range(n):
            bi = k % 2
            with torch.cuda.stream(s_in):
                if used[bi]:
                    s_in.wait_event(ev_done[bi])  # step k-2 has read fs[bi]
                fs[bi].copy_(f_pin, non_blocking=True)
                ev_in[bi].record(s_in)
            stream.wait_event(ev_in[bi])
            if used[bi]:
                stream.wait_event(ev_out[bi])  # Q and moments of step k-2 are on the host
            q.qdvm_eval_batched(plans, cp, co, fs[bi], "f32_kahan", out=Qs[bi], moments=Ms[bi], workspace=wss)
            ev_done[bi].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[bi])
                Q_pin.copy_(Qs[bi], non_blocking=True)
                M_pin.copy_(Ms[bi], non_blocking=True)
                ev_out[bi].record(s_out)
            used[bi] = True
        stream.wait_stream(s_out)

    e2e_pipelined(2)
    torch.cuda.synchronize(dev)
    a.record(stream)
    e2e_pipelined(n_e2e)
    z.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = a.elapsed_time(z) / n_e2e
    h2d = f_pin.numel() * 4
    d2h = Q_pin.numel() * 4 + M_pin.numel() * 8

    # plain single-cell FP64 GPU evaluation (one launch per cell, no batching)
    n_fp64 = 256
    f64_cells = [torch.tensor(b.cell(c).astype(np.float32).astype(np.float64), device=dev) for c in range(n_fp64)]
    pl = [plans[idx[int(b.Ns[c])]] for c in range(n_fp64)]
    wsf = [torch.empty(max(p.eval_workspace("f64"), 1), dtype=torch.uint8, device=dev) for p in plans]
    outs = [torch.empty_like(x) for x in f64_cells]
    for c in range(n_fp64):
        q.qdvm_eval(pl[c], f64_cells[c], "f64", out=outs[c], workspace=wsf[idx[int(b.Ns[c])]])
    torch.cuda.synchronize(dev)
    a.record(stream)
    for c in range(n_fp64):
        q.qdvm_eval(pl[c], f64_cells[c], "f64", out=outs[c], workspace=wsf[idx[int(b.Ns[c])]])
    z.record(stream)
    torch.cuda.synchronize(dev)
    fp64_pts = int((b.Ns[:n_fp64] ** 2).sum())
    fp64_value = fp64_pts / (a.elapsed_time(z) / 1e3)

    # accuracy of the timed path against the FP64 oracle (after the timed
    # region): Q and the conservation defects on cells sampled per size, the
    # mass defect on every cell
    accuracy = accuracy_leg(b, Qs[0].cpu().numpy().astype(np.float64), Ms[0].cpu().numpy())

    hbm_peak, peak_kind = peaks()
    alg_bytes = total_pts * (4 + 4) + N_CELLS * 4 * 8
    achieved_gbs = alg_bytes / (kernel_ms / 1e3) / 1e9
    alg_flops = FLOPS_PER_POINT_PAIR * point_pairs
    clocks = clk.summary()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_peak_tflops, peak_note = fp32_peak_tflops(n_sm, clocks)
    achieved_tflops = alg_flops / (kernel_ms / 1e3) / 1e12

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": workload_config({"parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                                   "tuning": key, "launch": "CUDA graph (schedule + persistent evaluator)"}),
        "e2e": {"value": total_pts / (e2e_ms / 1e3) * ws, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "pipelined": "two device buffer sets; copy-in of step k+1 and copy-out of step k-1 on their own "
                             "streams overlap step k", "serial_ms_per_step": e2e_serial_ms},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": sm_peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved_tflops / sm_peak_tflops, "traffic": profiled_traffic(key),
                     "kernel": "k_fused2d_batched", "kernel_ms": kernel_ms,
                     "note": f"{peak_note}; algorithmic flops = {FLOPS_PER_POINT_PAIR} per point-pair x "
                             f"{point_pairs} point-pairs"},
        "roofline_smem": smem_roofline(kernel_ms, clocks, key, n_sm),
        "roofline_hbm": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved_gbs / hbm_peak, "peak_kind": f"of {peak_kind}",
                         "alg_bytes": alg_bytes},
        "fp64_single_cell": {"value": fp64_value, "unit": UNIT, "cells": n_fp64,
                             "speedup_of_batched_f32": value / ws / fp64_value},
        "accuracy": accuracy,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        v, pts, dt, cores, n = oracle_sample(args.ref_cells)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"first {n} cells of the batch ({pts} points, {dt:.1f} s), FP64 direct sum"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_rk2_workload(args):
    """Time stepping: the 4096-cell batched 2D workload advanced by
    args.rk2_steps second-order TVD Runge-Kutta steps (two Q evaluations
    each) per CUDA-graph launch, on 6 rotating batch copies (> L2).  The
    value counts Q evaluations per second, like the default workload."""
    import torch

    import oracle
    import paper_1201_3986_gb300 as q

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    K = args.rk2_steps
    dt = 0.002
    b = synth.batch_2d(N_CELLS, Ns=NS, L=L, seed=0)
    plans = [q.Plan(2, n, NBAR, L, kernel="unit") for n in NS]
    idx = {n: i for i, n in enumerate(NS)}
    cp = torch.tensor([idx[int(n)] for n in b.Ns], dtype=torch.int32, device=dev)
    co = torch.tensor(b.offsets, dtype=torch.int64, device=dev)
    f_host = torch.from_numpy(b.f.astype(np.float32))
    fs = [f_host.to(dev) for _ in range(ROTATE)]
    q.qdvm_tune_batched(plans, cp, co, fs[0], "f32_kahan",
                        workspace=torch.empty(q.batched_workspace_bytes(plans, N_CELLS, "f32_kahan"),
                                              dtype=torch.uint8, device=dev))
    tuning = tuning_key({p.N: p.tuning() for p in plans})
    wsb = q.rk2_workspace_bytes(plans, N_CELLS, b.total, "f32_kahan")
    wss = [torch.empty(wsb, dtype=torch.uint8, device=dev) for _ in range(ROTATE)]
    Ms = [torch.empty((N_CELLS, 4), dtype=torch.float64, device=dev) for _ in range(ROTATE)]
    graphs = [q.RK2Graph(plans, cp, co, fs[k], dt, K, "f32_kahan", moments=Ms[k], workspace=wss[k])
              for k in range(ROTATE)]
    for g in graphs:
        g.launch()
    torch.cuda.synchronize(dev)
    for k in range(ROTATE):
        fs[k].copy_(f_host.to(dev))
    _, m0 = q.qdvm_rk2_batched(plans, cp, co, fs[0].clone(), dt, 0, "f32_kahan", moments=True)
    stream = torch.cuda.current_stream(dev)
    for k in range(args.warmup):
        graphs[k % ROTATE].launch()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        e0.record(stream)
        for k in range(args.steps):
            graphs[(args.warmup + k) % ROTATE].launch()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    # accuracy: one step of the first cell of each size against the oracle's stepping
    errs = []
    for n in NS:
        c = int(np.nonzero(b.Ns == n)[0][0])
        f0 = b.cell(c, b.f.astype(np.float32).astype(np.float64))
        ft = torch.tensor(f0, dtype=torch.float32, device=dev).reshape(-1)
        q.qdvm_rk2_batched([plans[idx[n]]], torch.zeros(1, dtype=torch.int32, device=dev),
                           torch.zeros(1, dtype=torch.int64, device=dev), ft, dt, 1, "f32_kahan")
        ref = oracle.rk2(f0, L, NBAR, dt, 1)
        sc = np.max(np.abs(f0)) + dt * np.max(oracle.q(f0, L, NBAR)["scale"])
        errs.append(float(np.max(np.abs(ft.cpu().numpy().reshape(f0.shape) - ref)) / sc))
    # mass of graph 0's batch after all its replays, against the start
    m_end = graphs[0].moments.cpu().numpy()
    m_start = m0.cpu().numpy()
    mass_defect = float(np.max(np.abs(m_end[:, 0] - m_start[:, 0]) / np.abs(m_start[:, 0])))
    evals = 2 * K * b.total
    line = {"metric": METRIC, "value": evals / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"time stepping: 4096-cell batched 2D workload (N~U{{16,32,48,64}}, Nbar=8, "
                                   f"seed 0), {K} TVD-RK2 steps of dt={dt} per graph launch (2 Q evaluations per "
                                   "step), FP32 state + compensated Q sums",
                       "rk2_steps_per_launch": K, "tuning": tuning,
                       "l2": "6 rotating batch copies with their own workspaces (> 129 MB L2)"},
            "rk2_ms_per_time_step": ms / K,
            "accuracy": {"one_step_rel_err_vs_fp64_oracle_rk2": max(errs), "mass_defect_rel": mass_defect},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_adaptive_workload(args):
    """Space-dependent Nbar on a 4096-cell 2D batch at various distances from
    equilibrium (synth.batch_2d_relaxing): each step computes the per-cell
    equilibrium indicator, selects Nbar in {2, 4, 8} with thresholds
    (0.02, 0.1) and evaluates the batch; one CUDA graph per rotating batch
    copy.  Compared with the fixed Nbar = 8 evaluation of the same batch."""
    import torch

    import oracle
    import paper_1201_3986_gb300 as q

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    nbars, thr = (2, 4, 8), (0.02, 0.1)
    b = synth.batch_2d_relaxing(N_CELLS, Ns=NS, L=L, seed=3)
    plans = [q.Plan(2, n, nb, L, kernel="unit") for n in NS for nb in nbars]
    level_plan = np.arange(len(plans)).reshape(len(NS), len(nbars))
    idx = {n: i for i, n in enumerate(NS)}
    cb = torch.tensor([idx[int(n)] for n in b.Ns], dtype=torch.int32, device=dev)
    co = torch.tensor(b.offsets, dtype=torch.int64, device=dev)
    f_host = torch.from_numpy(b.f.astype(np.float32))
    fs = [f_host.to(dev) for _ in range(ROTATE)]
    eps = [torch.empty(N_CELLS, dtype=torch.float64, device=dev) for _ in range(ROTATE)]
    cps = [torch.empty(N_CELLS, dtype=torch.int32, device=dev) for _ in range(ROTATE)]
    Qs = [torch.empty_like(fs[0]) for _ in range(ROTATE)]
    base = plans[::len(nbars)]  # one plan per N: the indicator needs each cell's N and L
    q.equilibrium_distance(base, cb, co, fs[0], "f32_kahan", out=eps[0])
    q.select_levels(eps[0], cb, thr, level_plan, out=cps[0])
    wsb = q.batched_workspace_bytes(plans, N_CELLS, "f32_kahan")
    ws = [torch.empty(wsb, dtype=torch.uint8, device=dev) for _ in range(ROTATE)]
    q.qdvm_tune_batched(plans, cps[0], co, fs[0], "f32_kahan", workspace=ws[0])
    tuning = [p.tuning() for p in plans]  # per plan: cell size x level
    # fixed Nbar = 8 on the same batch (level 2 for every cell)
    cp8 = (cb * len(nbars) + 2).to(torch.int32)

    def capture(fn):
        g = torch.cuda.CUDAGraph()
        fn()
        torch.cuda.synchronize(dev)
        with torch.cuda.graph(g):
            fn()
        return g

    def adaptive(k):
        return lambda: (q.equilibrium_distance(base, cb, co, fs[k], "f32_kahan", out=eps[k]),
                        q.select_levels(eps[k], cb, thr, level_plan, out=cps[k]),
                        q.qdvm_eval_batched(plans, cps[k], co, fs[k], "f32_kahan", out=Qs[k], moments=False,
                                            workspace=ws[k]))

    def fixed(k):
        return lambda: q.qdvm_eval_batched(plans, cp8, co, fs[k], "f32_kahan", out=Qs[k], moments=False,
                                           workspace=ws[k])

    def timed(graphs):
        for k in range(args.warmup):
            graphs[k % ROTATE].replay()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream(dev)
        e0.record(st)
        for k in range(args.steps):
            graphs[(args.warmup + k) % ROTATE].replay()
        e1.record(st)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / args.steps

    g_fix = [capture(fixed(k)) for k in range(ROTATE)]
    ms_fixed = timed(g_fix)
    Q8 = Qs[0].clone()
    g_ad = [capture(adaptive(k)) for k in range(ROTATE)]
    with ClockSampler(dev.index) as clk:
        ms = timed(g_ad)
    adaptive(0)()
    torch.cuda.synchronize(dev)
    lev = (cps[0].cpu().numpy() % len(nbars))
    fractions = [float((lev == i).mean()) for i in range(len(nbars))]
    Qa = Qs[0].cpu().numpy().astype(np.float64)
    Q8n = Q8.cpu().numpy().astype(np.float64)
    fin = fs[0].cpu().numpy().astype(np.float64)
    err, trunc = 0.0, 0.0
    for c in (0, 1, 2, 3, N_CELLS - 1):
        r = oracle.q(b.cell(c, fin), L, nbars[lev[c]])
        err = max(err, oracle.rel_linf(b.cell(c, Qa), r["Q"], r["scale"]))
        trunc = max(trunc, float(np.max(np.abs(b.cell(c, Qa) - b.cell(c, Q8n))) / np.max(r["scale"])))
    line = {"metric": METRIC, "value": b.total / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "space-dependent Nbar: 4096 2D cells N~U{16,32,48,64} at various distances from "
                                   "equilibrium (second-Maxwellian weight 0.5 U^3, seed 3), Nbar in {2,4,8} by the "
                                   "indicator sum|f-M[f]|/sum|f| with thresholds (0.02, 0.1); indicator, selection "
                                   "and evaluation in one CUDA graph per rotating batch copy (6 copies > L2)",
                       "tuning": tuning, "level_fractions_nbar_2_4_8": fractions},
            "fixed_nbar8_ms_per_step": ms_fixed, "speedup_vs_fixed_nbar8": ms_fixed / ms,
            "accuracy": {"rel_linf_vs_fp64_oracle_at_selected_nbar": err,
                         "truncation_vs_nbar8_rel_to_scale": trunc},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_dtr_workload(args):
    """The box-truncated operator D^tr (Section 2.3) term by term on a batch
    of 2D cells, with its conservation defects, beside the same direct sum
    with periodic indices and the fast evaluator of the periodised operator
    on the same batch."""
    import torch

    import paper_1201_3986_gb300 as q

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    Ns, nb, Lh = (16, 32, 48, 64), 8, 8.0
    b = synth.batch_2d(args.cells, Ns=Ns, L=Lh, seed=0)
    plans = [q.Plan(2, n, nb, Lh, kernel="hp") for n in Ns]
    cp = torch.tensor([Ns.index(int(n)) for n in b.Ns], dtype=torch.int32, device=dev)
    co = torch.tensor(b.offsets, dtype=torch.int64, device=dev)
    f = torch.tensor(b.f, dtype=torch.float32, device=dev)
    Q = torch.empty_like(f)
    M = torch.empty((b.n_cells, 4), dtype=torch.float64, device=dev)
    ws = torch.empty(q.batched_workspace_bytes(plans, b.n_cells, "f32_kahan"), dtype=torch.uint8, device=dev)

    def timeit(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream(dev)
        e0.record(st)
        for _ in range(args.steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / args.steps

    with ClockSampler(dev.index) as clk:
        ms_box = timeit(lambda: q.qdvm_eval_direct_batched(plans, cp, co, f, "f32_kahan", "box", out=Q, moments=M))
    mom_box = M.cpu().numpy()
    ms_per = timeit(lambda: q.qdvm_eval_direct_batched(plans, cp, co, f, "f32_kahan", "periodic", out=Q, moments=M))
    mom_per = M.cpu().numpy()
    ms_fast = timeit(lambda: q.qdvm_eval_batched(plans, cp, co, f, "f32_kahan", out=Q, moments=M, workspace=ws))
    # conservation: |moment| relative to the energy-weighted gain of the cell
    Qb, _ = q.qdvm_eval_direct_batched(plans, cp, co, f, "f32_kahan", "box")
    absq = torch.zeros(b.n_cells, dtype=torch.float64)
    Qa = Qb.abs().cpu().numpy().astype(np.float64)
    h2 = (2 * Lh / b.Ns.astype(np.float64)) ** 2
    for c in range(b.n_cells):
        absq[c] = h2[c] * b.cell(c, Qa).sum()
    ref = absq.numpy()
    defect = lambda m, k, w: float(np.max(np.abs(m[:, k]) / (w * ref)))
    line = {"metric": METRIC, "value": b.total / (ms_box / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_box, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"box-truncated D^tr, term by term: {b.n_cells} 2D cells N~U{{16,32,48,64}} "
                                   f"(seed 0), L=8, Nbar=8, h-scaled weights, FP32 + compensated sums, FP64 moments",
                       "n_cells": b.n_cells},
            "direct_periodic_ms": ms_per, "fast_periodic_ms": ms_fast,
            "conservation_defect_box": {"mass": defect(mom_box, 0, 1.0), "momentum": defect(mom_box, 1, Lh),
                                        "energy": defect(mom_box, 3, 2 * Lh * Lh)},
            "conservation_defect_periodic": {"momentum": defect(mom_per, 1, Lh),
                                             "energy": defect(mom_per, 3, 2 * Lh * Lh)},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_spectral_workload(args):
    """The pseudo-spectral route of Section 3.1 (eq. (sysDiff)): Q of a batch
    of 2D cells of one size through their Fourier modes with the dense table
    beta~, O(N^{2d}) per cell, beside the fast evaluator on the same cells.
    An L2 flush (a 256 MB write) separates the timed steps, each timed with
    its own events: the FP32 table (N^{2d} floats, 67 MB at N = 64) would
    otherwise stay in the 129 MB L2."""
    import torch

    import oracle
    import paper_1201_3986_gb300 as q

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    N, nb, Lh = args.n, args.nbar or 8, 8.0
    prec = args.prec
    n_cells = args.cells
    rng = np.random.default_rng(0)
    cells = np.stack([synth.mixture(2, N, Lh, rng) for _ in range(n_cells)])
    dtype = torch.float64 if prec == "f64" else torch.float32
    f = torch.tensor(cells, dtype=dtype, device=dev)
    plan = q.Plan(2, N, nb, Lh, kernel="unit")
    table = q.spectral_table(plan, prec)
    Q = torch.empty_like(f)
    ws = torch.empty(q.spectral_workspace_bytes(plan, n_cells, prec), dtype=torch.uint8, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        total = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize(dev)
            total += e0.elapsed_time(e1)
        return total / args.steps

    with ClockSampler(dev.index) as clk:
        ms = timed(lambda: q.qdvm_eval_spectral(plan, table, f, prec, out=Q, workspace=ws))
    Qn = Q.cpu().numpy().astype(np.float64)
    fin = f.cpu().numpy().astype(np.float64)
    errs = []
    for c in (0, n_cells - 1):
        r = oracle.q(fin[c], Lh, nb)
        errs.append(oracle.rel_linf(Qn[c], r["Q"], r["scale"]))
    # the fast evaluator on the same cells (FFT loss, tuned launch)
    cp = torch.zeros(n_cells, dtype=torch.int32, device=dev)
    co = torch.arange(n_cells, dtype=torch.int64, device=dev) * (N * N)
    plan.set_tuning(loss_fft=1)
    wsf = torch.empty(q.batched_workspace_bytes([plan], n_cells, prec), dtype=torch.uint8, device=dev)
    ff = f.reshape(-1)
    Qf = torch.empty_like(ff)
    ms_fast = timed(lambda: q.qdvm_eval_batched([plan], cp, co, ff, prec, out=Qf, moments=False, workspace=wsf))
    M = N * N
    flops = 10.0 * M * M * n_cells  # per (I, K, cell): complex product, scale, accumulate
    peak = 152 * 128 * 2 * 2.07e9 / 1e12
    line = {"metric": METRIC, "value": n_cells * M / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == "f64" else "f32", "data": "synthetic",
            "config": {"workload": f"pseudo-spectral route (eq. (sysDiff)): {n_cells} 2D cells N={N} on [-8,8]^2, "
                                   f"Nbar={nb} ({plan.n_lines} lines), unit kernel, two-Maxwellian mixtures "
                                   f"(seed 0), dense table of {M * M} entries, {prec}",
                       "N": N, "Nbar": nb, "n_cells": n_cells, "prec": prec,
                       "l2": "256 MB flush between timed steps"},
            "roofline": {"bound": "alu", "kernel": "k_spec_conv",
                         "achieved": flops / (ms / 1e3) / 1e12 if prec != "f64" else None,
                         "peak": peak if prec != "f64" else None, "unit": "TFLOP/s",
                         "frac": flops / (ms / 1e3) / 1e12 / peak if prec != "f64" else None,
                         "note": "10 flops per (I, K, cell); FP32 peak 152 x 128 x 2 x 2.07 GHz; the whole "
                                 "evaluation (DFTs included) timed"},
            "fast_evaluator_ms": ms_fast, "fast_over_spectral_speedup": ms / ms_fast,
            "accuracy": {"rel_linf_vs_fp64_oracle_max": max(errs)}, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


# Table 2 of the paper: CPU time (s) of the fast DVM to T = 1 with dt = 0.01
# (100 TVD-RK2 steps) on one 2D BKW cell, hardware unstated; keys (N, Nbar).
TABLE2_S = {(16, 3): 0.5, (32, 3): 3.19, (32, 7): 14.52, (64, 3): 16.2, (64, 7): 73.4, (64, 14): 283.0,
            (128, 3): 85.8, (128, 7): 378.0, (128, 14): 1382.0, (128, 28): 5531.0}
# velocity domain half-width per N used for those runs (Section 4)
TABLE2_L = {16: 5.5, 32: 7.0, 64: 8.0, 128: 8.0}


def run_bkw_workload(args):
    """The paper's timing run (Table 2): one 2D BKW cell, 100 TVD-RK2 steps of
    dt = 0.01 to T = 1, captured in one CUDA graph.  The weights are the
    h-scaled ones (c_e = h^3 |e|): with them a step changes f by about 1% on
    every grid, whereas the unscaled unit weights make dt = 0.01 unstable
    from N = 128 on.  The cost does not depend on the weights.  The value
    counts Q evaluations per second (200 per run)."""
    import torch

    import oracle
    import paper_1201_3986_gb300 as q

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    N, nb = args.n, args.nbar or 14
    prec = args.prec
    Lh = TABLE2_L.get(N, 8.0)
    dt, n_steps = 0.01, 100
    f_np = synth.bkw_2d(N, Lh)
    plan = q.Plan(2, N, nb, Lh, kernel="hp")
    plan.set_tuning(loss_fft=0 if args.loss_fft is None else args.loss_fft)
    dtype = torch.float64 if prec == "f64" else torch.float32
    f0 = torch.tensor(f_np, dtype=dtype, device=dev)
    f = f0.clone()
    wsb = q.rk2_workspace_single_bytes(plan, prec)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    q.qdvm_rk2(plan, f, dt, 1, prec, workspace=ws)  # first call outside capture
    torch.cuda.synchronize(dev)
    f.copy_(f0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        q.qdvm_rk2(plan, f, dt, n_steps, prec, workspace=ws)
    m0 = q.qdvm_moments(plan, f0, prec).cpu().numpy()
    f.copy_(f0)
    g.replay()  # one run to T = 1 from the datum
    torch.cuda.synchronize(dev)
    m1 = q.qdvm_moments(plan, f, prec).cpu().numpy()
    for _ in range(args.warmup):
        g.replay()
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    acc = {"mass_defect_rel_T1": float(abs(m1[0] - m0[0]) / abs(m0[0]))}
    if N <= 64:
        f.copy_(f0)
        q.qdvm_rk2(plan, f, dt, 1, prec, workspace=ws)
        ref = oracle.rk2(f_np, Lh, nb, dt, 1, kernel="hp")
        sc = np.max(np.abs(f_np)) + dt * np.max(oracle.q(f_np, Lh, nb, kernel="hp")["scale"])
        acc["one_step_rel_err_vs_fp64_oracle_rk2"] = float(np.max(np.abs(f.cpu().numpy() - ref)) / sc)
    evals = 2 * n_steps * N * N
    paper = TABLE2_S.get((N, nb))
    value = evals / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": (value / (evals / paper)) if paper else None, "dtype": "f64" if prec == "f64" else "f32",
            "data": "synthetic",
            "config": {"workload": f"paper Table 2 run: 2D BKW datum (S = 0.6), N={N} on [-{Lh},{Lh}]^2, Nbar={nb} "
                                   f"({plan.n_lines} lines), h-scaled weights c_e = h^3|e|, TVD-RK2 dt=0.01 to "
                                   f"T=1 (100 steps, 200 Q evaluations) per step of this line, one CUDA graph",
                       "N": N, "Nbar": nb, "prec": prec, "tuning": plan.tuning(),
                       "paper_table2_s": paper,
                       "vs_baseline_note": "Q evaluations per second against Table 2's time to T = 1 "
                                           "(CPU, hardware unstated): context, not a target"},
            "time_to_T1_ms": ms, "accuracy": acc, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_gpu_workload(args):
    """Other measured workloads (single GPU): 3D hard spheres on 32^3 cells.
      batch3d   Q on 256 cells, Nbar = 5 (577 lines), FP32
      jvp3d     JVP on the same batch with Gaussian tangents (seed 2)
      vjp3d     VJP with Gaussian cotangents (seed 2)
      single3d  one 32^3 cell, tri-axial Gaussian, Nbar = args.nbar (3, 5, 7)
    Same timing rules as the default workload (rotating inputs > L2 where the
    batch is smaller than L2, CUDA events, warm-up)."""
    import torch

    import oracle
    import paper_1201_3986_gb300 as q

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wl = args.workload
    if wl == "single3d":
        nb = args.nbar or 5
        f_np = synth.trimaxwellian_3d(32, 6.0)
        plan = q.Plan(3, 32, nb, 6.0, kernel="hp")
        plan.set_tuning(loss_fft=1 if args.loss_fft is None else args.loss_fft)
        rot = 8  # 8 x 128 KB inputs + outputs; the scratch dominates anyway
        fs = [torch.tensor(f_np, dtype=torch.float32, device=dev) for _ in range(rot)]
        outs = [torch.empty_like(fs[0]) for _ in range(rot)]
        ws = torch.empty(max(plan.eval_workspace("f32"), 1), dtype=torch.uint8, device=dev)

        def step(k):
            q.qdvm_eval(plan, fs[k % rot], "f32", out=outs[k % rot], workspace=ws)

        pts_per_step = 32 ** 3
        cfg = {"workload": f"3D hard spheres, one 32^3 cell on [-6,6]^3, Nbar={nb} ({plan.n_lines} lines), "
                           "tri-axial Gaussian T=(0.5,1,2), drift (0.5,0,0), FP32", "Nbar": nb,
               "tuning": plan.tuning()}
        check = lambda: (f_np, outs[0], None)
    else:
        nb = 5
        b = synth.batch_3d(args.cells, N=32, L=6.0, seed=1)
        a_np = synth.gaussian(b.f.shape, seed=2)
        plan = q.Plan(3, 32, nb, 6.0, kernel="hp")
        cp = torch.zeros(b.n_cells, dtype=torch.int32, device=dev)
        co = torch.tensor(b.offsets, dtype=torch.int64, device=dev)
        rot = 2  # 2 x (33.5 MB in + 33.5 MB aux + 33.5 MB out) > L2
        fs = [torch.tensor(b.f, dtype=torch.float32, device=dev) for _ in range(rot)]
        ats = [torch.tensor(a_np, dtype=torch.float32, device=dev) for _ in range(rot)]
        outs = [torch.empty_like(fs[0]) for _ in range(rot)]
        # room for both forward evaluators (line engine, FFT loss), the
        # derivatives and every line-chunk count the autotuner tries (up to 16)
        wsb = []
        for fft in (0, 1):
            for ch in (0, 16):
                plan.set_tuning(loss_fft=fft, line_chunks=ch)
                wsb.append(q.batched_workspace_bytes([plan], b.n_cells, "f32"))
        plan.set_tuning(line_chunks=0)
        ws = torch.empty(2 * max(wsb), dtype=torch.uint8, device=dev)
        plan.set_tuning(loss_fft=1 if args.loss_fft is None else args.loss_fft)
        if wl == "batch3d":
            if args.tuning:
                th, dj, fft, ch = (int(v) for v in args.tuning.split(","))
                plan.set_tuning(threads=th, direct_j=dj, loss_fft=fft, line_chunks=ch)
            else:
                plan.set_tuning(loss_fft=0)
                q.qdvm_tune_batched([plan], cp, co, fs[0], "f32", workspace=ws)

            def step(k):
                q.qdvm_eval_batched([plan], cp, co, fs[k % rot], "f32", out=outs[k % rot], moments=False,
                                    workspace=ws)
        elif wl == "jvp3d":
            def step(k):
                q.qdvm_jvp_batched([plan], cp, co, fs[k % rot], ats[k % rot], "f32", out=outs[k % rot], workspace=ws)
        else:
            def step(k):
                q.qdvm_vjp_batched([plan], cp, co, fs[k % rot], ats[k % rot], "f32", out=outs[k % rot], workspace=ws)
        pts_per_step = b.total
        cfg = {"workload": f"{wl}: {b.n_cells} cells of 32^3 on [-6,6]^3, Nbar=5 (577 lines), hard spheres, two-Maxwellian "
                           "mixtures (seed 1), Gaussian tangents/cotangents (seed 2), FP32", "Nbar": nb,
               "tuning": plan.tuning()}
        check = lambda: (b.cell(0, b.f.astype(np.float32).astype(np.float64)), outs[0][:32 ** 3].view(32, 32, 32),
                         b.cell(0, a_np.astype(np.float32).astype(np.float64)))
    stream = torch.cuda.current_stream(dev)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        e0.record(stream)
        for k in range(args.steps):
            step(k)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    # accuracy on sampled points of cell 0 (output of step 0 buffer)
    step(0)
    torch.cuda.synchronize(dev)
    fc, oc, ac = check()
    rng = np.random.default_rng(0)
    idx = np.unique(rng.choice(32 ** 3, size=64, replace=False)).astype(np.int64)
    oc = oc.cpu().numpy().astype(np.float64).ravel()
    if wl in ("single3d", "batch3d"):
        r = oracle.q_points(fc, 6.0, nb, idx, kernel="hp")
        err = float(np.max(np.abs(oc[idx] - r["Q"])) / np.max(r["scale"]))
    elif wl == "jvp3d":
        r, sc = oracle.jvp_points(fc, ac, 6.0, nb, idx, kernel="hp")
        err = float(np.max(np.abs(oc[idx] - r)) / np.max(sc))
    else:
        r, sc = oracle.vjp_points(fc, ac, 6.0, nb, idx, kernel="hp")
        err = float(np.max(np.abs(oc[idx] - r)) / np.max(sc))
    line = {"metric": METRIC, "value": pts_per_step / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "accuracy": {"rel_linf_vs_fp64_oracle_sampled": err, "points": int(idx.size)},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="qdvm", choices=["qdvm", "reference"])
    ap.add_argument("--ref-cells", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--loss-fft", type=int, default=None, choices=[0, 1, 2],
                    help="single3d, jvp3d, vjp3d (default 1): loss as an FFT convolution with row-form gain, or the "
                         "line engine (0); bkw (default 0): FFT loss in the single-cell 2D evaluator (2: the axis "
                         "window from the same transform)")
    ap.add_argument("--workload", default="batch2d",
                    choices=["batch2d", "batch3d", "jvp3d", "vjp3d", "single3d", "rk2", "bkw", "adaptive", "dtr",
                             "spectral"])
    ap.add_argument("--n", type=int, default=64, help="bkw, spectral: points per axis")
    ap.add_argument("--prec", default="f64", choices=["f64", "f32", "f32_kahan"], help="bkw, spectral: precision")
    ap.add_argument("--rk2-steps", type=int, default=10, help="rk2: time steps per graph launch")
    ap.add_argument("--nbar", type=int, default=None)
    ap.add_argument("--ns", default=None, help="batch2d: comma-separated cell sizes (default 16,32,48,64)")
    ap.add_argument("--cells", type=int, default=256, help="batch3d / jvp3d / vjp3d: number of 32^3 cells; dtr: 2D cells")
    ap.add_argument("--tuning", default=None,
                    help="pin the launch configuration instead of autotuning: batch2d threads,direct_j,loss_fft[,scan_j] "
                         "for every plan, or per cell size 'N=threads,direct_j,loss_fft,scan_j ...'; "
                         "batch3d threads,direct_j,loss_fft,line_chunks")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        args.ref_cells = args.ref_cells or REF_STEP_CELLS
        run_reference(args)
    elif args.workload == "rk2":
        run_rk2_workload(args)
    elif args.workload == "bkw":
        run_bkw_workload(args)
    elif args.workload == "adaptive":
        run_adaptive_workload(args)
    elif args.workload == "dtr":
        run_dtr_workload(args)
    elif args.workload == "spectral":
        run_spectral_workload(args)
    elif args.workload != "batch2d":
        run_gpu_workload(args)
    else:
        # other cell sizes or Nbar for the batched 2D workload (the default,
        # N in {16,32,48,64} with Nbar = 8, is the measured configuration)
        global NS, NBAR
        if args.nbar:
            NBAR = args.nbar
        if args.ns:
            NS = tuple(int(v) for v in args.ns.split(","))
        args.ref_cells = args.ref_cells or ORACLE_SAMPLE_CELLS
        run_gpu(args)


if __name__ == "__main__":
    main()
