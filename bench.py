#!/usr/bin/env python
"""HG GRAPE cost+gradient evaluations per second on GB300, with peak HBM against torch full-AD.

One step = one full cost+gradient evaluation (forward sweep, cost, backward sweep,
gradient) of the workload, inputs resident in HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank evaluates its own
independent instance of the workload (replicas, weak scaling); rank 0 prints the
aggregate.  ``--impl reference`` times the CPU oracle (the reference arm) on a
bounded sample of the same workload on this host's cores.
"""

from __future__ import annotations

import argparse
import json
import tempfile
import warnings

import numpy as np
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cost+gradient evals/s & peak HBM: HG kernels vs torch full-AD, 1 GB300"
DEFAULT_WORKLOAD = "c3_gate_d4000"
FP64_NOMINAL_GFLOPS = 152 * 2 * 2 * 2.07   # 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz (used if the probe fails)
HBM_FALLBACK_GBS = 6800.0                  # recipe fallback when MEASURED_PEAKS.json is absent
L2_FLUSH_BYTES = 256 << 20       # > 129 MB L2


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fullad", action="store_true")
    ap.add_argument("--fullad-steps", default="2,4")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--n-steps", type=int, default=None, help="override the workload's N (profiling a small case)")
    ap.add_argument("--batch", action="store_true", help="also measure the 64-instance batch (one graph launch)")
    ap.add_argument("--autotune", action="store_true", help="autotune every batch member (slower set-up)")
    ap.add_argument("--m-sweep", action="store_true", help="also sweep the checkpoint spacing M over {50, 200, 1000}")
    ap.add_argument("--c4", action="store_true", help="also run the d = 16000 workload in FP32 bulk and FP64")
    ap.add_argument("--dense", action="store_true", help="also run the dense d = 2048 variant on the tensor cores")
    ap.add_argument("--dense-steps", type=int, default=20)
    ap.add_argument("--extras-only", action="store_true",
                    help="skip the main measurement and print only the requested comparisons (for profiling them)")
    ap.add_argument("--eig", action="store_true",
                    help="also compare the eigendecomposition propagator (App. F) with the Taylor kernels")
    ap.add_argument("--families", action="store_true",
                    help="also time the three-transmon, qubit-chain and fluxonium-pair Hamiltonians (FP64, FP32 bulk)")
    ap.add_argument("--optimize", action="store_true",
                    help="also time steepest descent in a CUDA graph against a host-driven loop (c2_gate_d80)")
    ap.add_argument("--backward-mode", type=int, default=0, help="0 auto, 1 one team per column, 3 three-stage")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ distributed helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(local_seconds: float, local_units: int, world: int, reduce_max=None, reduce_sum=None):
    """Whole-job throughput: units of all ranks / the slowest rank's time (max over ranks)."""
    t = reduce_max(local_seconds) if reduce_max else local_seconds
    u = reduce_sum(local_units) if reduce_sum else local_units * world
    return u / t, t


def workload_description(p) -> str:
    return (f"{p.name}: d={p.dim}, K={p.n_controls} controls, n={p.n_states} states, N={p.n_steps} steps, "
            f"dt={p.dt} ns, tau={p.tau:g}, weights (fid, forbid, amp)=({p.w_fid}, {p.w_forbid}, {p.w_amp}), "
            f"seeded smooth controls (RMS 2pi*0.01 rad/ns), complex128")


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"grape_bench_clocks_rank{index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ algorithmic work model

def entry_classes(p):
    """Entries of the union pattern by the real work one product y += B_ij x_j takes per column:
    the diagonal when every H_ii is real (B_ii imaginary: 2 multiplies), off-diagonal entries whose
    every H_ij term is real or every one imaginary (B_ij imaginary or real: 2 multiply-adds, 4 flops),
    the rest (a complex multiply-add, 8 flops).  Returns (n_diag, n_single, n_general, n_ctrl)."""
    import scipy.sparse as sp
    ops = [sp.csr_matrix(p.H0)] + [sp.csr_matrix(h) for h in p.Hk]
    union = abs(ops[0]).astype(bool)
    for h in ops[1:]:
        union = union + abs(h).astype(bool)
    union = union.tocoo()
    rows, cols = union.row, union.col
    re_any = np.zeros(rows.size, bool)
    im_any = np.zeros(rows.size, bool)
    ctrl = np.zeros(rows.size, bool)
    for k, h in enumerate(ops):
        v = np.asarray(h.tocsr()[rows, cols]).ravel()
        re_any |= v.real != 0
        im_any |= v.imag != 0
        if k > 0:
            ctrl |= v != 0
    diag = rows == cols
    diag_real = bool(np.all(~im_any[diag]))
    n_diag = int(diag.sum()) if diag_real else 0
    single = (~diag) & (re_any ^ im_any)
    n_single = int(single.sum())
    return n_diag, n_single, int(rows.size) - n_diag - n_single, int(ctrl.sum())


def product_flops(cls, dim: int) -> float:
    """FP64 flops of one Taylor term's product and its row update, per column."""
    n_diag, n_single, n_general, _ = cls
    return 2.0 * n_diag + 4.0 * n_single + 8.0 * n_general + 4.0 * dim


def forward_flops(schedule_m, schedule_s, cls, dim: int, n: int) -> float:
    """k_forward: m_n s_n terms per step (Eqs. (eBm equation), (eBmpsi))."""
    return float(np.sum(np.asarray(schedule_m, float) * np.asarray(schedule_s, float))) * product_flops(cls, dim) * n


def costate_flops(schedule_m, schedule_s, cls, dim: int, n: int) -> float:
    """k_costate (all launches of one evaluation): one product and one Horner update per term."""
    return forward_flops(schedule_m, schedule_s, cls, dim, n)


def gradient_flops(schedule_m, schedule_s, cls, dim: int, n: int) -> float:
    """k_gradient (all launches of one evaluation): per step m s accumulations conj(w_p[i]) x_p[j] on the
    control entries (8 flops each) and m s - 1 products with their increment updates."""
    mu = np.asarray(schedule_m, float) * np.asarray(schedule_s, float)
    return float(np.sum(mu * 8.0 * cls[3] + (mu - 1.0) * product_flops(cls, dim))) * n


def fused_backward_flops(schedule_m, schedule_s, cls, dim: int, n: int) -> float:
    """The one-team backward: per substep 2m products (psi chain, Horner chain), m - 1
    products of the x chain and m accumulations on the control entries."""
    tot = 0.0
    for m, s in zip(schedule_m, schedule_s):
        m, s = int(m), int(s)
        tot += s * ((3 * m - 1) * product_flops(cls, dim) + m * 8.0 * cls[3])
    return tot * n


def measured_peaks():
    """HBM GB/s and its source: MEASURED_PEAKS.json when the driver wrote one, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for key in ("hbm_gbs", "hbm_GBps", "hbm"):
            if key in d:
                return float(d[key]), "MEASURED_PEAKS.json"
    except Exception:
        pass
    return HBM_FALLBACK_GBS, "fallback (no MEASURED_PEAKS.json)"


def read_traffic(kernel: str, workload: str):
    """DRAM bytes per launch recorded from an ncu capture in profiles/ (None if not recorded)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("traffic_bytes_per_launch:"):
            try:
                return float(line.split(":", 1)[1].strip().split()[0])
            except ValueError:
                return None
    return None


# ------------------------------------------------------------------ torch full-AD comparator (GPU)

def fullad_taylor_gpu(p, u, sched_m, sched_s, n_steps: int, device: int):
    """Full automatic differentiation of the same truncated-Taylor propagation in torch (Sec. IV.A, full-AD).

    B_n x = -i dt/s (H0 x + sum_k u_kn H_k x) with cuSPARSE CSR products; autograd records every
    Taylor term, so memory grows with N * mu (Table I).  Returns (seconds, peak bytes) for n_steps.
    """
    import numpy as np
    import torch

    dev = torch.device("cuda", device)

    def csr(m):
        m = m.tocsr()
        return torch.sparse_csr_tensor(torch.tensor(m.indptr, dtype=torch.int64), torch.tensor(m.indices, dtype=torch.int64),
                                       torch.tensor(m.data, dtype=torch.complex128), size=m.shape).to(dev)

    H0 = csr(p.H0)
    Hk = [csr(h) for h in p.Hk]
    psi0 = torch.tensor(np.asarray(p.psi0), dtype=torch.complex128, device=dev)
    target = torch.tensor(np.asarray(p.target), dtype=torch.complex128, device=dev)
    om = torch.tensor(np.asarray(p.omega), dtype=torch.float64, device=dev)[:, None] if p.omega is not None else None
    torch.cuda.synchronize(dev)
    torch.cuda.reset_peak_memory_stats(dev)
    base = torch.cuda.memory_allocated(dev)
    t0 = time.perf_counter()
    u_t = torch.tensor(np.asarray(u)[:, :n_steps], dtype=torch.float64, device=dev, requires_grad=True)
    psi = psi0
    c2 = torch.zeros((), dtype=torch.float64, device=dev)
    n = psi0.shape[1]
    for step in range(n_steps):
        m, s = int(sched_m[step]), int(sched_s[step])
        uc = u_t[:, step].to(torch.complex128)
        for _ in range(s):
            t = psi
            acc = psi
            for q in range(1, m + 1):
                y = torch.sparse.mm(H0, t)
                for k, h in enumerate(Hk):
                    y = y + uc[k] * torch.sparse.mm(h, t)
                t = y * (-1j * p.dt / (s * q))
                acc = acc + t
            psi = acc
        if om is not None:
            c2 = c2 + torch.sum(om * (psi.real ** 2 + psi.imag ** 2))
    g = torch.sum(torch.conj(target) * psi)
    cost = p.w_fid * (1.0 - (g.real ** 2 + g.imag ** 2) / n ** 2) + p.w_forbid * c2 / (n_steps * n) \
        + p.w_amp * torch.sum(u_t ** 2) / n_steps
    cost.backward()
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    peak = torch.cuda.max_memory_allocated(dev) - base
    del u_t, psi, c2, g, cost
    torch.cuda.empty_cache()
    return dt, peak


# ------------------------------------------------------------------ CPU oracle timing

def oracle_sample(workload: str, seed_offset: int = 0):
    """Time the CPU oracle on one step of the workload (a bounded sample); returns (seconds, steps)."""
    from oracle import cost_and_grad
    from workloads import build_config

    q = build_config(workload, n_steps=1)
    t0 = time.perf_counter()
    cost_and_grad(q, q.u0)
    return time.perf_counter() - t0, 1


def oracle_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        return max((i.get("num_threads", 1) for i in threadpool_info()), default=os.cpu_count() or 1)
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2304_06200_gb300 import GrapeProblem
    from paper_2304_06200_gb300._abi import lib
    from workloads import build_config

    lib()
    if args.extras_only:
        extra = {}
        if args.eig:
            extra["eig_vs_taylor"] = eig_compare(local)
        if args.dense:
            extra["dense_d2048_tc"] = dense_compare(local, args.dense_steps)
        if args.batch:
            extra["c5_batch"] = batch_compare(local, args.autotune)
        if args.c4:
            extra["c4"] = c4_compare(local)
        if args.m_sweep:
            extra["checkpoint_sweep"] = checkpoint_sweep(args.workload, local, args.n_steps)
        if args.families:
            extra["families"] = families_compare(local)
        if args.optimize:
            extra["steepest_descent"] = optimize_compare(local)
        print(json.dumps({"extras": extra}), flush=True)
        return
    p = build_config(args.workload, seed=None if rank == 0 else 1000 + rank, n_steps=args.n_steps)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats(dev)
    mem0 = torch.cuda.memory_allocated(dev)
    hg = GrapeProblem(p, device=local, backward_mode=args.backward_mode)
    u = torch.tensor(p.u0, dtype=torch.float64, device=dev)
    cost = torch.zeros((), dtype=torch.float64, device=dev)
    grad = torch.zeros((p.n_controls, p.n_steps), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 0)):
        hg.cost_device(u, cost, stream)
        hg.grad_device(grad, stream)
    hg.sync_status(stream)
    torch.cuda.synchronize()
    hg_peak = torch.cuda.max_memory_allocated(dev) - mem0
    info = hg.info()
    sched_m, sched_s, norms = hg.schedule()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    import ctypes
    fp64_peak = ctypes.c_double(0.0)
    peak_ok = lib().grape_fp64_fma_rate(local, ctypes.byref(fp64_peak)) == 0 and fp64_peak.value > 0
    fp64_peak = fp64_peak.value if peak_ok else FP64_NOMINAL_GFLOPS
    hg.set_kernel_tracing(True)
    hg.kernel_times()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        hg.cost_device(u, cost, stream)
        ev[i][1].record(stream)
        hg.grad_device(grad, stream)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    hg.sync_status(stream)
    ktimes = hg.kernel_times()
    hg.set_kernel_tracing(False)
    step_ms = [ev[i][0].elapsed_time(ev[i][2]) for i in range(args.steps)]
    fwd_ms = [ev[i][0].elapsed_time(ev[i][1]) for i in range(args.steps)]
    bwd_ms = [ev[i][1].elapsed_time(ev[i][2]) for i in range(args.steps)]
    local_s = sum(step_ms) / 1e3

    def rmax(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    def rsum(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
        return float(t.item())

    value, tmax = aggregate(local_s, args.steps, world, rmax, rsum)

    # ---- end to end through the host-pointer API (pinned host buffers, H2D + D2H inside the timed region)
    u_h = torch.tensor(p.u0, dtype=torch.float64).pin_memory()
    cost_h = torch.zeros(1, dtype=torch.float64).pin_memory()
    grad_h = torch.zeros((p.n_controls, p.n_steps), dtype=torch.float64).pin_memory()
    e2e_times, e2e_dev = [], []
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        flush.zero_()
        torch.cuda.synchronize()
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e_a.record(stream)
        st = hg._lib.grape_cost_and_grad(hg._h, ctypes.c_void_p(u_h.data_ptr()), ctypes.c_void_p(cost_h.data_ptr()),
                                         ctypes.c_void_p(grad_h.data_ptr()), 0, None)
        e_b.record(stream)
        t1 = time.perf_counter()
        if st != 0:
            raise RuntimeError(f"grape_cost_and_grad failed with status {st}")
        torch.cuda.synchronize()
        if i > 0:
            e2e_times.append(t1 - t0)
            e2e_dev.append(e_a.elapsed_time(e_b) / 1e3)
    e2e_local = sum(e2e_times)
    e2e_value = aggregate(e2e_local, len(e2e_times), world, rmax, rsum)[0] if e2e_times else None
    h2d = p.n_controls * p.n_steps * 8
    d2h = 8 + p.n_controls * p.n_steps * 8

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- roofline: every sweep kernel's algorithmic FP64 flops per launch over its live CUDA-event
    # duration (traced during the timed steps); the dominant kernel (largest summed time) is reported
    cls = entry_classes(p)
    mode = info["backward_mode"]
    total_flops = {"k_forward": forward_flops(sched_m, sched_s, cls, p.dim, p.n_states)}
    if mode == 3:
        total_flops["k_costate"] = costate_flops(sched_m, sched_s, cls, p.dim, p.n_states)
        total_flops["k_gradient"] = gradient_flops(sched_m, sched_s, cls, p.dim, p.n_states)
    else:
        total_flops["k_backward"] = fused_backward_flops(sched_m, sched_s, cls, p.dim, p.n_states)
    kern = {}
    for name, fl in total_flops.items():
        t = ktimes[name]
        if t["launches"] == 0:
            continue
        per_launch_ms = t["ms"] / t["launches"]
        launches_per_eval = t["launches"] / args.steps
        flops_per_launch = fl / launches_per_eval
        ach = flops_per_launch / (per_launch_ms * 1e-3) / 1e9
        kern[name] = {"launches_per_eval": launches_per_eval, "avg_launch_ms": round(per_launch_ms, 4),
                      "ms_per_eval": round(t["ms"] / args.steps, 2), "flops_per_launch": flops_per_launch,
                      "achieved": round(ach, 2), "frac": round(ach / fp64_peak, 4)}
    dom = max(kern, key=lambda k: kern[k]["ms_per_eval"])
    nnz = info["union_nnz"]
    mu_tot = float(np.sum(sched_m * sched_s))
    # Sec. 8(d)-style algorithmic bytes: per Taylor term the union pattern's values and indices once,
    # the input and output blocks once; three passes of terms (forward, costate chain, gradient) plus
    # the stored states and Horner vectors written and read once
    term_bytes = nnz * (16 + 4) + (p.dim + 1) * 4 + 2 * p.dim * p.n_states * 16
    passes = 3 if mode == 3 else 4
    eval_bytes = passes * mu_tot * term_bytes
    if mode == 3:
        eval_bytes += 2 * p.n_steps * p.dim * p.n_states * 16 + 2 * mu_tot * p.dim * p.n_states * 16
    hbm_peak, hbm_src = measured_peaks()
    hbm_ach = eval_bytes * value / 1e9
    roofline = {"bound": "alu", "kernel": dom, "achieved": kern[dom]["achieved"], "peak": round(fp64_peak, 1),
                "unit": "GFLOP/s", "frac": kern[dom]["frac"], "traffic": read_traffic(dom, args.workload),
                "peak_source": ("measured: grape_fp64_fma_rate (independent FP64 FMA chains on every SM, CUDA events) "
                                "on this GPU in this run" if peak_ok else "nominal 152 SMs x 2 FMA/clk x 2 x 2.07 GHz"),
                "flops_per_launch": kern[dom]["flops_per_launch"], "launch_ms": kern[dom]["avg_launch_ms"],
                "flop_model": "per Taylor term and column: 8 flops per general entry, 4 per single-phase entry, "
                              "2 per real-H diagonal entry, 4 per row update; k_gradient adds 8 per control entry",
                "entry_classes": {"diag": cls[0], "single_phase": cls[1], "general": cls[2], "control": cls[3]},
                "kernels": kern,
                "hbm": {"algorithmic_bytes_per_eval": eval_bytes, "achieved_GBps": round(hbm_ach, 1),
                        "peak_GBps": hbm_peak, "peak_source": hbm_src, "frac": round(hbm_ach / hbm_peak, 4)}}

    # ---- torch full-AD comparator (same GPU, same Taylor schedule) for peak HBM
    peak_hbm = {"hg_bytes": int(hg_peak), "hg_problem_bytes": int(info["device_bytes"])}
    if not args.no_fullad:
        try:
            pts = []
            for ns in [int(x) for x in args.fullad_steps.split(",") if x]:
                t_ad, b_ad = fullad_taylor_gpu(p, p.u0, sched_m, sched_s, ns, local)
                pts.append((ns, t_ad, b_ad))
            (n1, t1_, b1), (n2, t2_, b2) = pts[0], pts[-1]
            slope = (b2 - b1) / max(n2 - n1, 1)
            extrap = b2 + slope * (p.n_steps - n2)
            peak_hbm.update({
                "fullad_samples": [{"steps": a, "seconds": round(b, 3), "peak_bytes": int(c)} for a, b, c in pts],
                "fullad_bytes_extrapolated_full_N": int(extrap),
                "fullad_fits_in_hbm": bool(extrap < torch.cuda.get_device_properties(dev).total_memory),
                "fullad_evals_per_s_extrapolated": round(1.0 / (t2_ / n2 * p.n_steps), 6),
                "ratio_fullad_over_hg": round(extrap / max(hg_peak, 1), 1),
                "method": "torch autograd through the same truncated-Taylor steps (cuSPARSE CSR products), peak "
                          "torch.cuda.max_memory_allocated at two reduced N, extrapolated linearly in N"})
        except Exception as exc:  # the comparator is a reported baseline; report why it is missing
            peak_hbm["fullad_unavailable"] = f"{type(exc).__name__}: {exc}"[:300]

    # ---- CPU oracle baseline (bounded sample)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        secs, steps = oracle_sample(args.workload)
        per_eval = secs / steps * p.n_steps
        cpu = {"value": 1.0 / per_eval, "unit": "evals/s", "cores": oracle_threads(), "kind": "oracle",
               "sample": f"oracle (numpy eigh, stored states, divided differences) on {steps} of the "
                         f"{p.n_steps} steps ({secs:.1f} s), scaled to one full evaluation"}

    secondary = None
    if not args.no_secondary:
        secondary = {"c2_fp64": secondary_run("c2_gate_d80", "fp64", local),
                     "c2_fp32_bulk": secondary_run("c2_gate_d80", "fp32_bulk", local),
                     "c3_fp32_bulk": secondary_run(args.workload, "fp32_bulk", local, ref=(float(cost.item()), grad.cpu().numpy()),
                                                   n_steps=args.n_steps)}

    extra = {}
    if args.m_sweep:
        extra["checkpoint_sweep"] = checkpoint_sweep(args.workload, local, args.n_steps)
    if args.c4:
        extra["c4"] = c4_compare(local)
    if args.batch:
        extra["c5_batch"] = batch_compare(local, args.autotune)
    if args.dense:
        extra["dense_d2048_tc"] = dense_compare(local, args.dense_steps)
    if args.eig:
        extra["eig_vs_taylor"] = eig_compare(local)
    if args.families:
        extra["families"] = families_compare(local)
    if args.optimize:
        extra["steepest_descent"] = optimize_compare(local)

    # our kernels per evaluation: k_schedule, k_forward, k_finalize, the backward kernels, k_grad_reduce
    if mode == 3:
        nb = -(-p.n_steps // max(info["block_steps"], 1))
        per_eval = 3 + 1 + 2 * nb + 1 + 1          # + k_plan, per block k_costate and k_gradient, gated fallback
    else:
        per_eval = 5
    gpu_launches = per_eval * args.steps
    out = {
        "metric": METRIC, "value": round(value, 6), "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(tmax / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_description(p), "parallelism": f"replicas x{world}",
                   "l2": "flushed before every timed step (256 MB write)", "cluster_ctas_per_column_fwd": info["cluster_forward"],
                   "cluster_ctas_per_column_bwd": info["cluster"], "backward_mode": info["backward_mode"],
                   "gradient_team_ctas": info["grad_cluster"], "steps_per_block": info["block_steps"],
                   "ckpt_every": info["ckpt_every"], "total_taylor_terms_per_sweep": int(np.sum(sched_m * sched_s)),
                   "max_norm_A1": round(float(np.max(norms)), 4)},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 6) if e2e_value else None, "unit": "evals/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "grape_cost_and_grad with pinned host u/cost/grad",
                "samples_s": [round(t, 4) for t in e2e_times], "event_samples_s": [round(t, 4) for t in e2e_dev]},
        "gpu_launches": gpu_launches,
        "clocks": clk,
        "peak_hbm": peak_hbm,
    }
    if secondary:
        out["secondary"] = secondary
    out.update(extra)
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def hg_ctrl_entry_count(p) -> int:
    """Union-pattern entries that carry at least one control term (where W is accumulated)."""
    pat = abs(p.Hk[0]).astype(bool)
    for h in p.Hk[1:]:
        pat = pat + abs(h).astype(bool)
    return int(pat.nnz)


def secondary_run(name: str, precision: str, local: int, ref=None, n_steps=None, reps: int = 3):
    """Another workload or precision for context: evals/s (CUDA events) and, given an FP64 result of the
    same problem, the relative difference of cost and gradient to it."""
    import numpy as np
    import torch
    from paper_2304_06200_gb300 import GrapeProblem
    from workloads import build_config

    p = build_config(name, n_steps=n_steps)
    dev = torch.device("cuda", local)
    hg = GrapeProblem(p, device=local, precision=precision)
    u = torch.tensor(p.u0, dtype=torch.float64, device=dev)
    cost = torch.zeros((), dtype=torch.float64, device=dev)
    grad = torch.zeros((p.n_controls, p.n_steps), dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    hg.cost_device(u, cost, st)
    hg.grad_device(grad, st)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        hg.cost_device(u, cost, st)
        hg.grad_device(grad, st)
    e1.record(st)
    torch.cuda.synchronize()
    hg.sync_status(st)
    ms = e0.elapsed_time(e1) / reps
    info = hg.info()
    out = {"workload": workload_description(p), "precision": precision, "evals_per_s": round(1e3 / ms, 4),
           "ms_per_eval": round(ms, 3), "cluster_fwd": info["cluster_forward"], "cluster_bwd": info["cluster"],
           "backward_mode": info["backward_mode"], "gradient_team_ctas": info["grad_cluster"]}
    if ref is not None:
        c_ref, g_ref = ref
        g = grad.cpu().numpy()
        out["cost_rel_diff_vs_fp64"] = abs(float(cost.item()) - c_ref) / abs(c_ref)
        out["grad_rel_diff_vs_fp64"] = float(np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref))
    hg.close()
    return out


def _timed_eval(hg, u, cost, grad, reps=1):
    import torch
    hg.cost_and_grad_device(u, cost, grad)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        hg.cost_and_grad_device(u, cost, grad)
    e1.record()
    torch.cuda.synchronize()
    hg.sync_status()
    return e0.elapsed_time(e1) / reps


def checkpoint_sweep(name, local, n_steps=None):
    """Checkpoint spacing M: evals/s and peak HBM of the evaluation.  Three-stage backward with every
    state stored (M = 1) and with segments of M in {50, 200, 1000} recomputed from checkpoints (also
    with short blocks, the least memory), and the fused backward that re-propagates between
    checkpoints M apart (Sec. III.C; Table I's memory column)."""
    import torch
    from paper_2304_06200_gb300 import GrapeProblem
    from workloads import build_config

    p = build_config(name, n_steps=n_steps)
    dev = torch.device("cuda", local)
    out = []
    cases = [(3, 1, 0), (3, 50, 0), (3, 200, 0), (3, 1000, 0), (3, 200, 4), (1, 50, 0), (1, 200, 0), (1, 1000, 0)]
    for mode, M, steps in cases:
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats(dev)
        m0 = torch.cuda.memory_allocated(dev)
        hg = GrapeProblem(p, device=local, ckpt_every=M, backward_mode=mode, block_steps=steps)
        u = torch.tensor(p.u0, dtype=torch.float64, device=dev)
        cost = torch.zeros((), dtype=torch.float64, device=dev)
        grad = torch.zeros_like(u)
        ms = _timed_eval(hg, u, cost, grad)
        peak = torch.cuda.max_memory_allocated(dev) - m0
        inf = hg.info()
        out.append({"backward_mode": inf["backward_mode"], "M": inf["ckpt_every"], "steps_per_block": inf["block_steps"],
                    "evals_per_s": round(1e3 / ms, 4), "peak_bytes": int(peak), "problem_bytes": int(inf["device_bytes"]),
                    "cost": float(cost.item()), "grad_norm": float(torch.linalg.norm(grad).item())})
        hg.close()
        del u, cost, grad
    return out


def families_compare(local, n_steps=500):
    """The other Hamiltonian families at a few hundred to a thousand levels: three transmons (Hadamard
    gate, 8 levels each, d = 512), a 10-qubit chain (d = 1024) and a fluxonium pair (24 oscillator
    levels each, d = 576); N = 500 steps, controls at 3x their seeded amplitude, FP64 and FP32 bulk."""
    import numpy as np
    import torch
    from paper_2304_06200_gb300 import GrapeProblem
    from workloads import fluxonium_problem, hadamard3_problem, qubit_chain_problem

    dev = torch.device("cuda", local)
    out = {}
    for name, build, size, dt in (("h2_three_transmons", hadamard3_problem, 8, 0.5),
                                  ("h3_qubit_chain", qubit_chain_problem, 10, 0.2),
                                  ("h4_fluxonium_pair", fluxonium_problem, 24, 0.05)):
        p = build(size, n_steps, dt, seed=70 + size)
        res = {"dim": int(p.dim), "controls": len(p.Hk), "states": int(p.psi0.shape[1]), "N": n_steps, "dt_ns": dt}
        ref = None
        for prec in ("fp64", "fp32_bulk"):
            hg = GrapeProblem(p, device=local, precision=prec)
            u = torch.tensor(p.u0 * 3.0, dtype=torch.float64, device=dev)
            cost = torch.zeros((), dtype=torch.float64, device=dev)
            grad = torch.zeros_like(u)
            ms = _timed_eval(hg, u, cost, grad, reps=3)
            inf = hg.info()
            r = {"evals_per_s": round(1e3 / ms, 3), "ms_per_eval": round(ms, 2), "cluster_fwd": inf["cluster_forward"],
                 "cluster_bwd": inf["cluster"], "backward_mode": inf["backward_mode"],
                 "taylor_terms_per_sweep": inf["total_terms"], "union_nnz": inf["union_nnz"]}
            g = grad.cpu().numpy()
            if ref is None:
                ref = (float(cost.item()), g)
                r["cost"] = ref[0]
            else:
                r["cost_rel_diff_vs_fp64"] = abs(float(cost.item()) - ref[0]) / abs(ref[0])
                r["grad_rel_diff_vs_fp64"] = float(np.linalg.norm(g - ref[1]) / np.linalg.norm(ref[1]))
            res[prec] = r
            hg.close()
        out[name] = res
    return out


def optimize_compare(local, n_iter=20):
    """Steepest descent u <- u - eta grad (Eq. (4)) on c1_state_transfer_d30 and c2_gate_d80:
    grape_optimize, one recorded CUDA graph per iteration with u resident on the device, against a
    host loop of grape_cost_and_grad plus a NumPy update, at the same step size: the largest
    eta = 2^-k * 0.1 |u| / |grad| (k = 0..12) whose first two iterations lower the cost.  Wall time of
    the whole call on the host for both (both return host results)."""
    import numpy as np
    import torch
    from paper_2304_06200_gb300 import GrapeProblem
    from workloads import build_config

    out = {}
    for name in ("c1_state_transfer_d30", "c2_gate_d80"):
        p = build_config(name)
        hg = GrapeProblem(p, device=local)
        _, g0 = hg.cost_and_grad(p.u0)
        eta = 0.1 * float(np.linalg.norm(p.u0) / np.linalg.norm(g0))
        for _ in range(13):
            _, c2 = hg.optimize(p.u0, 3, eta)      # also records the iteration graph for this eta
            if c2[2] < c2[1] < c2[0]:
                break
            eta *= 0.5
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u_g, costs_g = hg.optimize(p.u0, n_iter, eta)
        t1 = time.perf_counter()
        u = np.array(p.u0, dtype=np.float64)
        costs_h = []
        t2 = time.perf_counter()
        for _ in range(n_iter):
            c, g = hg.cost_and_grad(u)
            costs_h.append(c)
            u = u - eta * g
        t3 = time.perf_counter()
        hg.close()
        costs_h = np.array(costs_h)
        out[name] = {"workload": workload_description(p), "iterations": n_iter, "eta": eta,
                     "graph_ms_per_iter": round((t1 - t0) * 1e3 / n_iter, 3),
                     "host_loop_ms_per_iter": round((t3 - t2) * 1e3 / n_iter, 3),
                     "cost_first": float(costs_g[0]), "cost_last": float(costs_g[-1]),
                     "monotone": bool(np.all(np.diff(costs_g) < 0)),
                     "max_cost_rel_diff_graph_vs_host": float(np.max(np.abs(costs_g - costs_h) / np.abs(costs_h))),
                     "u_rel_diff_graph_vs_host": float(np.linalg.norm(u_g - u) / np.linalg.norm(u))}
    return out


def c4_compare(local):
    """d = 16000, 16 states, N = 4000: FP32 bulk against the plain FP64 kernels (same problem)."""
    import numpy as np
    import torch
    from paper_2304_06200_gb300 import GrapeProblem
    from workloads import build_config

    p = build_config("c4_gate_d16000")
    dev = torch.device("cuda", local)
    res = {}
    ref = None
    for prec in ("fp64", "fp32_bulk"):
        hg = GrapeProblem(p, device=local, precision=prec)
        u = torch.tensor(p.u0, dtype=torch.float64, device=dev)
        cost = torch.zeros((), dtype=torch.float64, device=dev)
        grad = torch.zeros_like(u)
        ms = _timed_eval(hg, u, cost, grad)
        inf = hg.info()
        r = {"evals_per_s": round(1e3 / ms, 5), "ms_per_eval": round(ms, 1), "cluster_fwd": inf["cluster_forward"],
             "cluster_bwd": inf["cluster"], "backward_mode": inf["backward_mode"],
             "taylor_terms_per_sweep": inf["total_terms"], "device_bytes": inf["device_bytes"]}
        g = grad.cpu().numpy()
        if ref is None:
            ref = (float(cost.item()), g)
        else:
            r["cost_rel_diff_vs_fp64"] = abs(float(cost.item()) - ref[0]) / abs(ref[0])
            r["grad_rel_diff_vs_fp64"] = float(np.linalg.norm(g - ref[1]) / np.linalg.norm(ref[1]))
        res[prec] = r
        hg.close()
    res["workload"] = workload_description(p)
    res["speedup_fp32_bulk_over_fp64"] = round(res["fp64"]["ms_per_eval"] / res["fp32_bulk"]["ms_per_eval"], 2)
    return res


def dense_problem_d2048(n_steps):
    """Transmon (8 levels) x cavity (256 levels), d = 2048, stored dense, 16 states, dt = 0.5 ns."""
    from workloads.transmon import _gate_problem, _subspace_two, transmon_cavity

    H0, Hk = transmon_cavity(8, 256)
    dim = 2048
    omega = np.array([1.0 if (j // 256) == 7 else 0.0 for j in range(dim)])
    idx = [t * 256 + c for t in (0, 1) for c in range(8)]
    return _gate_problem("dense_d2048", H0.toarray(), [h.toarray() for h in Hk], dim, idx, 0.5, n_steps, 4, omega,
                         1.0, 1.0, 1e-2, 1e-10, {"stored": "dense"})


def dense_compare(local, n_steps):
    """Tensor-core dense path (tcgen05, FP16/BF16 hi/lo operand pairs, FP32 accumulation) at d = 2048,
    16 states: on a drift with every element non-zero (GUE, 11 qubits; the sparse kernels refuse it),
    and on the transmon-cavity Hamiltonian stored dense (against the FP64 sparse kernels)."""
    import torch
    from paper_2304_06200_gb300 import GrapeError, GrapeProblem
    from workloads import dense_register_gate

    dev = torch.device("cuda", local)
    bf16_peak, bf16_src = 1900.0, "fallback 1.9 PFLOP/s (no MEASURED_PEAKS.json)"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16_peak, bf16_src = float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        pass
    out = {}
    for key, p in (("gue_dense_drift", dense_register_gate(n_steps=n_steps)),
                   ("transmon_stored_dense", dense_problem_d2048(n_steps))):
        res = {"workload": workload_description(p) + ", H stored dense"}
        ref = None
        for prec in ("fp64", "tc_fp16", "tc_bf16"):
            try:
                hg = GrapeProblem(p, device=local, precision=prec)
            except GrapeError as exc:
                res[prec] = {"unsupported": str(exc).split(": ", 1)[-1][:160]}
                continue
            u = torch.tensor(p.u0, dtype=torch.float64, device=dev)
            cost = torch.zeros((), dtype=torch.float64, device=dev)
            grad = torch.zeros_like(u)
            hg.cost_device(u, cost)
            hg.grad_device(grad)
            torch.cuda.synchronize()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            hg.cost_device(u, cost)
            e[1].record()
            hg.grad_device(grad)
            e[2].record()
            torch.cuda.synchronize()
            hg.sync_status()
            inf = hg.info()
            fwd_ms, bwd_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
            r = {"ms_per_eval": round(fwd_ms + bwd_ms, 2), "fwd_ms": round(fwd_ms, 2), "bwd_ms": round(bwd_ms, 2),
                 "taylor_terms_per_sweep": inf["total_terms"]}
            g = grad.cpu().numpy()
            if ref is None:
                ref = (prec, float(cost.item()), g)
            else:
                r[f"cost_rel_diff_vs_{ref[0]}"] = abs(float(cost.item()) - ref[1]) / abs(ref[1])
                r[f"grad_rel_diff_vs_{ref[0]}"] = float(np.linalg.norm(g - ref[2]) / np.linalg.norm(ref[2]))
            if prec.startswith("tc"):
                # tensor work issued per forward product: 2 operators x 3 hi/lo products x 2 d^2 N_real;
                # the complex product itself is 8 d^2 n flops
                nreal = ((2 * p.n_states + 15) // 16) * 16
                issued = inf["total_terms"] * 2 * 3 * 2.0 * p.dim * p.dim * nreal
                alg = inf["total_terms"] * 8.0 * p.dim * p.dim * p.n_states
                r["forward_issued_tensor_tflops"] = round(issued / (fwd_ms / 1e3) / 1e12, 2)
                r["forward_algorithmic_tflops"] = round(alg / (fwd_ms / 1e3) / 1e12, 2)
                r["forward_issued_frac_of_bf16_peak"] = round(issued / (fwd_ms / 1e3) / 1e12 / bf16_peak, 4)
                r["bf16_peak"] = bf16_src
                r["forward_us_per_term"] = round(fwd_ms * 1e3 / inf["total_terms"], 2)
                r["operator_bytes_per_term"] = 4 * p.dim * p.dim * 2
                r["forward_l2_gbs"] = round(r["operator_bytes_per_term"] * inf["total_terms"] / (fwd_ms / 1e3) / 1e9, 1)
            res[prec] = r
            hg.close()
        out[key] = res
    return out


def _timed_fwd_bwd(hg, p, u0, dev, reps=3):
    """Median forward / backward milliseconds of one evaluation (CUDA events), plus its cost and gradient."""
    import torch
    u = torch.tensor(u0, dtype=torch.float64, device=dev)
    cost = torch.zeros((), dtype=torch.float64, device=dev)
    grad = torch.zeros_like(u)
    hg.cost_device(u, cost)
    hg.grad_device(grad)
    torch.cuda.synchronize()
    f, b = [], []
    for _ in range(reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        hg.cost_device(u, cost)
        e[1].record()
        hg.grad_device(grad)
        e[2].record()
        torch.cuda.synchronize()
        f.append(e[0].elapsed_time(e[1]))
        b.append(e[1].elapsed_time(e[2]))
    hg.sync_status()
    fwd, bwd = float(np.median(f)), float(np.median(b))
    return {"ms_per_eval": round(fwd + bwd, 3), "fwd_ms": round(fwd, 3), "bwd_ms": round(bwd, 3)}, \
        float(cost.item()), grad.cpu().numpy()


def eig_compare(local):
    """Eigendecomposition propagators (App. F) against the Taylor kernels (Sec. III.B), both FP64.

    Two workloads: the d = 80 transmon-cavity gate (8 columns, sparse H, N = 1000) and a dense
    random d = 96 full-rank gate (96 columns, every matrix element non-zero, N = 500).
    """
    import torch
    from paper_2304_06200_gb300 import GrapeProblem
    from workloads import build_config, random_problem

    dev = torch.device("cuda", local)
    out = {}
    cases = [("c2_gate_d80", build_config("c2_gate_d80"), 1.0),
             ("dense_random_d96_full_gate", random_problem(96, 4, 96, 500, seed=96, dt=0.3, density=1.0, tau=1e-10),
              1.0)]
    for name, p, scale in cases:
        u0 = p.u0 * scale
        res = {"workload": workload_description(p)}
        ref = None
        for prop in ("taylor", "eig"):
            hg = GrapeProblem(p, device=local, propagator=prop)
            r, c, g = _timed_fwd_bwd(hg, p, u0, dev)
            if prop == "taylor":
                r["taylor_terms_per_sweep"] = hg.info()["total_terms"]
                ref = (c, g)
            else:
                r["cost_rel_diff_vs_taylor"] = abs(c - ref[0]) / abs(ref[0])
                r["grad_rel_diff_vs_taylor"] = float(np.linalg.norm(g - ref[1]) / np.linalg.norm(ref[1]))
            res[prop] = r
            hg.close()
        res["speedup_eig_over_taylor"] = round(res["taylor"]["ms_per_eval"] / res["eig"]["ms_per_eval"], 2)
        out[name] = res
    return out


def batch_compare(local, tune=False):
    """64 uneven instances in one graph launch (FP32 bulk): the automatic recording, the work queue forced
    (single-CTA members in two persistent launches, the rest on lanes), lanes only, and the automatic one
    with the d = 4000 members in teams of 8, against the same 64 one at a time in plain FP64."""
    import numpy as np
    import torch
    from paper_2304_06200_gb300 import GrapeBatch, GrapeProblem, autotune
    from workloads import batch_instances

    insts = batch_instances()
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    members = []
    tune_report = []
    for p in insts:
        if tune:
            hg, rep = autotune(p, precision="fp32_bulk", device=local, probe_steps=32, m_caps=(0, 30),
                               clusters=[0, 1, 4, 8, 16], ckpt_choices=(0, 200))
            tune_report.append({"name": p.name, "cluster": rep["cluster"], "m_max": rep["m_max"],
                                "ckpt_every": rep["ckpt_every"]})
        else:
            hg = GrapeProblem(p, device=local, precision="fp32_bulk")
        members.append(hg)
    create_s = time.perf_counter() - t0
    # throughput variant: the d = 4000 members with teams of 8 CTAs (fewer barriers per unit of work;
    # in a batch the SMs are shared, so per-SM efficiency counts more than one member's latency)
    members_cl8 = [GrapeProblem(p, device=local, precision="fp32_bulk", cluster=8) if p.dim >= 4000 else hg
                   for p, hg in zip(insts, members)]
    us = [torch.tensor(p.u0, dtype=torch.float64, device=dev) for p in insts]
    res = {"instances": len(insts)}
    outs = {}
    for name, qc, mem in (("automatic", 0, members), ("queue_forced", 152, members), ("lanes_only", -1, members),
                          ("automatic_big_teams_of_8", 0, members_cl8)):
        t1 = time.perf_counter()
        batch = GrapeBatch(mem, n_streams=16, queue_ctas=qc)
        build_s = time.perf_counter() - t1
        grads = [torch.zeros_like(u) for u in us]
        costs = torch.zeros(len(insts), dtype=torch.float64, device=dev)
        batch.cost_and_grad_device(us, costs, grads)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record()
        for _ in range(reps):
            batch.cost_and_grad_device(us, costs, grads)
        e1.record()
        torch.cuda.synchronize()
        for m in members:
            m.sync_status()
        ms = e0.elapsed_time(e1) / reps
        outs[name] = (costs.cpu().numpy(), [g.cpu().numpy() for g in grads])
        res[name] = {"ms_per_eval_of_all": round(ms, 2), "evals_per_s": round(len(insts) * 1e3 / ms, 3),
                     "record_s": round(build_s, 1), **batch.info()}
        batch.close()
    for m in set(members) | set(members_cl8):
        m.close()
    # the same 64, one at a time, plain FP64 kernels
    seq_ms = 0.0
    err = {k: [0.0, 0.0] for k in outs}
    for i, p in enumerate(insts):
        hg = GrapeProblem(p, device=local, precision="fp64")
        cost = torch.zeros((), dtype=torch.float64, device=dev)
        g64 = torch.zeros_like(us[i])
        ms = _timed_eval(hg, us[i], cost, g64)
        seq_ms += ms
        c = float(cost.item())
        g = g64.cpu().numpy()
        for k, (cb, gb) in outs.items():
            err[k][0] = max(err[k][0], abs(cb[i] - c) / abs(c))
            err[k][1] = max(err[k][1], float(np.linalg.norm(gb[i] - g) / np.linalg.norm(g)))
        hg.close()
    for k in outs:
        res[k]["max_cost_rel_diff_vs_fp64"] = err[k][0]
        res[k]["max_grad_rel_diff_vs_fp64"] = err[k][1]
    dims = sorted({p.dim for p in insts})
    res.update({"dims": dims, "counts": {d: sum(p.dim == d for p in insts) for d in dims},
                "sequential_fp64_ms": round(seq_ms, 1),
                "sequential_fp64_evals_per_s": round(len(insts) * 1e3 / seq_ms, 3),
                "speedup_automatic_over_sequential_fp64": round(seq_ms / res["automatic"]["ms_per_eval_of_all"], 2),
                "speedup_teams_of_8_over_sequential_fp64": round(seq_ms / res["automatic_big_teams_of_8"]["ms_per_eval_of_all"], 2),
                "create_s": round(create_s, 1), "autotuned": tune, "tune": tune_report[:8]})
    return res


# ------------------------------------------------------------------ reference arm (CPU oracle)

def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    from workloads import build_config

    p = build_config(args.workload)
    # warm-up: the oracle has no compiled state to warm beyond the BLAS/LAPACK thread pools, which a
    # small instance wakes as well as a full step (keeps the untimed part of the run short)
    for _ in range(max(args.warmup, 0)):
        oracle_sample("c1_state_transfer_d30")
    secs = 0.0
    steps = 0
    for _ in range(args.steps):
        s, n = oracle_sample(args.workload)
        secs += s
        steps += n
    per_eval = secs / steps * p.n_steps
    value = 1.0 / per_eval
    cores = oracle_threads()
    sample = (f"oracle (numpy eigh, stored states, divided differences), each step one of the {p.n_steps} time "
              f"steps of the workload, scaled to one full evaluation")
    out = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": max(args.gpus, 1), "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": per_eval * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": workload_description(p), "parallelism": "host cores"},
           "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main(argv=None):
    warnings.filterwarnings("ignore", message=".*[Ss]parse.*")
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
