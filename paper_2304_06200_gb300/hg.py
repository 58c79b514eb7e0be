"""Python binding of the HG GRAPE C ABI: marshals arrays, owns the problem handle, exposes autograd.

Every step of the evaluation runs in the CUDA library; this module only converts
operators to CSR arrays, passes pointers and streams, and (optionally) routes the
library's device allocations through PyTorch's caching allocator so that
``torch.cuda.max_memory_allocated`` accounts for them.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi
from ._abi import GrapeBatchInfo, GrapeDesc, GrapeInfo, GrapeOp, check, lib

PRECISIONS = {"fp64": _abi.GRAPE_FP64, "fp32_bulk": _abi.GRAPE_FP32_BULK, "tc_fp16": _abi.GRAPE_TC_FP16,
              "tc_bf16": _abi.GRAPE_TC_BF16}
PROPAGATORS = {"taylor": _abi.GRAPE_PROP_TAYLOR, "eig": _abi.GRAPE_PROP_EIG}


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _csr_arrays(m, dim):
    """(rowptr int64, colind int32, values interleaved float64) of a scipy sparse or dense matrix."""
    import scipy.sparse as sp

    csr = sp.csr_matrix(m, dtype=np.complex128)
    csr.sum_duplicates()
    if csr.shape != (dim, dim):
        raise ValueError(f"operator shape {csr.shape} != ({dim}, {dim})")
    rowptr = np.ascontiguousarray(csr.indptr, dtype=np.int64)
    col = np.ascontiguousarray(csr.indices, dtype=np.int32)
    vals = np.ascontiguousarray(csr.data, dtype=np.complex128).view(np.float64)
    return rowptr, col, vals


class _TorchAllocator:
    """Device allocations through torch's caching allocator (keeps the ctypes callbacks alive)."""

    def __init__(self, device: int):
        import torch

        self.torch = torch
        self.device = device

        def _alloc(nbytes, _ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device))
            except Exception:  # out of memory -> NULL -> GRAPE_ENOMEM
                return None

        def _free(ptr, _nbytes, _ctx):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self.alloc = _abi.ALLOC_FN(_alloc)
        self.free = _abi.FREE_FN(_free)


class GrapeProblem:
    """One HG GRAPE problem on one GPU (see ``include/grape_hg.h`` for the definition of the cost).

    ``problem`` is any object with the attributes of ``workloads.Problem``: dim, dt,
    n_steps, H0, Hk (scipy sparse or dense), psi0, target (dim x n complex), omega
    (dim real or None), w_fid, w_forbid, w_amp, tau.
    """

    def __init__(self, problem, precision: str = "fp64", ckpt_every: int = 0, cluster: int = 0, device: int = 0,
                 tau: float | None = None, m_max: int = 0, torch_allocator: bool = True, n_steps: int | None = None,
                 backward_mode: int = 0, bulk_norm_cap: float = 0.0, propagator: str = "taylor",
                 grad_cluster: int = 0, block_steps: int = 0):
        L = lib()
        self._lib = L
        self.dim = int(problem.dim)
        self.K = len(problem.Hk)
        self.N = int(problem.n_steps if n_steps is None else n_steps)
        self.n = int(np.asarray(problem.psi0).shape[1])
        self.device = int(device)
        u0 = getattr(problem, "u0", None)   # the workload's seeded controls, when it has them (K x N)
        self.u0 = None if u0 is None or np.shape(u0) != (self.K, self.N) else np.ascontiguousarray(u0, dtype=np.float64)
        self._keep = []
        ops = [_csr_arrays(problem.H0, self.dim)] + [_csr_arrays(h, self.dim) for h in problem.Hk]
        self._keep.append(ops)

        def mkop(arrs):
            rp, ci, va = arrs
            return GrapeOp(_abi.GRAPE_CSR, int(ci.shape[0]), rp.ctypes.data_as(C.POINTER(C.c_int64)),
                           ci.ctypes.data_as(C.POINTER(C.c_int32)), _dptr(va))

        hk_arr = (GrapeOp * max(self.K, 1))(*[mkop(o) for o in ops[1:]])
        psi0 = np.asfortranarray(np.asarray(problem.psi0, dtype=np.complex128))
        target = np.asfortranarray(np.asarray(problem.target, dtype=np.complex128))
        psi0_c = np.ascontiguousarray(psi0.T).view(np.float64)      # column h contiguous
        target_c = np.ascontiguousarray(target.T).view(np.float64)
        omega = None if problem.omega is None else np.ascontiguousarray(problem.omega, dtype=np.float64)
        self._keep += [hk_arr, psi0_c, target_c, omega]
        d = GrapeDesc()
        d.dim = self.dim
        d.n_controls = self.K
        d.n_steps = self.N
        d.n_states = self.n
        d.dt = float(problem.dt)
        d.H0 = mkop(ops[0])
        d.Hk = C.cast(hk_arr, C.POINTER(GrapeOp))
        d.psi0 = _dptr(psi0_c)
        d.target = _dptr(target_c)
        d.omega_diag = _dptr(omega) if omega is not None else C.POINTER(C.c_double)()
        d.w_fid, d.w_forbid, d.w_amp = float(problem.w_fid), float(problem.w_forbid), float(problem.w_amp)
        d.tau = float(problem.tau if tau is None else tau)
        d.m_max = int(m_max)
        d.ckpt_every = int(ckpt_every)
        d.precision = PRECISIONS[precision]
        d.cluster = int(cluster)
        d.device = self.device
        self._alloc = None
        if torch_allocator:
            self._alloc = _TorchAllocator(self.device)
            d.alloc = self._alloc.alloc
            d.free = self._alloc.free
        else:
            d.alloc = _abi.ALLOC_FN()
            d.free = _abi.FREE_FN()
        d.alloc_ctx = None
        d.backward_mode = int(backward_mode)
        d.bulk_norm_cap = float(bulk_norm_cap)
        d.w_tint = float(getattr(problem, "w_tint", 0.0))
        d.propagator = PROPAGATORS[propagator]
        d.grad_cluster = int(grad_cluster)
        d.block_steps = int(block_steps)
        handle = C.c_void_p()
        check(L.grape_problem_create(C.byref(d), C.byref(handle)), "grape_problem_create")
        self._h = handle
        self.precision = precision
        self.propagator = propagator
        self.forward_count = 0   # forward sweeps run on this problem (the stored sweep state is the last one's)

    # ------------------------------------------------------------------ host-pointer API
    def cost_and_grad(self, u: np.ndarray, want_grad: bool = True):
        """(cost, grad) with host arrays; u has shape (K, N)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        if u.shape != (self.K, self.N):
            raise ValueError(f"u shape {u.shape} != {(self.K, self.N)}")
        cost = np.zeros(1)
        grad = np.zeros((self.K, self.N)) if want_grad else None
        self.forward_count += 1
        check(self._lib.grape_cost_and_grad(self._h, u.ctypes.data, cost.ctypes.data,
                                            grad.ctypes.data if want_grad else None, 0, None),
              "grape_cost_and_grad")
        return float(cost[0]), grad

    def cost(self, u: np.ndarray) -> float:
        u = np.ascontiguousarray(u, dtype=np.float64)
        cost = np.zeros(1)
        self.forward_count += 1
        check(self._lib.grape_cost(self._h, u.ctypes.data, cost.ctypes.data, 0, None), "grape_cost")
        return float(cost[0])

    # ------------------------------------------------------------------ device-pointer API (torch tensors)
    def cost_and_grad_device(self, u, cost, grad=None, stream=None):
        """Asynchronous evaluation on device tensors (float64, contiguous) on ``stream`` (default: torch's current)."""
        import torch

        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        self.forward_count += 1
        check(self._lib.grape_cost_and_grad(self._h, u.data_ptr(), cost.data_ptr(),
                                            grad.data_ptr() if grad is not None else None, 1, st),
              "grape_cost_and_grad")

    def cost_device(self, u, cost, stream=None):
        import torch

        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        self.forward_count += 1
        check(self._lib.grape_cost(self._h, u.data_ptr(), cost.data_ptr(), 1, st), "grape_cost")

    def grad_device(self, grad, stream=None):
        import torch

        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        check(self._lib.grape_grad(self._h, grad.data_ptr(), 1, st), "grape_grad")

    def sync_status(self, stream=None):
        import torch

        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        check(self._lib.grape_sync_status(self._h, st), "grape_sync_status")

    def optimize(self, u: np.ndarray, n_iter: int, eta: float):
        """Steepest descent (one recorded CUDA graph per iteration): returns (final u, costs per iteration)."""
        u = np.array(u, dtype=np.float64, order="C", copy=True)
        costs = np.zeros(int(n_iter))
        self.forward_count += 1
        check(self._lib.grape_optimize(self._h, u.ctypes.data, int(n_iter), float(eta), costs.ctypes.data, 0, None),
              "grape_optimize")
        return u, costs

    # ------------------------------------------------------------------ introspection
    def info(self) -> dict:
        inf = GrapeInfo()
        check(self._lib.grape_problem_info(self._h, C.byref(inf)), "grape_problem_info")
        return {f: getattr(inf, f) for f, _ in GrapeInfo._fields_}

    def set_kernel_tracing(self, enable: bool = True):
        """Record CUDA events around every sweep-kernel launch (measurement support)."""
        check(self._lib.grape_set_kernel_tracing(self._h, 1 if enable else 0), "grape_set_kernel_tracing")

    def kernel_times(self) -> dict:
        """Summed event durations (ms) and launch counts per sweep kernel since the last call."""
        from ._abi import GrapeKernelTimes
        t = GrapeKernelTimes()
        check(self._lib.grape_kernel_times(self._h, C.byref(t)), "grape_kernel_times")
        names = ["k_forward", "k_costate", "k_gradient", "k_backward", "k_forward_recompute"]
        return {nm: {"launches": int(t.launches[i]), "ms": float(t.ms[i])} for i, nm in enumerate(names)}

    def schedule(self):
        m = np.zeros(self.N, dtype=np.int32)
        s = np.zeros(self.N, dtype=np.int32)
        x = np.zeros(self.N, dtype=np.float64)
        check(self._lib.grape_step_schedule(self._h, m.ctypes.data, s.ctypes.data, x.ctypes.data), "grape_step_schedule")
        return m, s, x

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.grape_problem_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GrapeBatch:
    """Many independent problems evaluated by one CUDA-graph launch (``grape_batch_create``).

    Members with single-CTA column teams run in the persistent work-queue kernels, the others on
    graph lanes.  ``queue_ctas``: 0 automatic, > 0 that many CTAs, < 0 no queue.  ``u_warm``: the
    controls of the warm evaluation before the recording (default: each member's workload ``u0``
    when it has one).  The batch keeps references to the members so they outlive it.
    """

    def __init__(self, problems, n_streams: int = 8, queue_ctas: int = 0, u_warm=None):
        L = lib()
        self._lib = L
        self.problems = list(problems)
        handles = (C.c_void_p * len(self.problems))(*[p._h.value for p in self.problems])
        if u_warm is None:
            u_warm = [p.u0 for p in self.problems]
        self._u_warm = [None if u is None else np.ascontiguousarray(u, dtype=np.float64) for u in u_warm]
        warm = (C.c_void_p * len(self.problems))(*[0 if u is None else u.ctypes.data for u in self._u_warm])
        h = C.c_void_p()
        check(L.grape_batch_create(handles, len(self.problems), int(n_streams), int(queue_ctas), warm, C.byref(h)),
              "grape_batch_create")
        self._h = h

    def info(self) -> dict:
        out = GrapeBatchInfo()
        check(self._lib.grape_batch_info(self._h, C.byref(out)), "grape_batch_info")
        return {name: getattr(out, name) for name, _ in GrapeBatchInfo._fields_}

    def cost_and_grad(self, us):
        """Host arrays: list of (K_i, N_i) controls -> (costs array, list of gradients)."""
        us = [np.ascontiguousarray(u, dtype=np.float64) for u in us]
        grads = [np.zeros_like(u) for u in us]
        costs = np.zeros(len(us))
        up = (C.c_void_p * len(us))(*[u.ctypes.data for u in us])
        gp = (C.c_void_p * len(us))(*[g.ctypes.data for g in grads])
        for p in self.problems:
            p.forward_count += 1
        check(self._lib.grape_batch_cost_and_grad(self._h, up, costs.ctypes.data, gp, 0, None), "grape_batch_cost_and_grad")
        return costs, grads

    def cost_and_grad_device(self, us, costs, grads, stream=None):
        """Device tensors: list of (K_i, N_i) float64 controls, costs (count,), list of gradient tensors."""
        import torch

        st = (stream or torch.cuda.current_stream(self.problems[0].device)).cuda_stream
        up = (C.c_void_p * len(us))(*[u.data_ptr() for u in us])
        gp = (C.c_void_p * len(us))(*[g.data_ptr() for g in grads])
        for p in self.problems:
            p.forward_count += 1
        check(self._lib.grape_batch_cost_and_grad(self._h, up, costs.data_ptr(), gp, 1, st), "grape_batch_cost_and_grad")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.grape_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def checkpoint_bytes(ckpt_every: int, n_steps: int, dim: int, n_states: int) -> int:
    """Device bytes of the stored checkpoints for spacing M = ckpt_every (0: the default
    min(50, N); negative: none): floor((N - 1) / M) states of dim x n_states complex128."""
    m_eff = ckpt_every if ckpt_every != 0 else min(50, n_steps)
    if m_eff < 0:
        return 0
    return ((n_steps - 1) // max(m_eff, 1)) * dim * n_states * 16


def select_candidate(timed, tie: float = 0.02) -> dict:
    """The autotuner's choice among timed candidates (dicts with "ms" and
    "checkpoint_bytes_full_N"): the fastest, unless others lie within ``tie`` (relative) of it, in
    which case the one storing the fewest checkpoint bytes (then the faster of equals)."""
    if not timed:
        raise RuntimeError("autotune: no candidate configuration was accepted")
    fastest = min(r["ms"] for r in timed)
    near = [r for r in timed if r["ms"] <= fastest * (1.0 + tie)]
    return min(near, key=lambda r: (r["checkpoint_bytes_full_N"], r["ms"]))


def autotune(problem, precision: str = "fp64", device: int = 0, probe_steps: int = 48, backward_mode: int = 1,
             clusters=None, m_caps=(0, 30, 20), ckpt_choices=(0,), repeats: int = 2, tie: float = 0.02):
    """Pick the team size (CTAs per column), Taylor-order cap and checkpoint spacing M.

    Each candidate is timed (CUDA events, after one warm-up) on the first ``probe_steps`` steps of the
    problem.  The fastest wins; among candidates within ``tie`` (relative) of it, the one holding the
    least device memory (larger M stores fewer checkpoints).  Returns ``(GrapeProblem for the full
    problem, report)``.  Candidates whose descriptor is rejected (shared memory, co-residency) are
    skipped.  The Taylor-order cap changes the (m, s) the paper's rule returns (a smaller cap forces
    more substeps), never the tolerance; M changes the memory and the re-propagation drift bound,
    not the arithmetic between checkpoints.
    """
    import torch

    if clusters is None:
        clusters = [0] + [c for c in (1, 2, 4, 8, 12, 16) if c <= problem.dim]
    N = problem.n_steps
    ns = min(N, probe_steps)
    u = torch.tensor(np.asarray(problem.u0)[:, :ns], dtype=torch.float64, device=f"cuda:{device}")
    cost = torch.zeros((), dtype=torch.float64, device=u.device)
    grad = torch.zeros_like(u)
    report = []
    timed = []
    for cl in clusters:
        for mc in m_caps:
            for M in ckpt_choices:
                # the probe covers ns steps: checkpoints are spaced as they would be in the full problem
                # up to ns, and their memory is scaled to the full N below
                try:
                    hg = GrapeProblem(problem, precision=precision, cluster=cl, device=device, m_max=mc,
                                      n_steps=ns, backward_mode=backward_mode, ckpt_every=M)
                except Exception as exc:  # rejected configuration
                    report.append({"cluster": cl, "m_max": mc, "ckpt_every": M, "skipped": str(exc)[:80]})
                    continue
                hg.cost_and_grad_device(u, cost, grad)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(repeats):
                    hg.cost_and_grad_device(u, cost, grad)
                e1.record()
                torch.cuda.synchronize()
                hg.sync_status()
                ms = e0.elapsed_time(e1) / repeats
                inf = hg.info()
                ckpt_bytes = checkpoint_bytes(M, N, problem.dim, problem.n_states)
                rec = {"cluster": cl, "m_max": mc, "ckpt_every": M, "ms": ms, "cluster_used": inf["cluster"],
                       "terms": inf["total_terms"], "checkpoint_bytes_full_N": int(ckpt_bytes)}
                report.append(rec)
                timed.append(rec)
                hg.close()
    best = select_candidate(timed, tie)
    cl, mc, M = best["cluster"], best["m_max"], best["ckpt_every"]
    full = GrapeProblem(problem, precision=precision, cluster=cl, device=device, m_max=mc, backward_mode=backward_mode,
                        ckpt_every=M)
    return full, {"cluster": cl, "m_max": mc, "ckpt_every": M, "candidates": report}


def select_ms(x: float, tau: float, sigma: int, precision: str = "fp64", m_max: int = 60, s_max: int = 4096):
    """The library's host-side (m, s) rule (Sec. III.B): returns (m, s) or None when infeasible."""
    m = C.c_int32()
    s = C.c_int32()
    st = lib().grape_select_ms(float(x), float(tau), int(sigma), PRECISIONS[precision], int(m_max), int(s_max),
                               C.byref(m), C.byref(s))
    if st == 4:
        return None
    check(st, "grape_select_ms")
    return m.value, s.value


def error_bound(x: float, m: int, s: int, sigma: int, precision: str = "fp64") -> float:
    return lib().grape_error_bound(float(x), int(m), int(s), int(sigma), PRECISIONS[precision])


def _make_function():
    import torch

    class GrapeHG(torch.autograd.Function):
        """cost = GrapeHG.apply(u, problem): forward sweep in forward(), backward sweep in backward().

        The backward sweep uses the checkpoints of the problem's last forward sweep; if another
        evaluation ran on the problem in between (a second forward, finite differences), the
        forward sweep is run again at the saved controls first.
        """

        @staticmethod
        def forward(ctx, u, prob):
            u = u.detach().to(dtype=torch.float64).contiguous()
            cost = torch.empty((), dtype=torch.float64, device=u.device)
            prob.cost_device(u, cost)
            ctx.prob = prob
            ctx.u = u
            ctx.forward_index = prob.forward_count
            return cost

        @staticmethod
        def backward(ctx, grad_out):
            prob = ctx.prob
            if prob.forward_count != ctx.forward_index:
                redo = torch.empty((), dtype=torch.float64, device=ctx.u.device)
                prob.cost_device(ctx.u, redo)
                ctx.forward_index = prob.forward_count
            g = torch.empty((prob.K, prob.N), dtype=torch.float64, device=grad_out.device)
            prob.grad_device(g)
            return grad_out * g, None

    return GrapeHG


_GRAPE_HG = None


def grape_hg():
    """The ``torch.autograd.Function`` wrapping the HG forward and backward sweeps."""
    global _GRAPE_HG
    if _GRAPE_HG is None:
        _GRAPE_HG = _make_function()
    return _GRAPE_HG
