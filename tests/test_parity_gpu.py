"""GPU parity: the CUDA HG path (through the C ABI) against the CPU FP64 oracle.

Tolerances (FP64 path): relative 1e-10 on the cost, normwise relative 1e-8 on the
gradient.  The oracle uses the exact exponential, the GPU the truncated-Taylor
approximant chosen by the paper's bound, so tau is set small enough that the
approximation error stays below these tolerances (tau <= 1e-12 here).
"""

import numpy as np
import pytest

from oracle import cost_and_grad as oracle_cost_and_grad
from oracle import select_ms as oracle_select
from workloads import build_config, random_problem

pytestmark = pytest.mark.gpu

COST_RTOL = 1e-10
GRAD_RTOL = 1e-8


def _hg(p, **kw):
    from paper_2304_06200_gb300 import GrapeProblem
    return GrapeProblem(p, **kw)


def _check(p, u, cost, grad, cost_rtol=COST_RTOL, grad_rtol=GRAD_RTOL, ref=None):
    r = ref if ref is not None else oracle_cost_and_grad(p, u)
    assert abs(cost - r.cost) <= cost_rtol * abs(r.cost), (cost, r.cost)
    gerr = np.linalg.norm(grad - r.grad) / np.linalg.norm(r.grad)
    assert gerr <= grad_rtol, gerr
    return r


def test_c1_state_transfer_full_size():
    p = build_config("c1_state_transfer_d30")
    hg = _hg(p)
    cost, grad = hg.cost_and_grad(p.u0)
    _check(p, p.u0, cost, grad)


def test_c2_gate_full_size():
    p = build_config("c2_gate_d80")
    hg = _hg(p)
    cost, grad = hg.cost_and_grad(p.u0)
    r = _check(p, p.u0, cost, grad)
    # a stronger drive exercises every cost term (C2 becomes sizeable)
    u = p.u0 * 30
    cost, grad = hg.cost_and_grad(u)
    _check(p, u, cost, grad)


@pytest.mark.parametrize("dim,K,n,N,cluster", [
    (2, 1, 1, 3, 1), (7, 2, 3, 5, 1), (33, 3, 2, 9, 2), (65, 2, 4, 6, 4), (130, 4, 3, 7, 8),
    (257, 3, 2, 5, 16), (40, 5, 1, 11, 16), (97, 1, 5, 4, 0), (31, 0, 2, 3, 0),
])
def test_random_ragged_problems(dim, K, n, N, cluster):
    """Row blocks that do not divide d (ragged last CTA, empty CTAs for d < 16 * R), every team size."""
    p = random_problem(dim, K, n, N, seed=1000 + dim + K + n + N)
    hg = _hg(p, cluster=cluster)
    assert hg.info()["cluster"] == (cluster or hg.info()["cluster"])
    if K == 0:
        cost = hg.cost(p.u0)
        r = oracle_cost_and_grad(p, p.u0)
        assert abs(cost - r.cost) <= COST_RTOL * abs(r.cost)
        return
    cost, grad = hg.cost_and_grad(p.u0)
    _check(p, p.u0, cost, grad)


def test_schedule_follows_the_paper_rule():
    """(m_n, s_n) on the device equals the oracle's direct rule on the oracle's norms (integers, exact)."""
    p = build_config("c2_gate_d80", n_steps=200)
    u = p.u0 * 20
    hg = _hg(p)
    hg.cost_and_grad(u)
    m, s, x = hg.schedule()
    sigma = hg.info()["sigma"]
    H0, Hk = p.dense()
    mism = 0
    for n in range(p.n_steps):
        H = H0 + sum(u[k, n] * Hk[k] for k in range(len(Hk)))
        xn = p.dt * np.max(np.sum(np.abs(H), axis=1))
        assert x[n] == pytest.approx(xn, rel=1e-13)
        want = oracle_select(xn, p.tau, sigma)
        if (m[n], s[n]) != want:
            mism += 1
    assert mism == 0


def test_gradient_is_derivative_of_the_gpu_cost():
    """Central differences of the GPU's own cost (schedule unchanged by the perturbation) match its gradient."""
    p = random_problem(24, 3, 2, 6, seed=77, tau=1e-12)
    hg = _hg(p)
    u = p.u0.copy()
    cost, grad = hg.cost_and_grad(u)
    m0, s0, _ = hg.schedule()
    h = 1e-6
    fd = np.zeros_like(u)
    for k in range(u.shape[0]):
        for n in range(u.shape[1]):
            up = u.copy(); up[k, n] += h
            um = u.copy(); um[k, n] -= h
            cp = hg.cost(up)
            m1, s1, _ = hg.schedule()
            cm = hg.cost(um)
            m2, s2, _ = hg.schedule()
            assert (m1 == m0).all() and (s1 == s0).all() and (m2 == m0).all() and (s2 == s0).all()
            fd[k, n] = (cp - cm) / (2 * h)
    assert np.linalg.norm(fd - grad) / np.linalg.norm(grad) < 1e-7


def test_repeat_evaluations_are_bitwise_identical():
    p = build_config("c2_gate_d80", n_steps=50)
    hg = _hg(p)
    c1, g1 = hg.cost_and_grad(p.u0)
    c2, g2 = hg.cost_and_grad(p.u0)
    assert c1 == c2
    assert np.array_equal(g1, g2)


@pytest.mark.parametrize("ckpt", [-1, 1, 7, 50])
def test_checkpoint_spacing_does_not_change_the_result(ckpt):
    p = build_config("c2_gate_d80", n_steps=120)
    u = p.u0 * 10
    ref = oracle_cost_and_grad(p, u)
    hg = _hg(p, ckpt_every=ckpt)
    cost, grad = hg.cost_and_grad(u)
    _check(p, u, cost, grad, ref=ref)


def _single_phase_entries(p, seed, diag_imag=0.0):
    """p with every off-diagonal pair of every operator made real (imaginary B_ij), imaginary (real
    B_ij) or left complex, by a seeded choice per pair; each pair stays Hermitian.  With diag_imag > 0
    the drift's diagonal gets an imaginary part that tiny (within the Hermitian check's tolerance),
    which turns the diagonal into a general entry."""
    import dataclasses

    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    kind = {}

    def fix(m, drift):
        m = sp.csr_matrix(m).tocoo()
        data = m.data.astype(np.complex128)
        for t, (i, j) in enumerate(zip(m.row, m.col)):
            if i == j:
                if drift and diag_imag:
                    data[t] = data[t].real + 1j * diag_imag
                continue
            key = (min(i, j), max(i, j))
            if key not in kind:
                kind[key] = int(rng.integers(0, 3))
            if kind[key] == 0:
                data[t] = data[t].real
            elif kind[key] == 1:
                data[t] = 1j * data[t].imag
        return sp.csr_matrix((data, (m.row, m.col)), shape=m.shape)

    q = dataclasses.replace(p, H0=fix(p.H0, True), Hk=[fix(h, False) for h in p.Hk])
    return q, [sum(1 for v in kind.values() if v == c) for c in range(3)]


@pytest.mark.parametrize("cluster,mode,diag_imag", [(4, 1, 0.0), (4, 3, 0.0), (8, 3, 0.0), (16, 1, 0.0),
                                                    (4, 3, 1e-14)])
def test_single_phase_entries_in_cluster_sweeps(cluster, mode, diag_imag):
    """Real, imaginary and general H_ij in the same rows (and a diagonal that is not exactly real):
    the one-row-per-thread cluster sweeps that apply the single-phase entries with two multiplies
    agree with the oracle and, where the diagonal is real, with a generic-loop run (one CTA)."""
    p, counts = _single_phase_entries(random_problem(600, 3, 2, 6, seed=4242, band=4, density=0.004),
                                      seed=7, diag_imag=diag_imag)
    assert min(counts) > 100
    u = p.u0 * 3
    hg = _hg(p, cluster=cluster, backward_mode=mode)
    inf = hg.info()
    assert inf["cluster"] == cluster and inf["backward_mode"] == mode
    cost, grad = hg.cost_and_grad(u)
    _check(p, u, cost, grad)
    if not diag_imag:
        c1, g1 = _hg(p, cluster=1, backward_mode=1).cost_and_grad(u)
        assert abs(cost - c1) <= 1e-13 * abs(c1)
        assert np.linalg.norm(grad - g1) <= 1e-11 * np.linalg.norm(g1)


@pytest.mark.parametrize("cluster", [1, 2, 4, 8, 16])
def test_team_sizes_agree(cluster):
    """Same problem split over 1..16 CTAs per column: identical cost and gradient within rounding."""
    p = build_config("c2_gate_d80", n_steps=40)
    u = p.u0 * 15
    ref = oracle_cost_and_grad(p, u)
    hg = _hg(p, cluster=cluster)
    cost, grad = hg.cost_and_grad(u)
    _check(p, u, cost, grad, ref=ref)


@pytest.mark.parametrize("name,N,cluster,gcl,steps,drive,prec", [
    ("c2_gate_d80", 60, 0, 0, 0, 10.0, "fp64"),
    ("c2_gate_d80", 37, 4, 2, 5, 20.0, "fp64"),
    ("c1_state_transfer_d30", 40, 16, 4, 1, 5.0, "fp64"),
    ("c2_gate_d80", 25, 12, 16, 25, 10.0, "fp64"),
    ("c1_state_transfer_d30", 21, 7, 3, 4, 3.0, "fp64"),
    ("c2_gate_d80", 30, 0, 0, 0, 10.0, "fp32_bulk"),
    ("c2_gate_d80", 30, 8, 2, 3, 10.0, "fp32_bulk"),
])
def test_three_stage_backward_matches_the_oracle(name, N, cluster, gcl, steps, drive, prec):
    """Costate chain + per-step gradient kernels on the states the forward stored: against the oracle
    and against the fused one-team backward, for team sizes 1..16 of both kernels and block lengths
    from one step to all steps (with a ragged last block)."""
    p = build_config(name, n_steps=N)
    u = p.u0 * drive
    hg = _hg(p, cluster=cluster, backward_mode=3, grad_cluster=gcl, block_steps=steps, precision=prec)
    inf = hg.info()
    assert inf["backward_mode"] == 3 and inf["ckpt_every"] == 1
    assert (gcl == 0 or inf["grad_cluster"] == gcl) and (steps == 0 or inf["block_steps"] == min(steps, N))
    cost, grad = hg.cost_and_grad(u)
    assert hg.info()["fused_fallback"] == 0
    tol = (COST_RTOL, GRAD_RTOL) if prec == "fp64" else (FP32_RTOL, FP32_RTOL)
    _check(p, u, cost, grad, *tol)
    fused = _hg(p, cluster=cluster, backward_mode=1, precision=prec)
    c1, g1 = fused.cost_and_grad(u)
    assert c1 == cost                          # same forward sweep
    gtol = 1e-12 if prec == "fp64" else 1e-6
    assert np.linalg.norm(g1 - grad) <= gtol * np.linalg.norm(g1)
    c2, g2 = hg.cost_and_grad(u)               # repeatable: block buffers and flags reset every call
    assert c2 == cost and np.array_equal(g2, grad)


@pytest.mark.parametrize("dim,K,n,N,cluster,gcl,steps", [
    (2, 1, 1, 3, 1, 1, 1), (33, 3, 2, 9, 2, 3, 4), (130, 4, 3, 7, 8, 5, 2), (257, 3, 2, 5, 16, 16, 5),
    (97, 1, 5, 4, 0, 0, 0), (65, 5, 2, 6, 4, 1, 3),
])
def test_three_stage_random_ragged_problems(dim, K, n, N, cluster, gcl, steps):
    p = random_problem(dim, K, n, N, seed=2000 + dim + K + n + N)
    hg = _hg(p, cluster=cluster, backward_mode=3, grad_cluster=gcl, block_steps=steps)
    cost, grad = hg.cost_and_grad(p.u0)
    assert hg.info()["fused_fallback"] == 0
    _check(p, p.u0, cost, grad)


@pytest.mark.parametrize("name,N,M,steps,prec", [
    ("c2_gate_d80", 60, 10, 0, "fp64"), ("c2_gate_d80", 61, 7, 3, "fp64"), ("c1_state_transfer_d30", 45, 50, 4, "fp64"),
    ("c2_gate_d80", 40, 8, 8, "fp32_bulk"), ("c2_gate_d80", 33, 2, 1, "fp64"),
])
def test_three_stage_with_recomputed_segments(name, N, M, steps, prec):
    """Checkpoints M > 1 steps apart: each segment's states are recomputed before the costate chain
    enters it (blocks never straddle segments; a ragged last segment).  Against the oracle, and the
    states held are two segments instead of all N."""
    p = build_config(name, n_steps=N)
    u = p.u0 * 10.0
    hg = _hg(p, backward_mode=3, ckpt_every=M, block_steps=steps, precision=prec)
    inf = hg.info()
    M = min(M, N)
    assert inf["backward_mode"] == 3 and inf["ckpt_every"] == M and M % inf["block_steps"] == 0
    cost, grad = hg.cost_and_grad(u)
    assert hg.info()["fused_fallback"] == 0
    tol = (COST_RTOL, GRAD_RTOL) if prec == "fp64" else (FP32_RTOL, FP32_RTOL)
    _check(p, u, cost, grad, *tol)
    c2, g2 = hg.cost_and_grad(u)
    assert c2 == cost and np.array_equal(g2, grad)
    kt = None
    hg.set_kernel_tracing(True)
    hg.kernel_times()
    hg.cost_and_grad(u)
    kt = hg.kernel_times()
    assert kt["k_forward_recompute"]["launches"] == -(-N // M)


def _weak_drift_problem():
    p = random_problem(40, 2, 2, 6, seed=77)
    p.H0 = p.H0 * 1e-3
    p.Hk = [h * 1e-3 for h in p.Hk]
    return p


def test_three_stage_block_buffers_grow_with_the_schedule():
    """The block buffers start from the drift's schedule; a call whose controls need more Taylor terms
    grows them (outside stream capture) and still runs the three stages."""
    p = _weak_drift_problem()
    hg = _hg(p, backward_mode=3, block_steps=1)
    b0 = hg.info()["device_bytes"]
    u = p.u0 * 2e4
    cost, grad = hg.cost_and_grad(u)
    inf = hg.info()
    assert inf["fused_fallback"] == 0 and inf["device_bytes"] > b0
    _check(p, u, cost, grad)


def test_three_stage_under_stream_capture_falls_back_when_the_buffers_are_small():
    """Inside a CUDA-graph capture the schedule cannot be read back: if the block buffers are too small
    for it, the device-side plan runs the fused backward instead, with the same result."""
    import torch
    p = _weak_drift_problem()
    hg = _hg(p, backward_mode=3, block_steps=1)
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream(dev)
    cost = torch.zeros((), dtype=torch.float64, device=dev)
    grad = torch.zeros((p.n_controls, p.n_steps), dtype=torch.float64, device=dev)
    u_small = torch.tensor(p.u0, dtype=torch.float64, device=dev)
    with torch.cuda.stream(s):
        hg.cost_device(u_small, cost, s)
        hg.grad_device(grad, s)
    torch.cuda.synchronize()
    assert hg.info()["fused_fallback"] == 0
    u_big = p.u0 * 2e4
    ug = torch.tensor(u_big, dtype=torch.float64, device=dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        hg.cost_device(ug, cost, s)
        hg.grad_device(grad, s)
    graph.replay()
    torch.cuda.synchronize()
    assert hg.info()["fused_fallback"] == 1
    _check(p, u_big, float(cost.item()), grad.cpu().numpy())


def test_medium_two_transmon_cavity_parity():
    """Two transmons x cavity (the d = 4000 system's structure) at d = 4*4*40 = 640, clustered."""
    from workloads.transmon import _gate_problem, _subspace_two, two_transmon_cavity
    H0, Hk = two_transmon_cavity(4, 40)
    dim = 640
    t1 = np.arange(dim) // 160
    t2 = (np.arange(dim) // 40) % 4
    omega = ((t1 == 3) | (t2 == 3)).astype(float)
    p = _gate_problem("tt4c40", H0, Hk, dim, _subspace_two(4, 40, 4, 1), 1.0, 12, 9, omega, 1.0, 1.0, 1e-2,
                      1e-12, {})
    u = p.u0 * 10
    ref = oracle_cost_and_grad(p, u)
    for cl in (0, 16):
        hg = _hg(p, cluster=cl)
        cost, grad = hg.cost_and_grad(u)
        _check(p, u, cost, grad, ref=ref)


def test_c3_full_dimension_one_step():
    """The d = 4000, 6-control, 4-state system against the oracle (one step: dense eigh at d = 4000)."""
    p = build_config("c3_gate_d4000", n_steps=1, tau=1e-12)
    hg = _hg(p)
    assert hg.info()["cluster"] > 1
    cost, grad = hg.cost_and_grad(p.u0)
    _check(p, p.u0, cost, grad)


def test_autograd_function_matches_direct_call():
    import torch
    from paper_2304_06200_gb300 import grape_hg
    p = build_config("c2_gate_d80", n_steps=30)
    hg = _hg(p)
    c_ref, g_ref = hg.cost_and_grad(p.u0)
    u = torch.tensor(p.u0, device="cuda", requires_grad=True)
    cost = grape_hg().apply(u, hg)
    (3.0 * cost).backward()
    assert float(cost) == c_ref
    np.testing.assert_allclose(u.grad.cpu().numpy(), 3.0 * g_ref, rtol=0, atol=1e-15)


def test_error_paths():
    from paper_2304_06200_gb300 import GrapeError, GrapeProblem
    p = build_config("c1_state_transfer_d30", n_steps=5)
    hg = _hg(p)
    u = p.u0.copy()
    u[1, 2] = np.nan
    with pytest.raises(GrapeError) as ei:
        hg.cost_and_grad(u)
    assert ei.value.name == "GRAPE_ENONFINITE"
    with pytest.raises(GrapeError) as ei:
        hg.cost_and_grad(p.u0 * 1e6)        # ||A||_1 beyond every feasible (m, s)
    assert ei.value.name == "GRAPE_ETOL"
    c, g = hg.cost_and_grad(p.u0)           # the problem stays usable after device-side errors
    assert np.isfinite(c) and np.all(np.isfinite(g))
    q = build_config("c1_state_transfer_d30", n_steps=5)
    q.Hk[0] = q.Hk[0] * 1j                  # i (b + b^+) is anti-Hermitian
    with pytest.raises(GrapeError) as ei:
        GrapeProblem(q)
    assert ei.value.name == "GRAPE_ENOTHERMITIAN"
    fresh = _hg(p)
    st = fresh._lib.grape_grad(fresh._h, np.zeros((4, 5)).ctypes.data, 0, None)
    assert st == 7   # GRAPE_ESTATE


# ---------------------------------------------------------------- FP32-bulk path (Taylor terms in complex64)

FP32_RTOL = 1e-5


@pytest.mark.parametrize("name,N", [("c1_state_transfer_d30", None), ("c2_gate_d80", None)])
def test_fp32_bulk_parity_full_size(name, N):
    """FP32 increments, FP64 states/overlaps/gradient sums: relative 1e-5 on cost and gradient."""
    p = build_config(name, n_steps=N)
    hg = _hg(p, precision="fp32_bulk")
    cost, grad = hg.cost_and_grad(p.u0)
    _check(p, p.u0, cost, grad, cost_rtol=FP32_RTOL, grad_rtol=FP32_RTOL)


@pytest.mark.parametrize("dim,K,n,N,cluster", [(130, 4, 3, 40, 0), (257, 3, 2, 12, 16), (65, 2, 5, 9, 5)])
def test_fp32_bulk_parity_random(dim, K, n, N, cluster):
    p = random_problem(dim, K, n, N, seed=2000 + dim)
    hg = _hg(p, precision="fp32_bulk", cluster=cluster)
    cost, grad = hg.cost_and_grad(p.u0)
    _check(p, p.u0, cost, grad, cost_rtol=FP32_RTOL, grad_rtol=FP32_RTOL)


def _small_batch(precision):
    from paper_2304_06200_gb300 import GrapeProblem
    from workloads.transmon import _gate_problem, _subspace_one, transmon_cavity
    probs, raw = [], []
    specs = [(3, 10, 1, 4, 37), (4, 20, 8, 3, 61), (4, 60, 2, 2, 45), (3, 10, 5, 4, 90), (4, 20, 3, 4, 23),
             (4, 60, 7, 3, 30)]
    for i, (nt, nc, n, K, N) in enumerate(specs):
        H0, Hk = transmon_cavity(nt, nc)
        dim = nt * nc
        omega = np.array([1.0 if (j // nc) == nt - 1 else 0.0 for j in range(dim)])
        p = _gate_problem(f"b{i}", H0, Hk[:K], dim, _subspace_one(nt, nc, n), 1.0, N, 7000 + i, omega, 1.0, 1.0,
                          1e-2, 1e-12, {})
        p.u0 = p.u0 * 10
        raw.append(p)
        probs.append(GrapeProblem(p, precision=precision, backward_mode=1))
    return raw, probs


def _single_cta_teams(hg):
    inf = hg.info()
    return inf["cluster_forward"] == 1 and inf["cluster"] == 1


def _batch_rtol(precision):
    return (COST_RTOL, GRAD_RTOL) if precision == "fp64" else (FP32_RTOL, FP32_RTOL)


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
@pytest.mark.parametrize("queue_ctas", [0, 2, -1])
def test_batch_matches_individual_evaluations_and_the_oracle(precision, queue_ctas):
    """Every member of the batch (work queue: automatic or 2 CTAs; or lanes only) against its own
    evaluation and against the oracle, over repeated launches of the recorded graph."""
    from paper_2304_06200_gb300 import GrapeBatch
    raw, probs = _small_batch(precision)
    singles = [hg.cost_and_grad(p.u0) for p, hg in zip(raw, probs)]
    batch = GrapeBatch(probs, n_streams=3, queue_ctas=queue_ctas)
    inf = batch.info()
    single = [p for p, hg in zip(raw, probs) if _single_cta_teams(hg)]
    if queue_ctas < 0:
        assert inf["queued"] == 0 and inf["lane_members"] == len(raw)
    else:
        assert len(single) >= 4
        assert inf["queued"] == len(single) and inf["lane_members"] == len(raw) - len(single)
        assert inf["queue_items"] == sum(p.n_states for p in single)
        assert inf["queue_ctas"] == 2 if queue_ctas == 2 else inf["queue_ctas"] >= 1
    crt, grt = _batch_rtol(precision)
    for _ in range(2):                                # the graph is launched repeatedly
        costs, grads = batch.cost_and_grad([p.u0 for p in raw])
        for (c, g), cb, gb in zip(singles, costs, grads):
            if queue_ctas < 0:                        # the members' own launches: the same bits
                assert c == cb and np.array_equal(g, gb)
            else:                                     # one CTA per column at the queue's block size
                assert abs(cb - c) <= 1e-12 * abs(c)
                assert np.linalg.norm(gb - g) <= 1e-11 * np.linalg.norm(g)
    for p, cb, gb in zip(raw, costs, grads):          # every member is right, not just consistent
        _check(p, p.u0, cb, gb, cost_rtol=crt, grad_rtol=grt)
    batch.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_batch_mixes_the_queue_with_cluster_and_three_stage_members(precision):
    """Queued single-CTA members beside lane members: a clustered fused-backward member and a clustered
    three-stage member (block buffers sized by the warm evaluation), every one against the oracle."""
    from paper_2304_06200_gb300 import GrapeBatch, GrapeProblem
    raw, probs = _small_batch(precision)
    big = random_problem(600, 3, 3, 12, seed=6161, band=4, density=0.004)
    big.u0 = big.u0 * 3
    tri = build_config("c2_gate_d80", n_steps=40)
    tri.u0 = tri.u0 * 10
    raw += [big, tri]
    probs += [GrapeProblem(big, precision=precision, cluster=4, backward_mode=1),
              GrapeProblem(tri, precision=precision, cluster=2, backward_mode=3)]
    assert probs[-1].info()["backward_mode"] == 3
    batch = GrapeBatch(probs, n_streams=3, queue_ctas=8)   # the queue forced beside the lanes
    inf = batch.info()
    queued = sum(_single_cta_teams(hg) for hg in probs)
    assert queued >= 4 and not _single_cta_teams(probs[-1]) and not _single_cta_teams(probs[-2])
    assert inf["queued"] == queued and inf["lane_members"] == len(raw) - queued
    costs, grads = batch.cost_and_grad([p.u0 for p in raw])
    crt, grt = _batch_rtol(precision)
    for p, cb, gb in zip(raw, costs, grads):
        _check(p, p.u0, cb, gb, cost_rtol=crt, grad_rtol=grt)
    batch.close()


def test_batch_keeps_three_stage_buffers_and_falls_back_on_the_device():
    """While a batch exists a member's block buffers are not replaced (the recording refers to them):
    controls needing more Taylor terms than the warm evaluation's run the fused backward on the device,
    with the same result; after the batch is gone the buffers grow again."""
    from paper_2304_06200_gb300 import GrapeBatch
    p = _weak_drift_problem()
    hg = _hg(p, backward_mode=3, block_steps=1, cluster=2)
    batch = GrapeBatch([hg], u_warm=[p.u0])
    u_big = p.u0 * 2e4
    costs, grads = batch.cost_and_grad([u_big])
    assert hg.info()["fused_fallback"] == 1
    _check(p, u_big, costs[0], grads[0])
    b0 = hg.info()["device_bytes"]
    cost, grad = hg.cost_and_grad(u_big)             # the member alone: buffers kept, fallback again
    assert hg.info()["fused_fallback"] == 1 and hg.info()["device_bytes"] == b0
    _check(p, u_big, cost, grad)
    batch.close()
    cost, grad = hg.cost_and_grad(u_big)             # no batch left: the buffers grow
    assert hg.info()["fused_fallback"] == 0 and hg.info()["device_bytes"] > b0
    _check(p, u_big, cost, grad)


def test_removed_backward_mode_is_rejected():
    from paper_2304_06200_gb300 import GrapeError
    p = build_config("c1_state_transfer_d30", n_steps=10)
    with pytest.raises(GrapeError):      # the two-team mode 2 no longer exists
        _hg(p, backward_mode=2)


def test_autotune_returns_a_correct_problem():
    from paper_2304_06200_gb300 import autotune
    p = build_config("c2_gate_d80", n_steps=40)
    hg, rep = autotune(p, clusters=[0, 1, 2], m_caps=(0, 20), ckpt_choices=(0, 10, -1), probe_steps=8)
    assert any("ms" in r for r in rep["candidates"])
    assert rep["ckpt_every"] in (0, 10, -1)
    cost, grad = hg.cost_and_grad(p.u0)
    _check(p, p.u0, cost, grad)


# ---------------------------------------------------------------- dense operator on tensor cores (tcgen05)

TC_RTOL = 1e-5


def _dense_problem(n_t, n_c, n, N, seed, drive=10.0):
    from workloads.transmon import _gate_problem, _subspace_one, transmon_cavity
    H0, Hk = transmon_cavity(n_t, n_c)
    dim = n_t * n_c
    omega = np.array([1.0 if (j // n_c) == n_t - 1 else 0.0 for j in range(dim)])
    p = _gate_problem(f"dense{dim}", H0, Hk, dim, _subspace_one(n_t, n_c, n), 0.5, N, seed, omega, 1.0, 1.0, 1e-2,
                      1e-12, {})
    p.u0 = p.u0 * drive
    return p


# BF16 pairs carry 16 significant bits against FP16's 22: a looser bound for the BF16 mode
TC_BF16_RTOL = 1e-3


@pytest.mark.parametrize("precision", ["tc_fp16", "tc_bf16"])
@pytest.mark.parametrize("n_t,n_c,n,N", [(4, 32, 4, 5), (8, 32, 8, 4), (8, 16, 3, 6)])
def test_tensor_core_dense_path_parity(n_t, n_c, n, N, precision):
    """Dense H: every Taylor product on tcgen05 (FP16 or BF16 hi/lo pairs, FP32 accumulation), FP64 states."""
    p = _dense_problem(n_t, n_c, n, N, seed=800 + n_t * n_c)
    hg = _hg(p, precision=precision)
    cost, grad = hg.cost_and_grad(p.u0)
    tol = TC_RTOL if precision == "tc_fp16" else TC_BF16_RTOL
    _check(p, p.u0, cost, grad, cost_rtol=tol, grad_rtol=tol)
    c2, g2 = hg.cost_and_grad(p.u0)        # repeatable (deterministic cluster reduction)
    assert c2 == cost and np.array_equal(g2, grad)


def test_tensor_core_dense_d2048_matches_fp64_path():
    """d = 2048 (transmon 8 x cavity 256): tensor-core dense path against the FP64 sparse kernels."""
    p = _dense_problem(8, 256, 16, 3, seed=4242, drive=5.0)
    c64, g64 = _hg(p, precision="fp64").cost_and_grad(p.u0)
    ctc, gtc = _hg(p, precision="tc_fp16").cost_and_grad(p.u0)
    assert abs(ctc - c64) <= TC_RTOL * abs(c64)
    assert np.linalg.norm(gtc - g64) / np.linalg.norm(g64) <= TC_RTOL


# ---------------------------------------------------------------- time-integrated infidelity C3 (App. A)

@pytest.mark.parametrize("name,N,drive", [("c2_gate_d80", 150, 20.0), ("c1_state_transfer_d30", None, 1.0)])
def test_time_integrated_infidelity_parity(name, N, drive):
    p = build_config(name, n_steps=N)
    p.w_tint = 0.7
    u = p.u0 * drive
    ref = oracle_cost_and_grad(p, u)
    assert ref.parts["C3"] > 0.1
    for mode in (1, 3):
        hg = _hg(p, backward_mode=mode)
        cost, grad = hg.cost_and_grad(u)
        _check(p, u, cost, grad, ref=ref)


def test_time_integrated_infidelity_random_and_reduced_precision():
    p = random_problem(130, 3, 3, 9, seed=3131)
    p.w_tint = 1.3
    ref = oracle_cost_and_grad(p, p.u0)
    cost, grad = _hg(p, cluster=4).cost_and_grad(p.u0)
    _check(p, p.u0, cost, grad, ref=ref)
    cost, grad = _hg(p, precision="fp32_bulk").cost_and_grad(p.u0)
    _check(p, p.u0, cost, grad, cost_rtol=FP32_RTOL, grad_rtol=FP32_RTOL, ref=ref)
    q = _dense_problem(4, 32, 4, 5, seed=77)
    q.w_tint = 0.9
    refq = oracle_cost_and_grad(q, q.u0)
    cost, grad = _hg(q, precision="tc_fp16").cost_and_grad(q.u0)
    _check(q, q.u0, cost, grad, cost_rtol=TC_RTOL, grad_rtol=TC_RTOL, ref=refq)


def _oracle_descent(p, u, eta, n_iter):
    """Steepest descent a <- a - eta grad C (Sec. II) driven by the oracle's exact gradient."""
    costs = []
    for _ in range(n_iter):
        r = oracle_cost_and_grad(p, u)
        costs.append(r.cost)
        u = u - eta * r.grad
    return u, np.array(costs)


@pytest.mark.parametrize("backward_mode", [0, 1])
def test_steepest_descent_graph(backward_mode):
    """grape_optimize: first iterate bitwise equal to one host-driven step, trajectory against the oracle."""
    p = build_config("c1_state_transfer_d30", n_steps=40)
    hg = _hg(p, backward_mode=backward_mode)
    eta = 0.02
    c0, g0 = hg.cost_and_grad(p.u0)
    u1, costs = hg.optimize(p.u0, 1, eta)
    assert costs[0] == c0
    assert np.array_equal(u1, np.subtract(p.u0, np.multiply(eta, g0)))
    u5, costs5 = hg.optimize(p.u0, 5, eta)
    ref_u, ref_c = _oracle_descent(p, np.array(p.u0), eta, 5)
    assert np.allclose(costs5, ref_c, rtol=1e-9, atol=0), (costs5, ref_c)
    assert np.linalg.norm(u5 - ref_u) <= 1e-8 * np.linalg.norm(ref_u)
    # more iterations replay the same recorded graph; the cost decreases for this step size
    _, costs30 = hg.optimize(p.u0, 30, eta)
    assert np.array_equal(costs30[:5], costs5)
    assert np.all(np.diff(costs30) < 0), costs30
    # a changed step size records the iteration again
    u1b, _ = hg.optimize(p.u0, 1, 2 * eta)
    assert np.array_equal(u1b, np.subtract(p.u0, np.multiply(2 * eta, g0)))
    # a normal evaluation after the optimizer sees the controls it is given
    c0b, g0b = hg.cost_and_grad(p.u0)
    assert c0b == c0 and np.array_equal(g0b, g0)


def test_steepest_descent_rejects_bad_arguments():
    from paper_2304_06200_gb300 import GrapeError
    p = build_config("c1_state_transfer_d30", n_steps=10)
    hg = _hg(p)
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(GrapeError):
            hg.optimize(p.u0, 3, bad)
    with pytest.raises(GrapeError):
        hg.optimize(p.u0, 0, 0.01)


@pytest.mark.parametrize("family,size,N,dt,drive", [
    ("h2", 4, 30, 0.5, 3.0), ("h2", 6, 8, 0.5, 3.0),
    ("h3", 6, 30, 0.2, 3.0), ("h3", 9, 6, 0.2, 3.0),
    ("h4", 8, 30, 0.05, 3.0), ("h4", 14, 6, 0.05, 3.0),
])
def test_hamiltonian_families_parity(family, size, N, dt, drive):
    """Three transmons (H_2), qubit chain (H_3) and fluxonium pair (H_4): FP64 and FP32-bulk paths vs the oracle."""
    from workloads import fluxonium_problem, hadamard3_problem, qubit_chain_problem
    build = {"h2": hadamard3_problem, "h3": qubit_chain_problem, "h4": fluxonium_problem}[family]
    p = build(size, N, dt, seed=40 + size)
    p.tau = 1e-12
    u = p.u0 * drive
    r = oracle_cost_and_grad(p, u)
    cost, grad = _hg(p).cost_and_grad(u)
    _check(p, u, cost, grad, ref=r)
    cost, grad = _hg(p, precision="fp32_bulk").cost_and_grad(u)
    _check(p, u, cost, grad, cost_rtol=FP32_RTOL, grad_rtol=FP32_RTOL, ref=r)


# ---------------------------------------------------------------- eigendecomposition propagator (App. F)

EIG_COST_RTOL = 1e-11
EIG_GRAD_RTOL = 1e-9


@pytest.mark.parametrize("dim,K,n,N,density", [
    (1, 1, 1, 4, 0.0), (2, 1, 1, 5, 0.0), (3, 2, 2, 6, 0.0), (33, 3, 5, 7, 0.3), (64, 2, 64, 3, 0.5),
    (65, 4, 3, 9, 0.2), (96, 3, 7, 5, 1.0), (31, 0, 2, 3, 0.0),
])
def test_eig_propagator_random_problems(dim, K, n, N, density):
    """Ragged and dense random problems, a full-rank gate (n = d), one-dimensional and control-free cases."""
    p = random_problem(dim, K, n, N, seed=2000 + dim + K + n + N, density=density)
    hg = _hg(p, propagator="eig")
    assert hg.info()["propagator"] == 1
    r = oracle_cost_and_grad(p, p.u0)
    if K == 0:
        assert abs(hg.cost(p.u0) - r.cost) <= EIG_COST_RTOL * abs(r.cost)
        return
    cost, grad = hg.cost_and_grad(p.u0)
    _check(p, p.u0, cost, grad, cost_rtol=EIG_COST_RTOL, grad_rtol=EIG_GRAD_RTOL, ref=r)


@pytest.mark.parametrize("name,N,tint", [("c1_state_transfer_d30", 200, 0.0), ("c2_gate_d80", 150, 0.0),
                                         ("c2_gate_d80", 60, 0.7), ("c1_state_transfer_d30", 300, 0.4)])
def test_eig_propagator_workloads(name, N, tint):
    p = build_config(name, n_steps=N)
    p.w_tint = tint
    u = p.u0 * 20
    r = oracle_cost_and_grad(p, u)
    cost, grad = _hg(p, propagator="eig").cost_and_grad(u)
    _check(p, u, cost, grad, cost_rtol=EIG_COST_RTOL, grad_rtol=EIG_GRAD_RTOL, ref=r)


def test_eig_propagator_degenerate_spectra():
    """Zero drift and zero controls: every eigenvalue coincides (Phi_ij -> e^{D_i}, App. F limit)."""
    import scipy.sparse as sp
    from workloads import Problem, haar_unitary
    d, N = 12, 4
    H0 = sp.csr_matrix(np.diag(np.repeat([0.0, 1.0, 1.0, 2.5], 3)).astype(np.complex128))
    rng = np.random.default_rng(3)
    Hk = []
    for _ in range(2):
        a = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
        Hk.append(sp.csr_matrix(0.5 * (a + a.conj().T)))
    psi0 = haar_unitary(d, 4)[:, :3]
    p = Problem(name="degenerate", dim=d, dt=0.4, n_steps=N, H0=H0, Hk=Hk, psi0=psi0,
                target=psi0 @ haar_unitary(3, 5), omega=None, w_fid=1.0, w_amp=0.1, u0=np.zeros((2, N)))
    hg = _hg(p, propagator="eig")
    for u in (np.zeros((2, N)), 0.3 * rng.standard_normal((2, N))):
        cost, grad = hg.cost_and_grad(u)
        _check(p, u, cost, grad, cost_rtol=EIG_COST_RTOL, grad_rtol=EIG_GRAD_RTOL)


def test_eig_and_taylor_propagators_agree_on_a_three_transmon_gate():
    from workloads import hadamard3_problem
    p = hadamard3_problem(4, 40, 0.5, seed=7)
    u = p.u0 * 5
    c_t, g_t = _hg(p, tau=1e-12).cost_and_grad(u)
    c_e, g_e = _hg(p, propagator="eig").cost_and_grad(u)
    assert abs(c_t - c_e) <= 1e-10 * abs(c_e)
    assert np.linalg.norm(g_t - g_e) <= 1e-8 * np.linalg.norm(g_e)


@pytest.mark.parametrize("N", [40, 300])
def test_eig_propagator_optimizer_and_errors(N):
    """Steepest descent recorded in a graph (N = 300: the step chunks run on forked streams)."""
    from paper_2304_06200_gb300 import GrapeError
    p = build_config("c1_state_transfer_d30", n_steps=N)
    hg = _hg(p, propagator="eig")
    c0, g0 = hg.cost_and_grad(p.u0)
    u1, costs = hg.optimize(p.u0, 3, 0.02)
    assert costs[0] == c0
    ref_u, ref_c = _oracle_descent(p, np.array(p.u0), 0.02, 3)
    assert np.allclose(costs, ref_c, rtol=1e-11, atol=0)
    assert np.linalg.norm(u1 - ref_u) <= 1e-9 * np.linalg.norm(ref_u)
    bad = np.array(p.u0)
    bad[1, 7] = np.nan
    with pytest.raises(GrapeError):
        hg.cost_and_grad(bad)
    with pytest.raises(GrapeError):
        hg.schedule()
    c1, _ = hg.cost_and_grad(p.u0)     # the problem stays usable after a reported error
    assert c1 == c0


@pytest.mark.parametrize("propagator", ["taylor", "eig"])
def test_closed_form_golden_values(propagator):
    """Both propagators against the 40-digit closed forms of tests/golden/rabi_closed_forms.txt."""
    from test_golden import TERMS, golden_rows, rabi_case
    for delta, u, dt, N, vals in golden_rows():
        for term, col in TERMS.items():
            p, uu = rabi_case(delta, u, dt, N, term)
            cost, grad = _hg(p, propagator=propagator).cost_and_grad(uu)
            assert abs(cost - vals[col]) <= 1e-11, (term, delta, u, cost, vals[col])
            assert abs(np.sum(grad) - vals[col + 1]) <= 1e-10 * max(1.0, abs(vals[col + 1])), (term, delta, u)


def test_c3_full_size_in_the_bench_configuration():
    """d = 4000, N = 2000 with the partitions bench.py times (forward 16 CTAs per column, three-stage
    backward): the same cost as the fused one-team backward with the forward's partition and its
    gradient within rounding, and sampled gradient entries equal to central differences of the GPU's
    own cost (schedule unchanged by the perturbation)."""
    p = build_config("c3_gate_d4000")
    hg = _hg(p)
    inf = hg.info()
    assert inf["backward_mode"] == 3 and inf["cluster_forward"] == 16
    u = np.array(p.u0)
    cost, grad = hg.cost_and_grad(u)
    assert hg.info()["fused_fallback"] == 0
    m0, s0, _ = hg.schedule()
    one_team = _hg(p, cluster=inf["cluster_forward"], backward_mode=1)
    c1, g1 = one_team.cost_and_grad(u)
    assert c1 == cost
    assert np.linalg.norm(g1 - grad) <= 1e-11 * np.linalg.norm(grad)
    one_team.close()
    h = 1e-5
    for k, n in ((0, 3), (3, 1000), (5, 1996)):
        up = u.copy(); up[k, n] += h
        um = u.copy(); um[k, n] -= h
        cp = hg.cost(up)
        assert np.array_equal(hg.schedule()[0], m0) and np.array_equal(hg.schedule()[1], s0)
        cm = hg.cost(um)
        fd = (cp - cm) / (2 * h)
        assert abs(fd - grad[k, n]) <= 1e-6 * np.abs(grad).max(), (k, n, fd, grad[k, n])


def test_allocation_failure_is_reported():
    """An allocator that refuses (the torch caching allocator under a memory-fraction cap) gives
    GRAPE_ENOMEM from create, and nothing is left allocated."""
    import torch
    from paper_2304_06200_gb300 import GrapeError
    p = build_config("c3_gate_d4000", n_steps=200)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    before = torch.cuda.memory_allocated()
    torch.cuda.set_per_process_memory_fraction(1e-5)
    try:
        with pytest.raises(GrapeError) as ei:
            _hg(p)
        assert ei.value.name == "GRAPE_ENOMEM"
    finally:
        torch.cuda.set_per_process_memory_fraction(1.0)
    assert torch.cuda.memory_allocated() == before
    c, _ = _hg(build_config("c1_state_transfer_d30", n_steps=5)).cost_and_grad(build_config(
        "c1_state_transfer_d30", n_steps=5).u0)
    assert np.isfinite(c)


def test_batch_with_eigendecomposition_members():
    """A batch mixing Taylor and eigendecomposition members (the latter forking their step chunks
    onto their own streams inside the recorded graph, the Taylor member in the work queue): the
    eigendecomposition members equal their individual evaluations bit for bit, all match the oracle."""
    from paper_2304_06200_gb300 import GrapeBatch
    raw = [build_config("c1_state_transfer_d30", n_steps=300), build_config("c2_gate_d80", n_steps=70),
           random_problem(48, 2, 3, 20, seed=5151, density=0.5)]
    probs = [_hg(raw[0], propagator="eig"), _hg(raw[1], backward_mode=1), _hg(raw[2], propagator="eig")]
    singles = [hg.cost_and_grad(p.u0) for p, hg in zip(raw, probs)]
    batch = GrapeBatch(probs, n_streams=2)
    for _ in range(2):
        costs, grads = batch.cost_and_grad([p.u0 for p in raw])
        for i, ((c, g), cb, gb) in enumerate(zip(singles, costs, grads)):
            if i == 1:                                # queued Taylor member: the queue's block size
                assert abs(cb - c) <= 1e-12 * abs(c)
                assert np.linalg.norm(gb - g) <= 1e-11 * np.linalg.norm(g)
            else:
                assert c == cb
                assert np.array_equal(g, gb)
    for i, p in enumerate(raw):
        if i == 1:
            _check(p, p.u0, costs[i], grads[i])
        else:
            _check(p, p.u0, costs[i], grads[i], cost_rtol=EIG_COST_RTOL, grad_rtol=EIG_GRAD_RTOL)
    batch.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_maximum_controls_and_full_rank_gate(precision):
    """K = 32 controls (the maximum) on a full-rank gate (n = d = 40), and zero controls (H = H0)."""
    p = random_problem(40, 32, 40, 3, seed=3232, density=0.2)
    hg = _hg(p, precision=precision)
    tol = COST_RTOL if precision == "fp64" else FP32_RTOL
    gtol = GRAD_RTOL if precision == "fp64" else FP32_RTOL
    for u in (p.u0, np.zeros_like(p.u0)):
        cost, grad = hg.cost_and_grad(u)
        _check(p, u, cost, grad, cost_rtol=tol, grad_rtol=gtol)
    from paper_2304_06200_gb300 import GrapeError
    q = random_problem(8, 33, 1, 2, seed=1)
    with pytest.raises(GrapeError):
        _hg(q)


def test_memory_does_not_grow_with_the_number_of_steps():
    """HG keeps no per-step states (Table I: memory independent of N): without checkpoints the device
    memory grows only by the per-step controls, gradient, schedule and overlap arrays."""
    p = build_config("c3_gate_d4000")
    b = {}
    for N in (100, 400):
        hg = _hg(p, n_steps=N, ckpt_every=-1)
        inf = hg.info()
        b[N] = inf["device_bytes"]
        hg.close()
    per_step = (b[400] - b[100]) / 300
    # per step: u and the gradient (K doubles each), per-CTA gradient partials (K doubles per backward
    # CTA), per-CTA overlap partials (one complex per forward CTA), the schedule and the overlaps
    parts_b = 2 * p.n_states * inf["cluster"]
    parts_f = p.n_states * inf["cluster_forward"]
    bound = 8 * p.n_controls * (2 + parts_b) + 16 * parts_f + 64
    assert per_step <= bound, (per_step, bound)
    assert per_step < 0.02 * p.dim * p.n_states * 16          # far below one stored state block


def test_c4_dimension_reduced_n_properties():
    """d = 16000, 16 states (the C4 system) at N = 3: central differences of the GPU's own cost match
    sampled gradient entries, and the FP32-bulk result agrees with FP64 at the stated accuracy."""
    p = build_config("c4_gate_d16000", n_steps=3)
    hg = _hg(p)
    u = np.array(p.u0) * 20
    cost, grad = hg.cost_and_grad(u)
    m0, s0, _ = hg.schedule()
    h = 1e-5
    for k, n in ((0, 0), (4, 2)):
        up = u.copy(); up[k, n] += h
        um = u.copy(); um[k, n] -= h
        cp = hg.cost(up)
        assert np.array_equal(hg.schedule()[0], m0) and np.array_equal(hg.schedule()[1], s0)
        cm = hg.cost(um)
        assert abs((cp - cm) / (2 * h) - grad[k, n]) <= 1e-6 * np.abs(grad).max()
    c32, g32 = _hg(p, precision="fp32_bulk").cost_and_grad(u)
    assert abs(c32 - cost) <= FP32_RTOL * abs(cost)
    assert np.linalg.norm(g32 - grad) <= FP32_RTOL * np.linalg.norm(grad)


def test_autograd_gradcheck():
    """torch.autograd.gradcheck of the Function (analytic Jacobian against finite differences)."""
    import torch
    from paper_2304_06200_gb300 import grape_hg
    p = build_config("c1_state_transfer_d30", n_steps=5)
    hg = _hg(p)
    u = torch.tensor(p.u0 * 5, device="cuda", dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: grape_hg().apply(x, hg), (u,), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_autograd_backward_after_an_interleaved_forward():
    """A second forward on the same problem before the first backward: the backward still returns
    the gradient at its own forward's controls."""
    import torch
    from paper_2304_06200_gb300 import grape_hg
    p = build_config("c2_gate_d80", n_steps=20)
    hg = _hg(p)
    _, g_ref = hg.cost_and_grad(p.u0)
    u1 = torch.tensor(p.u0, device="cuda", requires_grad=True)
    u2 = torch.tensor(p.u0 * 3, device="cuda", requires_grad=True)
    c1 = grape_hg().apply(u1, hg)
    c2 = grape_hg().apply(u2, hg)       # overwrites the problem's sweep state
    c1.backward()
    np.testing.assert_array_equal(u1.grad.cpu().numpy(), g_ref)
    c2.backward()
    _, g2 = hg.cost_and_grad(p.u0 * 3)
    np.testing.assert_array_equal(u2.grad.cpu().numpy(), g2)
