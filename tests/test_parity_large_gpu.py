"""GPU parity in the benchmarked configuration against stored exact-exponential references.

The reference values under tests/golden/ were written by tests/golden/make_large_reference.py from
oracle/ alone: the dense-eigh oracle (App. F) for the first 3 steps of the d = 4000 workload, and the
sparse exact-action reference (expm_multiply, auxiliary block-matrix derivative, Sec. III.B) for its
full N = 2000 and for the d = 16,000 workload's first 3 steps.  The GPU runs the truncated Taylor
approximant at the workload's tau = 1e-10 (the bench setting), so these tests bound its deviation
from the exact exponential where it is timed.
"""

import os

import numpy as np
import pytest

from workloads import build_config

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
COST_RTOL = 1e-10
GRAD_RTOL = 1e-8
FP32_RTOL = 1e-5


def _golden(name):
    rows = [ln for ln in open(os.path.join(GOLDEN, name)) if not ln.startswith("#")]
    head = [float(v) for v in rows[0].split()]
    grad = np.array([[float(v) for v in r.split()] for r in rows[1:]])
    return head[0], grad


def _hg(p, **kw):
    from paper_2304_06200_gb300 import GrapeProblem
    return GrapeProblem(p, **kw)


def _errors(cost, grad, ref_cost, ref_grad):
    return abs(cost - ref_cost) / abs(ref_cost), float(np.linalg.norm(grad - ref_grad) / np.linalg.norm(ref_grad))


@pytest.mark.parametrize("mode", [0, 1])
def test_c3_bench_tau_reduced_n_against_the_dense_oracle(mode):
    """d = 4000, 6 controls, 4 states, tau = 1e-10, first 3 steps, both backward kinds."""
    p = build_config("c3_gate_d4000", n_steps=3)
    assert p.tau == 1e-10
    ref_cost, ref_grad = _golden("c3_gate_d4000_n3_dense.txt")
    hg = _hg(p, backward_mode=mode)
    cost, grad = hg.cost_and_grad(p.u0)
    ce, ge = _errors(cost, grad, ref_cost, ref_grad)
    assert ce <= COST_RTOL and ge <= GRAD_RTOL, (ce, ge)


def test_c3_bench_configuration_full_size_against_the_exact_reference():
    """The timed problem itself (d = 4000, N = 2000, tau = 1e-10, automatic partitions)."""
    p = build_config("c3_gate_d4000")
    ref_cost, ref_grad = _golden("c3_gate_d4000_full_exact.txt")
    hg = _hg(p)
    cost, grad = hg.cost_and_grad(p.u0)
    ce, ge = _errors(cost, grad, ref_cost, ref_grad)
    print(f"c3 full size vs exact exponential: cost {ce:.2e}, gradient {ge:.2e}, backward mode "
          f"{hg.info()['backward_mode']}")
    assert ce <= COST_RTOL and ge <= GRAD_RTOL, (ce, ge)


@pytest.mark.parametrize("name,golden", [("c3_gate_d4000", "c3_gate_d4000_n3_dense.txt"),
                                         ("c4_gate_d16000", "c4_gate_d16000_n3_exact.txt")])
def test_fp32_bulk_reduced_n_against_the_oracle(name, golden):
    p = build_config(name, n_steps=3)
    ref_cost, ref_grad = _golden(golden)
    hg = _hg(p, precision="fp32_bulk")
    cost, grad = hg.cost_and_grad(p.u0)
    ce, ge = _errors(cost, grad, ref_cost, ref_grad)
    assert ce <= FP32_RTOL and ge <= FP32_RTOL, (ce, ge)


def test_fp64_c4_reduced_n_against_the_exact_reference():
    p = build_config("c4_gate_d16000", n_steps=3)
    ref_cost, ref_grad = _golden("c4_gate_d16000_n3_exact.txt")
    hg = _hg(p)
    cost, grad = hg.cost_and_grad(p.u0)
    ce, ge = _errors(cost, grad, ref_cost, ref_grad)
    assert ce <= COST_RTOL and ge <= GRAD_RTOL, (ce, ge)


def test_fp32_bulk_full_size_against_the_exact_reference():
    """The compensated FP32 bulk at d = 4000, N = 2000 (three-stage backward: its costate chain is
    fast, so consecutive gradient blocks run side by side on the two gradient streams)."""
    p = build_config("c3_gate_d4000")
    ref_cost, ref_grad = _golden("c3_gate_d4000_full_exact.txt")
    hg = _hg(p, precision="fp32_bulk")
    assert hg.info()["backward_mode"] == 3
    cost, grad = hg.cost_and_grad(p.u0)
    ce, ge = _errors(cost, grad, ref_cost, ref_grad)
    print(f"c3 full size, compensated FP32 bulk vs exact exponential: cost {ce:.2e}, gradient {ge:.2e}")
    assert ce <= FP32_RTOL and ge <= FP32_RTOL, (ce, ge)


def test_repeated_device_pointer_evaluations_at_full_size():
    """Evaluations through device pointers, back to back on one stream (as the benchmark runs them),
    the first one growing the Horner block buffers: every one equals the exact reference."""
    import torch
    p = build_config("c3_gate_d4000")
    ref_cost, ref_grad = _golden("c3_gate_d4000_full_exact.txt")
    hg = _hg(p)
    dev = torch.device("cuda", 0)
    u = torch.tensor(p.u0, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    for _ in range(3):
        cost = torch.zeros((), dtype=torch.float64, device=dev)
        grad = torch.zeros((p.n_controls, p.n_steps), dtype=torch.float64, device=dev)
        hg.cost_device(u, cost, st)
        hg.grad_device(grad, st)
        torch.cuda.synchronize()
        ce, ge = _errors(float(cost.item()), grad.cpu().numpy(), ref_cost, ref_grad)
        assert ce <= COST_RTOL and ge <= GRAD_RTOL, (ce, ge)


# FP16 hi/lo pairs carry 22 significant bits, BF16 pairs 16: the tensor-core modes' bounds
TC_FP16_RTOL = 1e-5
TC_BF16_RTOL = 1e-3


@pytest.mark.parametrize("precision,tol", [("tc_fp16", TC_FP16_RTOL), ("tc_bf16", TC_BF16_RTOL)])
def test_tensor_core_dense_drift_d2048_against_the_dense_oracle(precision, tol):
    """A drift with every matrix element non-zero (GUE, 11 qubits, d = 2048, 16 states), first 2 steps
    against the dense-eigh oracle: the workload the tensor-core products exist for (Sec. V, dense H)."""
    from workloads import dense_register_gate
    p = dense_register_gate(n_steps=2)
    ref_cost, ref_grad = _golden("dense_gue_q11_n2_dense.txt")
    hg = _hg(p, precision=precision)
    cost, grad = hg.cost_and_grad(p.u0)
    ce, ge = _errors(cost, grad, ref_cost, ref_grad)
    print(f"dense GUE d = 2048, {precision}: cost {ce:.2e}, gradient {ge:.2e}")
    assert ce <= tol and ge <= tol, (ce, ge)


def test_dense_drift_is_refused_by_the_sparse_kernels():
    """The sparse sweeps keep a team's pattern in shared memory: a dense d = 2048 drift does not fit
    and is refused at creation (no launch), which is why the tensor-core path carries dense H."""
    from paper_2304_06200_gb300 import GrapeError
    from workloads import dense_register_gate
    p = dense_register_gate(n_steps=2)
    with pytest.raises(GrapeError):
        _hg(p, precision="fp64")
