"""The allocation-free entry point grape_taylor_step_noalloc, called through the C ABI.

It serves callers that cannot allocate device memory (graph capture, allocation-free real-time
loops, fixed device pools).  Its output is checked on two calls in a row (the built-in scratch
array keeps the first call's contents) against
  - the oracle's truncated-Taylor action at the same (m, s), element by element, and
  - the regular entry point: for a one-step problem, the cost computed from the propagated block
    must equal grape_cost's cost for the same (m, s).
This file is collected last so that a run stopping at the first failure has run every other test.
"""

import ctypes as C

import numpy as np
import pytest

from workloads import build_config, random_problem

pytestmark = pytest.mark.gpu

COST_RTOL = 1e-10
# Same (m, s) and the same term recursion on both sides: only the order of rounding differs, a few
# units of 2^-53 per product over s * m products.
STATE_RTOL = 1e-12


def _cost_from_block(p, u, psi):
    n = psi.shape[1]
    g = np.sum(np.conj(p.target) * psi)
    c = p.w_fid * (1.0 - abs(g / n) ** 2)
    if p.omega is not None:
        c += p.w_forbid * float(np.sum(p.omega[:, None] * np.abs(psi) ** 2)) / n
    return c + p.w_amp * float(np.sum(u ** 2))


@pytest.mark.parametrize("case", ["c2", "random"])
def test_noalloc_step_matches_regular_entry_point_twice(case):
    import torch
    from oracle import taylor_action
    from paper_2304_06200_gb300 import GrapeProblem
    from paper_2304_06200_gb300._abi import lib

    if case == "c2":
        p = build_config("c2_gate_d80", n_steps=1)
        u = p.u0 * 30.0
    else:
        p = random_problem(37, 2, 3, 1, seed=4242)
        u = p.u0
    hg = GrapeProblem(p)
    cost_ref = hg.cost(u)
    m, s, _ = hg.schedule()
    H = (p.H0 + sum(u[k, 0] * p.Hk[k] for k in range(len(p.Hk)))).tocsr()
    H.sort_indices()
    dev = torch.device("cuda", 0)
    rowptr = torch.tensor(H.indptr, dtype=torch.int64, device=dev)
    colind = torch.tensor(H.indices, dtype=torch.int32, device=dev)
    vals = torch.tensor(np.ascontiguousarray(H.data, dtype=np.complex128).view(np.float64), device=dev)
    psi_in = torch.tensor(np.ascontiguousarray(p.psi0.T).view(np.float64), device=dev)   # column-major block
    psi_out = torch.empty_like(psi_in)
    expect = taylor_action(-1j * p.dt * H.toarray(), p.psi0, int(m[0]), int(s[0]))
    L = lib()
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call in range(2):
        psi_out.fill_(float("nan"))
        st = L.grape_taylor_step_noalloc(p.dim, H.nnz, p.n_states, rowptr.data_ptr(), colind.data_ptr(), vals.data_ptr(),
                                         float(p.dt), int(m[0]), int(s[0]), psi_in.data_ptr(), psi_out.data_ptr(),
                                         C.c_void_p(stream))
        assert st == 0, L.grape_last_error()
        torch.cuda.synchronize()
        psi = psi_out.cpu().numpy().view(np.complex128).reshape(p.n_states, p.dim).T
        scale = np.linalg.norm(expect, axis=0)
        assert np.all(np.abs(psi - expect) <= STATE_RTOL * scale[None, :]), (call, np.max(np.abs(psi - expect)))
        cost = _cost_from_block(p, u, psi)
        assert abs(cost - cost_ref) <= COST_RTOL * abs(cost_ref), (call, cost, cost_ref)
    hg.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    from paper_2304_06200_gb300._abi import lib

    L = lib()
    dev = torch.device("cuda", 0)
    dummy = torch.zeros(8, dtype=torch.float64, device=dev)
    ptr = dummy.data_ptr()
    # 3 * dim * n_states complex numbers must fit in 16 MiB: 349525 is the largest product allowed
    st = L.grape_taylor_step_noalloc(349526, 1, 1, ptr, ptr, ptr, 0.1, 4, 1, ptr, ptr, None)
    assert st == 1
    assert b"16 MiB" in L.grape_last_error()
    # s beyond the cap of 4096 substeps, and a negative nnz, are refused before any launch
    assert L.grape_taylor_step_noalloc(8, 1, 1, ptr, ptr, ptr, 0.1, 4, 4097, ptr, ptr, None) == 1
    assert b"4096" in L.grape_last_error()
    assert L.grape_taylor_step_noalloc(8, -1, 1, ptr, ptr, ptr, 0.1, 4, 1, ptr, ptr, None) == 1
