"""Second CPU reference: full automatic differentiation in complex128 torch (CPU).

TEST INFRASTRUCTURE ONLY.  This is the "full-AD" strategy the paper compares
HG with (Sec. IV.A, "Full automatic differentiation"): the forward pass builds
the whole computational graph (one dense ``torch.linalg.matrix_exp`` per step)
and reverse mode returns the gradient.  It shares nothing with ``grape_oracle``
(no eigendecomposition, no hand-written costates) and so pins it.
"""

from __future__ import annotations

import numpy as np


def cost_and_grad_fullad(problem, u):
    """(cost, grad) of the composite cost of ``grape_oracle`` via torch autograd through matrix_exp."""
    import torch

    def dense(m):
        return torch.tensor(m.toarray() if hasattr(m, "toarray") else np.asarray(m), dtype=torch.complex128)

    u_t = torch.tensor(np.asarray(u, dtype=np.float64), dtype=torch.float64, requires_grad=True)
    K, N = u_t.shape
    H0 = dense(problem.H0)
    Hk = torch.stack([dense(h) for h in problem.Hk])
    psi = torch.tensor(np.asarray(problem.psi0), dtype=torch.complex128)
    target = torch.tensor(np.asarray(problem.target), dtype=torch.complex128)
    n = psi.shape[1]
    om = None
    if problem.omega is not None:
        om = torch.tensor(np.asarray(problem.omega), dtype=torch.float64)[:, None]
    c2 = torch.zeros((), dtype=torch.float64)
    c3 = torch.zeros((), dtype=torch.float64)
    for step in range(N):
        H = H0 + torch.einsum("k,kij->ij", u_t[:, step].to(torch.complex128), Hk)
        U = torch.linalg.matrix_exp(-1j * problem.dt * H)
        psi = U @ psi
        if om is not None:
            c2 = c2 + torch.sum(om * (psi.real ** 2 + psi.imag ** 2))
        gk = torch.sum(torch.conj(target) * psi)
        c3 = c3 + gk.real ** 2 + gk.imag ** 2
    g = torch.sum(torch.conj(target) * psi)
    C1 = 1.0 - (g.real ** 2 + g.imag ** 2) / n ** 2
    C2 = c2 / (N * n)
    Camp = torch.sum(u_t ** 2) / N
    C3 = 1.0 - c3 / (N * n ** 2)
    cost = problem.w_fid * C1 + problem.w_forbid * C2 + problem.w_amp * Camp + getattr(problem, "w_tint", 0.0) * C3
    cost.backward()
    return float(cost.detach()), u_t.grad.detach().numpy().copy()
