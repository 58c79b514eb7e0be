"""Exact-exponential HG GRAPE cost and gradient for large sparse problems, CPU FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).  It computes the same cost
and gradient as ``grape_oracle`` (Sec. II composite cost; gradients of Sec. III.A
and App. A) but never forms a step propagator: every exponential is applied to a
block of vectors by ``scipy.sparse.linalg.expm_multiply``, a library routine that
computes e^{A} V to double precision.  That makes the d = 4000, N = 2000
transmon-cavity workload a matter of minutes instead of days of dense ``eigh``.

* forward:   psi_n = e^{A_n} psi_{n-1},  A_n = -i H_n dt,  H_n = H_s + sum_k u_kn h_k  (Sec. II)
* costates:  the separate vectors of ``grape_oracle`` (phi for C1, Phi for C2, Phi_T for C3),
             each step applying U_n^+ = e^{-A_n} (A_n is anti-Hermitian)
* gradient:  the derivative of U_n psi_{n-1} in the direction E_k = -i h_k dt from the
             block-triangular (auxiliary-matrix) identity of Sec. III.B,
                 exp([[A, E], [0, A]]) [0; psi] = [ L(A, E) psi ; e^{A} psi ],
             with L(A, E) the Frechet derivative of exp at A in direction E; all K
             directions share one exponential of the (K+1)-block upper triangular matrix
             whose diagonal blocks are A and whose last block column holds E_1..E_K.

The step gradients are independent once all psi_n and costates are stored, so they
may be spread over worker processes (``workers`` > 1, spawned).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import expm_multiply

from .grape_oracle import OracleResult


def _step_generator(H0, Hk, u, n, dt):
    """A_n = -i dt (H_s + sum_k u_kn h_k) as a CSR matrix (Sec. II)."""
    H = sp.csr_matrix(H0, dtype=np.complex128)
    for k, h in enumerate(Hk):
        H = H + u[k, n] * sp.csr_matrix(h, dtype=np.complex128)
    return (-1j * dt) * H


def _cost_parts(problem, u, psi_list):
    """Cost from stored states: same definitions as grape_oracle (Eq. (C1st), gate form, (c2st), App. A)."""
    n = problem.psi0.shape[1]
    N = u.shape[1]
    target = np.asarray(problem.target, dtype=np.complex128)
    g = np.sum(np.conj(target) * psi_list[N])
    C1 = 1.0 - abs(g / n) ** 2
    if problem.omega is not None:
        om = np.asarray(problem.omega, dtype=np.float64)
        C2 = sum(float(np.sum(om[:, None] * np.abs(psi_list[k]) ** 2)) for k in range(1, N + 1)) / (N * n)
    else:
        C2 = 0.0
    Camp = float(np.sum(u ** 2)) / N
    gs = np.array([np.sum(np.conj(target) * psi_list[k]) for k in range(1, N + 1)])
    C3 = 1.0 - float(np.sum(np.abs(gs) ** 2)) / (N * n ** 2)
    w_tint = getattr(problem, "w_tint", 0.0)
    cost = problem.w_fid * C1 + problem.w_forbid * C2 + problem.w_amp * Camp + w_tint * C3
    return cost, {"C1": C1, "C2": C2, "C_amp": Camp, "C3": C3, "g": g, "g_steps": gs}


def forward_states(problem, u):
    """psi_0..psi_N by psi_n = e^{A_n} psi_{n-1} (Eq. (statepropagation)), all stored."""
    u = np.asarray(u, dtype=np.float64)
    psi = [np.asarray(problem.psi0, dtype=np.complex128)]
    for n in range(u.shape[1]):
        A = _step_generator(problem.H0, problem.Hk, u, n, problem.dt)
        psi.append(expm_multiply(A, psi[-1]))
    return psi


def cost_only(problem, u) -> float:
    u = np.asarray(u, dtype=np.float64)
    return _cost_parts(problem, u, forward_states(problem, u))[0]


def derivative_actions(A, E_list, psi):
    """[L(A, E_k) psi for k = 1..K] via one exponential of the block upper-triangular matrix (Sec. III.B)."""
    K = len(E_list)
    d, ncol = psi.shape
    blocks = [[None] * (K + 1) for _ in range(K + 1)]
    for k in range(K + 1):
        blocks[k][k] = A
    for k, E in enumerate(E_list):
        blocks[k][K] = E
    M = sp.bmat(blocks, format="csr")
    v = np.zeros(((K + 1) * d, ncol), dtype=np.complex128)
    v[K * d:] = psi
    w = expm_multiply(M, v)
    return [w[k * d:(k + 1) * d] for k in range(K)]


def _step_gradient(args):
    """Gradient entries of one step n (1-based) from psi_{n-1} and the costates at n (Eqs. (gategradient), (C2stgrad))."""
    (H0, Hk, u_col, dt, psi_prev, phi, Phi, PhiT, g, n_cols, N) = args
    K = len(Hk)
    H = sp.csr_matrix(H0, dtype=np.complex128)
    for k, h in enumerate(Hk):
        H = H + u_col[k] * sp.csr_matrix(h, dtype=np.complex128)
    A = (-1j * dt) * H
    E_list = [(-1j * dt) * sp.csr_matrix(h, dtype=np.complex128) for h in Hk]
    dpsi = derivative_actions(A, E_list, psi_prev)
    d1 = np.zeros(K)
    d2 = np.zeros(K)
    d3 = np.zeros(K)
    for k in range(K):
        d1[k] = -(2.0 / n_cols ** 2) * np.real(np.conj(g) * np.sum(np.conj(phi) * dpsi[k]))
        if Phi is not None:
            d2[k] = (2.0 / (N * n_cols)) * np.real(np.sum(np.conj(Phi) * dpsi[k]))
        if PhiT is not None:
            d3[k] = -(2.0 / (N * n_cols ** 2)) * np.real(np.sum(np.conj(PhiT) * dpsi[k]))
    return d1, d2, d3


def cost_and_grad(problem, u, workers: int = 1) -> OracleResult:
    """Composite cost and its gradient (exact exponential, FP64), sparse exponential actions throughout."""
    u = np.asarray(u, dtype=np.float64)
    K, N = u.shape
    n_cols = problem.psi0.shape[1]
    psi = forward_states(problem, u)
    cost, parts = _cost_parts(problem, u, psi)
    g = parts["g"]
    gs = parts["g_steps"]
    target = np.asarray(problem.target, dtype=np.complex128)
    use_c2 = problem.omega is not None and problem.w_forbid != 0.0
    om = np.asarray(problem.omega, dtype=np.float64)[:, None] if problem.omega is not None else None
    w_tint = getattr(problem, "w_tint", 0.0)
    use_c3 = w_tint != 0.0
    # costates at every step n = N..1 (the values paired with step n's derivative)
    phi = target.copy()
    Phi = om * psi[N] if use_c2 else None
    PhiT = target * gs[N - 1] if use_c3 else None
    costates = [None] * (N + 1)
    for step in range(N, 0, -1):
        costates[step] = (phi, Phi, PhiT)
        A = _step_generator(problem.H0, problem.Hk, u, step - 1, problem.dt)
        cols = [phi] + ([Phi] if use_c2 else []) + ([PhiT] if use_c3 else [])
        back = expm_multiply(-A, np.concatenate(cols, axis=1))   # U_n^+ = e^{-A_n}
        phi = back[:, :n_cols]
        j = n_cols
        if use_c2:
            Phi = back[:, j:j + n_cols] + (om * psi[step - 1] if step - 1 >= 1 else 0.0)
            j += n_cols
        if use_c3:
            PhiT = back[:, j:j + n_cols] + (target * gs[step - 2] if step - 1 >= 1 else 0.0)
    jobs = [(problem.H0, problem.Hk, u[:, step - 1], problem.dt, psi[step - 1], costates[step][0], costates[step][1],
             costates[step][2], g, n_cols, N) for step in range(1, N + 1)]
    if workers > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(workers) as pool:
            out = pool.map(_step_gradient, jobs, chunksize=max(1, N // (8 * workers)))
    else:
        out = [_step_gradient(j) for j in jobs]
    dC1 = np.stack([o[0] for o in out], axis=1)
    dC2 = np.stack([o[1] for o in out], axis=1)
    dC3 = np.stack([o[2] for o in out], axis=1)
    grad = problem.w_fid * dC1 + (problem.w_forbid * dC2 if use_c2 else 0.0) + problem.w_amp * 2.0 * u / N
    if use_c3:
        grad = grad + w_tint * dC3
    return OracleResult(cost=cost, grad=grad, parts=parts, psi_N=psi[N])
