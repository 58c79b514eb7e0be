"""Exact-exponential HG GRAPE cost and gradient, plain CPU FP64 (numpy + LAPACK).

TEST INFRASTRUCTURE ONLY (see the package docstring).  This is the oracle the
CUDA path is compared with.  It is deliberately slow and obvious:

* every step propagator is formed densely from a Hermitian eigendecomposition
  (App. F, eqs. (matrix dia)-(propagator der));
* all forward states psi_0..psi_N are stored (no checkpointing);
* the costates are the paper's separate vectors phi_n^h (C1, Sec. III.A) and
  Phi_n^h (C2, App. A), each obtained by its own backward recursion;
* the propagator derivative uses the divided-difference (Daleckii-Krein)
  form of App. F with the degenerate-eigenvalue limit written out correctly.

Cost (Sec. II composite cost, with the readings listed in the design notes):

    C   = w_fid * C1 + w_forbid * C2 + w_amp * C_amp + w_tint * C3
    C1  = 1 - |g / n|^2,      g = sum_h <phi_T^h | psi_N^h>          (Eq. (C1st); gate form Sec. III.A)
    C2  = 1/(N n) sum_{n'=1..N} sum_h <psi_n'^h | Omega | psi_n'^h>   (App. A, Eq. (c2st))
    C_amp = 1/N sum_{k,n} u_kn^2                                      (Sec. II "maximal power" penalty)
    C3  = 1 - 1/(N n^2) sum_{n'=1..N} |g_n'|^2,  g_n' = sum_h <phi_T^h|psi_n'^h>   (App. A, C3st / C3g)

Gradient (Eqs. (stgradient), (gategradient), (C2stgrad)):

    dC1/du_kn = -(2/n^2) Re[ conj(g) sum_h <phi_n^h | dU_n/du_kn | psi_{n-1}^h> ]
    dC2/du_kn =  (2/(N n)) Re[ sum_h <Phi_n^h | dU_n/du_kn | psi_{n-1}^h> ]
    dC_amp/du_kn = 2 u_kn / N

    dC3/du_kn = -(2/(N n^2)) Re[ sum_h <Phi_T,n^h | dU_n/du_kn | psi_{n-1}^h> ]     (App. A, Eq. (state time gradient))

with phi_n = U_{n+1}^+ phi_{n+1}, phi_N = phi_T; Phi_n = U_{n+1}^+ Phi_{n+1} + Omega psi_n,
Phi_N = Omega psi_N; Phi_T,n = U_{n+1}^+ Phi_T,n+1 + phi_T g_n, Phi_T,N = phi_T g_N (App. A).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _dense(m) -> np.ndarray:
    if hasattr(m, "toarray"):
        return np.asarray(m.toarray(), dtype=np.complex128)
    return np.asarray(m, dtype=np.complex128)


def step_hamiltonians(H0, Hk, u):
    """H_n = H_s + sum_k u_kn h_k for n = 1..N (Sec. II; one row of u per control channel)."""
    H0d = _dense(H0)
    Hkd = [_dense(h) for h in Hk]
    u = np.asarray(u, dtype=np.float64)
    for n in range(u.shape[1]):
        H = H0d.copy()
        for k, h in enumerate(Hkd):
            H = H + u[k, n] * h
        yield H


def propagator(H: np.ndarray, dt: float):
    """U = exp(-i H dt) via H = V diag(lam) V^+ (App. F: A = S D S^+, e^A = S e^D S^+ with A = -i H dt).

    Returns (U, lam, V).
    """
    lam, V = np.linalg.eigh(H)
    U = (V * np.exp(-1j * lam * dt)[None, :]) @ V.conj().T
    return U, lam, V


def propagator_derivative(lam: np.ndarray, V: np.ndarray, Hc: np.ndarray, dt: float) -> np.ndarray:
    """dU/du for U = exp(-i (H + u Hc) dt) at u = 0, given H = V diag(lam) V^+ (App. F, Eq. (propagator der)).

    dU/du = V ( Phi o (V^+ dA/du V) ) V^+ with dA/du = -i Hc dt and Phi_ij the divided
    difference of exp at D_ii = -i lam_i dt and D_jj = -i lam_j dt:

        Phi_ij = (e^{D_ii} - e^{D_jj}) / (D_ii - D_jj)      (i != j, D_ii != D_jj)
        Phi_ij = e^{D_ii}                                   (D_ii == D_jj, including i == j)

    The paper's F matrix sets the degenerate off-diagonal entries to zero, which
    drops their contribution; the limit above is the correct value.  It is
    evaluated without cancellation as exp((D_ii + D_jj)/2) * sin(theta)/theta with
    theta = (lam_i - lam_j) dt / 2.
    """
    D = -1j * lam * dt
    theta = 0.5 * (lam[:, None] - lam[None, :]) * dt
    Phi = np.exp(0.5 * (D[:, None] + D[None, :])) * np.sinc(theta / np.pi)
    E = V.conj().T @ _dense(Hc) @ V
    return V @ ((-1j * dt * E) * Phi) @ V.conj().T


def forward_states(problem, u):
    """psi_n = U_n psi_{n-1}, n = 1..N (Eq. (statepropagation)); returns (list of psi_n, list of (U, lam, V))."""
    psi = [np.asarray(problem.psi0, dtype=np.complex128)]
    steps = []
    for H in step_hamiltonians(problem.H0, problem.Hk, u):
        U, lam, V = propagator(H, problem.dt)
        psi.append(U @ psi[-1])
        steps.append((U, lam, V))
    return psi, steps


@dataclass
class OracleResult:
    cost: float
    grad: np.ndarray | None
    parts: dict = field(default_factory=dict)
    psi_N: np.ndarray | None = None


def _cost_parts(problem, u, psi):
    n = problem.psi0.shape[1]
    N = u.shape[1]
    target = np.asarray(problem.target, dtype=np.complex128)
    g = np.sum(np.conj(target) * psi[N])
    C1 = 1.0 - abs(g / n) ** 2
    if problem.omega is not None:
        om = np.asarray(problem.omega, dtype=np.float64)
        C2 = sum(float(np.sum(om[:, None] * np.abs(psi[k]) ** 2)) for k in range(1, N + 1)) / (N * n)
    else:
        C2 = 0.0
    Camp = float(np.sum(np.asarray(u) ** 2)) / N
    gs = np.array([np.sum(np.conj(target) * psi[k]) for k in range(1, N + 1)])
    C3 = 1.0 - float(np.sum(np.abs(gs) ** 2)) / (N * n ** 2)
    w_tint = getattr(problem, "w_tint", 0.0)
    cost = problem.w_fid * C1 + problem.w_forbid * C2 + problem.w_amp * Camp + w_tint * C3
    return cost, {"C1": C1, "C2": C2, "C_amp": Camp, "C3": C3, "g": g, "g_steps": gs}


def cost_only(problem, u) -> float:
    """Composite cost only (forward sweep), used for finite differences."""
    u = np.asarray(u, dtype=np.float64)
    psi, _ = forward_states(problem, u)
    return _cost_parts(problem, u, psi)[0]


def cost_and_grad(problem, u) -> OracleResult:
    """Composite cost and its gradient with respect to every u_kn (exact exponential, FP64)."""
    u = np.asarray(u, dtype=np.float64)
    K, N = u.shape
    n = problem.psi0.shape[1]
    psi, steps = forward_states(problem, u)
    cost, parts = _cost_parts(problem, u, psi)
    g = parts["g"]
    Hkd = [_dense(h) for h in problem.Hk]
    target = np.asarray(problem.target, dtype=np.complex128)
    use_c2 = problem.omega is not None and problem.w_forbid != 0.0
    om = np.asarray(problem.omega, dtype=np.float64)[:, None] if problem.omega is not None else None

    w_tint = getattr(problem, "w_tint", 0.0)
    use_c3 = w_tint != 0.0
    gs = parts["g_steps"]
    dC1 = np.zeros((K, N))
    dC2 = np.zeros((K, N))
    dC3 = np.zeros((K, N))
    phi = target.copy()                       # phi_N^h = U_T psi_0^h  (gate) / phi_T (state)
    Phi = om * psi[N] if use_c2 else None     # Phi_N^h = Omega psi_N^h (App. A)
    PhiT = target * gs[N - 1] if use_c3 else None   # Phi_T,N^h = phi_T^h g_N (App. A)
    for step in range(N, 0, -1):              # descending n, as in Fig. 1(b)
        U, lam, V = steps[step - 1]
        for k in range(K):
            dU = propagator_derivative(lam, V, Hkd[k], problem.dt)
            dpsi = dU @ psi[step - 1]
            dC1[k, step - 1] = -(2.0 / n ** 2) * np.real(np.conj(g) * np.sum(np.conj(phi) * dpsi))
            if use_c2:
                dC2[k, step - 1] = (2.0 / (N * n)) * np.real(np.sum(np.conj(Phi) * dpsi))
            if use_c3:
                dC3[k, step - 1] = -(2.0 / (N * n ** 2)) * np.real(np.sum(np.conj(PhiT) * dpsi))
        phi = U.conj().T @ phi                            # phi_{n-1} = U_n^+ phi_n
        if use_c2 and step - 1 >= 1:
            Phi = U.conj().T @ Phi + om * psi[step - 1]    # Phi_{n-1} = U_n^+ Phi_n + Omega psi_{n-1}
        if use_c3 and step - 1 >= 1:
            PhiT = U.conj().T @ PhiT + target * gs[step - 2]   # Phi_T,n-1 = U_n^+ Phi_T,n + phi_T g_{n-1}
    grad = problem.w_fid * dC1 + (problem.w_forbid * dC2 if use_c2 else 0.0) + problem.w_amp * 2.0 * u / N
    if use_c3:
        grad = grad + w_tint * dC3
    return OracleResult(cost=cost, grad=grad, parts=parts, psi_N=psi[N])
