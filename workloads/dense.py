"""A genuinely dense Hamiltonian: an 11-qubit register with a random-matrix drift.

Input builder only (no propagation, cost or gradient).  The paper's dense-storage case
(Sec. V decision tree; the Fig. 3 gate benchmark stores H dense) is exercised here by a
drift whose every matrix element is non-zero, so that the dense tensor-core products do
no wasted work:

* H_s: a GUE-distributed Hermitian matrix (complex Gaussian G, H_s = (G + G^+) / 2),
  rescaled so that its matrix 1-norm is ``norm1_ghz`` x 2 pi rad/ns;
* two controls: the x and y Pauli drives of qubit 0 (the lowest bit of the basis index),
  H_1 = 1 (x) sigma_x, H_2 = 1 (x) sigma_y, 2048 non-zeros each;
* ``n_states`` initial states: the first basis vectors; the target applies a seeded
  Haar unitary inside their span (gate form of C1);
* the forbidden projector Omega: basis states whose highest qubit is set (C2).

Units as in ``transmon``: rad/ns and ns.  The 1-norm fixes ||A_n||_1 = dt ||H_n||_1 and
with it the (m, s) choice of App. C, independently of the dimension.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .transmon import TWO_PI, Problem, haar_unitary, smooth_controls


def gue_drift(dim: int, seed: int, norm1: float) -> np.ndarray:
    """Dense Hermitian d x d drift with i.i.d. complex Gaussian entries, scaled to matrix 1-norm ``norm1``."""
    rng = np.random.default_rng(seed)
    g = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / np.sqrt(2.0)
    h = 0.5 * (g + g.conj().T)
    return h * (norm1 / np.max(np.sum(np.abs(h), axis=0)))


def qubit0_drives(dim: int):
    """(sigma_x, sigma_y) on qubit 0 (basis index bit 0) of a register of log2(dim) qubits, CSR."""
    sx = sp.csr_matrix(np.array([[0, 1], [1, 0]], dtype=np.complex128))
    sy = sp.csr_matrix(np.array([[0, -1j], [1j, 0]], dtype=np.complex128))
    eye = sp.identity(dim // 2, format="csr", dtype=np.complex128)
    return sp.kron(eye, sx, format="csr"), sp.kron(eye, sy, format="csr")


def dense_register_gate(n_qubits: int = 11, n_states: int = 16, n_steps: int = 20, seed: int = 2048,
                        dt: float = 1.0, norm1_ghz: float = 0.5, tau: float = 1e-10) -> Problem:
    """d = 2^n_qubits gate problem whose drift is dense (every H_ij != 0); N steps of dt ns."""
    dim = 1 << n_qubits
    H0 = sp.csr_matrix(gue_drift(dim, seed, TWO_PI * norm1_ghz))
    Hk = list(qubit0_drives(dim))
    psi0 = np.zeros((dim, n_states), dtype=np.complex128)
    psi0[np.arange(n_states), np.arange(n_states)] = 1.0
    target = psi0 @ haar_unitary(n_states, seed + 1)
    omega = ((np.arange(dim) >> (n_qubits - 1)) & 1).astype(np.float64)
    u0 = smooth_controls(len(Hk), n_steps, dt, seed + 2, rms_ghz=0.05)
    return Problem(name=f"dense_gue_q{n_qubits}", dim=dim, dt=dt, n_steps=n_steps, H0=H0, Hk=Hk, psi0=psi0,
                   target=target, omega=omega, w_fid=1.0, w_forbid=1.0, w_amp=1e-2, u0=u0, tau=tau,
                   meta={"seed": seed, "stored": "dense", "drift": "GUE, every element non-zero"})
