"""Structure of the Hamiltonian families (H_2, H_3, H_4) and oracle agreement on them.

The builders hold no GRAPE arithmetic; these checks pin their physics (Hermiticity,
conserved quantities, commutators) and check the oracle's gradient against full
automatic differentiation on each sparsity shape.
"""

import numpy as np
import pytest

from oracle import cost_and_grad
from oracle.fullad_torch import cost_and_grad_fullad
from workloads import (fluxonium_pair, fluxonium_problem, hadamard3_problem, qubit_chain, qubit_chain_problem,
                       three_transmons)
from workloads.families import _fluxonium_ops


def _herm(m):
    d = m.toarray()
    return np.abs(d - d.conj().T).max()


def test_three_transmons_conserve_excitations():
    """Exchange g (b_i b_j^+ + h.c.) and the anharmonic terms conserve the total excitation number."""
    n_t = 4
    H0, Hk = three_transmons(n_t)
    assert len(Hk) == 3 and H0.shape == (64, 64)
    assert _herm(H0) == 0.0 and all(_herm(h) == 0.0 for h in Hk)
    levels = np.array([[i // 16, (i // 4) % 4, i % 4] for i in range(64)]).sum(axis=1)
    Ntot = np.diag(levels.astype(float))
    assert np.abs(H0.toarray() @ Ntot - Ntot @ H0.toarray()).max() < 1e-12
    # each drive changes the excitation number by exactly one
    for h in Hk:
        r, c = h.nonzero()
        assert np.all(np.abs(levels[r] - levels[c]) == 1)


def test_hadamard_target_is_the_tensor_hadamard():
    p = hadamard3_problem(4, 5, 0.5, seed=1)
    U = p.psi0.conj().T @ p.target
    assert np.allclose(U @ U, np.eye(8))          # H (x) H (x) H squares to one
    assert np.allclose(np.abs(U), 1 / np.sqrt(8))


def test_qubit_chain_pauli_structure():
    n_q = 4
    H0, Hk = qubit_chain(n_q)
    assert len(Hk) == 2 * n_q
    d = H0.toarray()
    assert np.count_nonzero(d - np.diag(np.diag(d))) == 0     # sigma_z sigma_z couplings are diagonal
    for k in range(0, 2 * n_q, 2):
        x, y = Hk[k].toarray(), Hk[k + 1].toarray()
        assert np.allclose(x @ x, np.eye(16)) and np.allclose(y @ y, np.eye(16))
        assert np.allclose(x @ y - y @ x, 2 * (x @ y))          # [sx, sy] = 2 i sz = 2 sx sy
    # spectrum of the drift: g * (sum of N_q - 1 products of signs)
    assert np.isclose(np.abs(np.diag(d)).max(), 2 * np.pi * 0.01 * (n_q - 1))


def test_fluxonium_operators_commute_canonically():
    """[phi, n] = i away from the truncation edge; the single-fluxonium drift is Hermitian."""
    H, phi, nop = _fluxonium_ops(20, 1.0, 4.0, 1.0)
    comm = phi @ nop - nop @ phi
    assert np.allclose(comm[:15, :15], 1j * np.eye(15), atol=1e-12)
    assert np.abs(H - H.conj().T).max() < 1e-12
    H0, Hk = fluxonium_pair(6)
    assert H0.shape == (36, 36) and len(Hk) == 2
    assert _herm(H0) == 0.0 and all(_herm(h) == 0.0 for h in Hk)
    # cos(phi) is even in phi, so it only couples oscillator levels of equal parity
    ev = np.arange(6) % 2
    from workloads.families import _fluxonium_ops as ops
    h1 = ops(6, 1.0, 4.0, 1.0)[0]
    assert np.all(np.abs(h1[ev[:, None] != ev[None, :]]) < 1e-12)


def test_fluxonium_psi0_are_drift_eigenstates():
    p = fluxonium_problem(6, 4, 0.05, seed=3)
    H = p.H0.toarray()
    E = p.psi0.conj().T @ H @ p.psi0
    assert np.allclose(E, np.diag(np.diag(E)), atol=1e-9)
    assert np.allclose(p.psi0.conj().T @ p.psi0, np.eye(4), atol=1e-12)


@pytest.mark.parametrize("build", [
    lambda: hadamard3_problem(3, 6, 0.5, seed=11),
    lambda: qubit_chain_problem(4, 6, 0.2, seed=12),
    lambda: fluxonium_problem(5, 6, 0.05, seed=13),
])
def test_oracle_matches_fullad_on_each_family(build):
    p = build()
    u = p.u0 * 5
    r = cost_and_grad(p, u)
    c, g = cost_and_grad_fullad(p, u)
    assert abs(r.cost - c) <= 1e-12 * abs(c)
    assert np.linalg.norm(r.grad - g) <= 1e-10 * np.linalg.norm(g)


def test_dense_register_is_dense_hermitian_with_the_stated_norm():
    """The d = 2048 register's drift: Hermitian, every element non-zero, matrix 1-norm 2 pi x 0.5 rad/ns;
    the controls are sigma_x, sigma_y on qubit 0 (Hermitian, unitary, anticommuting); 16 orthonormal
    states and a target in their span (a unitary on the subspace)."""
    from workloads import dense_register_gate
    p = dense_register_gate(n_steps=2)
    H0 = p.H0.toarray()
    assert p.dim == 2048 and p.H0.nnz == 2048 * 2048
    assert np.allclose(H0, H0.conj().T, atol=0, rtol=0)
    assert np.isclose(np.max(np.sum(np.abs(H0), axis=0)), 2 * np.pi * 0.5, rtol=1e-12)
    X, Y = (h.toarray() for h in p.Hk)
    for h in (X, Y):
        assert np.array_equal(h, h.conj().T) and np.allclose(h @ h, np.eye(p.dim))
    assert np.allclose(X @ Y + Y @ X, 0)
    assert np.allclose(X[0, 1], 1) and np.allclose(Y[1, 0], 1j)   # qubit 0 = the lowest index bit
    assert np.allclose(p.psi0.conj().T @ p.psi0, np.eye(16))
    ov = p.psi0.conj().T @ p.target
    assert np.allclose(ov.conj().T @ ov, np.eye(16))
