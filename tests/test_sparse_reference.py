"""Pins for oracle.sparse_reference: the exact-exponential cost and gradient computed with sparse
exponential actions must equal the dense-eigh oracle (App. F) on problems small enough for both."""

import numpy as np
import pytest

from oracle import cost_and_grad, cost_only
from oracle import sparse_reference as sr
from workloads import build_config, random_problem, two_level_rabi


@pytest.mark.parametrize("case", ["c2", "random", "random_c3"])
def test_sparse_reference_equals_dense_oracle(case):
    if case == "c2":
        p = build_config("c2_gate_d80", n_steps=12)
        u = p.u0 * 10
    elif case == "random":
        p = random_problem(23, 3, 2, 7, seed=5)
        u = p.u0
    else:
        p = random_problem(31, 2, 3, 6, seed=9)
        p.w_tint = 0.7
        u = p.u0
    a = cost_and_grad(p, u)
    b = sr.cost_and_grad(p, u)
    assert abs(a.cost - b.cost) <= 1e-13 * abs(a.cost)
    assert np.linalg.norm(a.grad - b.grad) <= 1e-12 * np.linalg.norm(a.grad)
    assert sr.cost_only(p, u) == pytest.approx(cost_only(p, u), rel=1e-13)


def test_sparse_reference_gradient_matches_rabi_closed_form():
    """H = u sigma_x from |g> to |e>: C1 = cos^2(u N dt), dC1/du_n = -dt sin(2 u N dt) (exact, commuting steps)."""
    N, dt, u0 = 9, 0.3, 0.41
    p = two_level_rabi(N, dt)
    u = np.full((1, N), u0)
    r = sr.cost_and_grad(p, u)
    assert r.cost == pytest.approx(np.cos(u0 * N * dt) ** 2, rel=1e-13)
    assert np.allclose(r.grad[0], -dt * np.sin(2 * u0 * N * dt), rtol=1e-12, atol=1e-14)


def test_derivative_actions_match_finite_differences_of_the_exponential():
    """L(A, E) psi from the block-triangular identity vs central differences of e^{A + hE} psi."""
    import scipy.linalg as sla
    import scipy.sparse as sp

    rng = np.random.default_rng(3)
    d = 9
    X = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    Y = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    A = sp.csr_matrix(-1j * 0.4 * (X + X.conj().T))
    E = sp.csr_matrix(-1j * 0.4 * (Y + Y.conj().T))
    psi = rng.standard_normal((d, 2)) + 1j * rng.standard_normal((d, 2))
    (L,) = sr.derivative_actions(A, [E], psi)
    h = 1e-6
    fd = (sla.expm((A + h * E).toarray()) @ psi - sla.expm((A - h * E).toarray()) @ psi) / (2 * h)
    assert np.linalg.norm(L - fd) <= 1e-8 * np.linalg.norm(fd)
    Lx = sla.expm_frechet(A.toarray(), E.toarray(), compute_expm=False) @ psi
    assert np.linalg.norm(L - Lx) <= 1e-12 * np.linalg.norm(Lx)
