"""Pins for the CPU oracle: closed forms, library routines, brute force, finite differences, full AD.

Each pin checks the oracle against something other than itself, chosen so that
a plausible mistake (a dropped term, a wrong sign or index, a transposed
operand, a wrong normalisation) fails at least one of them.
"""

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import cost_and_grad, cost_only, propagator, propagator_derivative, forward_states
from oracle.fullad_torch import cost_and_grad_fullad
from workloads import build_config, random_problem, two_level_rabi, transmon_cavity


def _const_u(N, val):
    return np.full((1, N), val)


# ---------------------------------------------------------------- closed forms (two-level Rabi)

@pytest.mark.parametrize("u_val", [0.0, 0.3, -0.7, 1.3])
def test_resonant_rabi_cost_and_gradient(u_val):
    """H = u sigma_x, all H_n commute: C1 = cos^2(uT) for target |e>, dC1/du_n = -dt sin(2uT)."""
    N, dt = 7, 0.37
    p = two_level_rabi(N, dt, target_excited=True)
    u = _const_u(N, u_val)
    r = cost_and_grad(p, u)
    T = N * dt
    assert r.cost == pytest.approx(np.cos(u_val * T) ** 2, abs=1e-14)
    np.testing.assert_allclose(r.grad[0], -dt * np.sin(2 * u_val * T), atol=1e-13)


def test_resonant_rabi_target_ground():
    """Target |g>: C1 = 1 - cos^2(uT) = sin^2(uT), gradient +dt sin(2uT)."""
    N, dt, uv = 5, 0.5, 0.8
    p = two_level_rabi(N, dt, target_excited=False)
    r = cost_and_grad(p, _const_u(N, uv))
    T = N * dt
    assert r.cost == pytest.approx(np.sin(uv * T) ** 2, abs=1e-14)
    np.testing.assert_allclose(r.grad[0], dt * np.sin(2 * uv * T), atol=1e-13)


@pytest.mark.parametrize("delta,om", [(0.4, 0.9), (1.7, 0.3), (-0.8, 2.1)])
def test_detuned_rabi_closed_form(delta, om):
    """H = (delta/2) sigma_z + (Omega/2) sigma_x: P_e = Omega^2/W^2 sin^2(W T / 2), W = sqrt(Omega^2 + delta^2).

    The sum over n of dC/du_n is the derivative with respect to a constant drive u = Omega/2.
    """
    N, dt = 9, 0.41
    p = two_level_rabi(N, dt, delta=delta, target_excited=True)
    u = _const_u(N, om / 2)
    r = cost_and_grad(p, u)
    T = N * dt
    W = np.sqrt(om ** 2 + delta ** 2)
    P = om ** 2 / W ** 2 * np.sin(W * T / 2) ** 2
    assert r.cost == pytest.approx(1 - P, abs=1e-13)
    dP_dOm = (2 * om * delta ** 2 / W ** 4) * np.sin(W * T / 2) ** 2 + (om ** 3 * T / (2 * W ** 3)) * np.sin(W * T)
    assert np.sum(r.grad[0]) == pytest.approx(-2 * dP_dOm, abs=1e-12)


def test_forbidden_penalty_rabi_closed_form():
    """Omega = |e><e|, H = u sigma_x: C2 = 1/N sum_n sin^2(n u dt); dC2/du_n = 1/N sum_{n'>=n} dt sin(2 n' u dt)."""
    N, dt, uv = 8, 0.3, 0.9
    p = two_level_rabi(N, dt)
    p.w_fid, p.w_forbid, p.w_amp = 0.0, 1.0, 0.0
    r = cost_and_grad(p, _const_u(N, uv))
    ns = np.arange(1, N + 1)
    assert r.cost == pytest.approx(np.mean(np.sin(ns * uv * dt) ** 2), abs=1e-14)
    expect = np.array([np.sum(dt * np.sin(2 * ns[n - 1:] * uv * dt)) for n in ns]) / N
    np.testing.assert_allclose(r.grad[0], expect, atol=1e-13)


def test_amplitude_penalty_closed_form():
    rng = np.random.default_rng(0)
    p = random_problem(5, 2, 2, 6, seed=3)
    p.w_fid, p.w_forbid, p.w_amp = 0.0, 0.0, 0.7
    u = rng.standard_normal((2, 6))
    r = cost_and_grad(p, u)
    assert r.cost == pytest.approx(0.7 * np.sum(u ** 2) / 6, rel=1e-14)
    np.testing.assert_allclose(r.grad, 0.7 * 2 * u / 6, rtol=1e-14)


# ---------------------------------------------------------------- library routines

def _rand_herm(d, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    return scale * (a + a.conj().T) / 2


@pytest.mark.parametrize("d,dt", [(2, 0.3), (7, 1.1), (30, 0.5), (80, 0.2)])
def test_propagator_matches_expm_and_is_unitary(d, dt):
    H = _rand_herm(d, d)
    U, lam, V = propagator(H, dt)
    np.testing.assert_allclose(U, sla.expm(-1j * dt * H), atol=1e-12)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(d), atol=1e-13)


@pytest.mark.parametrize("d,dt,seed", [(3, 0.4, 1), (9, 1.3, 2), (24, 0.7, 3)])
def test_propagator_derivative_matches_frechet(d, dt, seed):
    """dU/du equals scipy's Frechet derivative of expm (Pade-based, independent) in direction -i Hc dt."""
    H = _rand_herm(d, seed)
    Hc = _rand_herm(d, seed + 100)
    _, lam, V = propagator(H, dt)
    dU = propagator_derivative(lam, V, Hc, dt)
    _, L = sla.expm_frechet(-1j * dt * H, -1j * dt * Hc)
    np.testing.assert_allclose(dU, L, atol=1e-11)


def test_propagator_derivative_degenerate_spectrum():
    """The transmon-cavity drift is highly degenerate at u = 0; the divided-difference limit must hold there."""
    H0, Hk = transmon_cavity(3, 6)
    H = H0.toarray()
    lam = np.linalg.eigvalsh(H)
    assert np.sum(np.isclose(lam[:, None], lam[None, :])) > 2 * len(lam)  # really degenerate
    for k, hc in enumerate(Hk):
        _, lam, V = propagator(H, 0.8)
        dU = propagator_derivative(lam, V, hc, 0.8)
        _, L = sla.expm_frechet(-1j * 0.8 * H, -1j * 0.8 * hc.toarray())
        np.testing.assert_allclose(dU, L, atol=1e-12)


# ---------------------------------------------------------------- brute force double sum (App. A)

def test_forbidden_gradient_double_sum_bruteforce():
    """dC2/da_n = (1/(N n)) sum_{n'>=n} 2 Re <psi_n'| Omega U_n'..U_{n+1} dU_n |psi_{n-1}> (App. A, first lines
    of Eq. (C2stgrad)), with dU_n from scipy's Frechet derivative; no costate recursion involved."""
    p = random_problem(6, 2, 2, 4, seed=11)
    p.w_fid, p.w_forbid, p.w_amp = 0.0, 1.0, 0.0
    u = p.u0
    K, N = u.shape
    ncol = p.n_states
    psi, steps = forward_states(p, u)
    om = np.diag(p.omega)
    H0, Hk = p.dense()
    G = np.zeros((K, N))
    for n in range(1, N + 1):
        Hn = H0 + sum(u[k, n - 1] * Hk[k] for k in range(K))
        for k in range(K):
            _, dU = sla.expm_frechet(-1j * p.dt * Hn, -1j * p.dt * Hk[k])
            tot = 0.0
            for n2 in range(n, N + 1):
                prod = np.eye(p.dim, dtype=complex)
                for j in range(n + 1, n2 + 1):
                    prod = steps[j - 1][0] @ prod
                v = prod @ (dU @ psi[n - 1])
                tot += 2 * np.real(np.sum(np.conj(psi[n2]) * (om @ v)))
            G[k, n - 1] = tot / (N * ncol)
    r = cost_and_grad(p, u)
    np.testing.assert_allclose(r.grad, G, atol=1e-12)


# ---------------------------------------------------------------- finite differences and full AD

def _fd_grad(p, u, h=1e-6):
    G = np.zeros_like(u)
    for k in range(u.shape[0]):
        for n in range(u.shape[1]):
            up = u.copy(); up[k, n] += h
            um = u.copy(); um[k, n] -= h
            G[k, n] = (cost_only(p, up) - cost_only(p, um)) / (2 * h)
    return G


@pytest.mark.parametrize("seed,gate", [(21, True), (22, False), (23, True)])
def test_gradient_matches_central_differences(seed, gate):
    p = random_problem(7, 3, 2, 5, seed=seed, gate=gate)
    r = cost_and_grad(p, p.u0)
    G = _fd_grad(p, p.u0)
    err = np.linalg.norm(r.grad - G) / np.linalg.norm(G)
    assert err < 1e-8


def test_gradient_matches_fullad_c1_reduced():
    p = build_config("c1_state_transfer_d30", n_steps=20)
    r = cost_and_grad(p, p.u0)
    c_ad, g_ad = cost_and_grad_fullad(p, p.u0)
    assert r.cost == pytest.approx(c_ad, rel=1e-12)
    assert np.linalg.norm(r.grad - g_ad) / np.linalg.norm(g_ad) < 1e-9


def test_gradient_matches_fullad_c2_reduced():
    p = build_config("c2_gate_d80", n_steps=12)
    u = p.u0 * 40.0   # stronger drive so every term of the cost matters
    r = cost_and_grad(p, u)
    c_ad, g_ad = cost_and_grad_fullad(p, u)
    assert r.cost == pytest.approx(c_ad, rel=1e-12)
    assert np.linalg.norm(r.grad - g_ad) / np.linalg.norm(g_ad) < 1e-9
    assert r.parts["C2"] > 1e-6


def test_pins_detect_a_planted_sign_error():
    """Flipping one gradient entry's sign (a plausible costate sign slip) must fail the FD pin."""
    p = random_problem(5, 2, 1, 4, seed=31, gate=False)
    r = cost_and_grad(p, p.u0)
    G = _fd_grad(p, p.u0)
    bad = r.grad.copy()
    bad[1, 2] = -bad[1, 2]
    assert np.linalg.norm(bad - G) / np.linalg.norm(G) > 1e-3


# ---------------------------------------------------------------- invariants

def test_cost_bounds_and_target_equal_realized():
    p = random_problem(6, 2, 3, 4, seed=41)
    p.w_forbid = p.w_amp = 0.0
    r = cost_and_grad(p, p.u0)
    assert 0.0 <= r.parts["C1"] <= 1.0
    # U_T := U_R makes C1 = 0 at its minimum: the gradient vanishes
    p.target = r.psi_N.copy()
    r2 = cost_and_grad(p, p.u0)
    assert abs(r2.cost) < 1e-13
    assert np.max(np.abs(r2.grad)) < 1e-12


def test_global_phase_and_basis_permutation_invariance():
    p = random_problem(7, 2, 2, 4, seed=51)
    r = cost_and_grad(p, p.u0)
    q = random_problem(7, 2, 2, 4, seed=51)
    q.target = q.target * np.exp(0.83j)
    r2 = cost_and_grad(q, q.u0)
    assert r2.cost == pytest.approx(r.cost, rel=1e-13)
    np.testing.assert_allclose(r2.grad, r.grad, atol=1e-13)
    perm = np.random.default_rng(5).permutation(7)
    P = np.eye(7)[perm]
    q2 = random_problem(7, 2, 2, 4, seed=51)
    q2.H0 = P @ q2.H0.toarray() @ P.T
    q2.Hk = [P @ h.toarray() @ P.T for h in q2.Hk]
    q2.psi0 = P @ q2.psi0
    q2.target = P @ q2.target
    q2.omega = q2.omega[perm]
    r3 = cost_and_grad(q2, q2.u0)
    assert r3.cost == pytest.approx(r.cost, rel=1e-12)
    np.testing.assert_allclose(r3.grad, r.grad, atol=1e-12)


def test_norm_conservation_of_oracle_states():
    p = build_config("c2_gate_d80", n_steps=30)
    psi, _ = forward_states(p, p.u0)
    np.testing.assert_allclose(np.linalg.norm(psi[-1], axis=0), 1.0, atol=1e-13)


# ---------------------------------------------------------------- time-integrated infidelity C3 (App. A)

def test_time_integrated_infidelity_rabi_closed_form():
    """H = u sigma_x, target |e>: |<e|psi_n>|^2 = sin^2(n u dt), C3 = 1 - 1/N sum_n sin^2(n u dt),
    dC3/du_n = -1/N sum_{n'>=n} dt sin(2 n' u dt) (all H_n commute)."""
    N, dt, uv = 9, 0.27, 0.6
    p = two_level_rabi(N, dt)
    p.w_fid, p.w_forbid, p.w_amp, p.w_tint = 0.0, 0.0, 0.0, 1.0
    r = cost_and_grad(p, _const_u(N, uv))
    ns = np.arange(1, N + 1)
    assert r.cost == pytest.approx(1 - np.mean(np.sin(ns * uv * dt) ** 2), abs=1e-14)
    expect = -np.array([np.sum(dt * np.sin(2 * ns[n - 1:] * uv * dt)) for n in ns]) / N
    np.testing.assert_allclose(r.grad[0], expect, atol=1e-13)


@pytest.mark.parametrize("gate", [True, False])
def test_time_integrated_infidelity_gradient_fd_and_fullad(gate):
    p = random_problem(6, 2, 2, 5, seed=61, gate=gate)
    p.w_tint = 0.8
    r = cost_and_grad(p, p.u0)
    G = _fd_grad(p, p.u0)
    assert np.linalg.norm(r.grad - G) / np.linalg.norm(G) < 1e-8
    c_ad, g_ad = cost_and_grad_fullad(p, p.u0)
    assert r.cost == pytest.approx(c_ad, rel=1e-12)
    assert np.linalg.norm(r.grad - g_ad) / np.linalg.norm(g_ad) < 1e-9
