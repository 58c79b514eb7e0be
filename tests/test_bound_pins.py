"""Pins for the oracle's error bound E_A(m, s) and (m, s) rule (Sec. III.B, App. C)."""

import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import error_bound, gamma, select_ms, tail_remainder, taylor_action
from oracle.taylor_bound import U64, one_norm, rounding_bound, truncation_bound


@pytest.mark.parametrize("b,m", [(0.5, 3), (1.0, 10), (2.92, 25), (6.0, 32), (1.4, 19), (10.0, 60), (0.01, 1)])
def test_tail_remainder_matches_high_precision(b, m):
    """R_m(b) = e^b - sum_{q<=m} b^q/q!, evaluated in 80-digit decimal arithmetic (no cancellation there)."""
    getcontext().prec = 80
    B = Decimal(repr(b))
    partial = Decimal(0)
    term = Decimal(1)
    for q in range(m + 1):
        if q > 0:
            term = term * B / q
        partial += term
    exact = float(B.exp() - partial)
    assert tail_remainder(b, m) == pytest.approx(exact, rel=1e-13)


@pytest.mark.parametrize("n", [1, 3, 47, 500])
def test_gamma_exact_rational(n):
    u = Fraction(1, 2 ** 53)
    # u' = 2 sqrt(2) u / (1 - 2u); sqrt(2) is irrational, so compare at float precision
    up = 2 * math.sqrt(2.0) * float(u) / float(1 - 2 * u)
    assert gamma(n) == pytest.approx(n * up / (1 - n * up), rel=1e-15)
    assert gamma(n) > n * 2 * math.sqrt(2) * 2.0 ** -53  # strictly above n u'


@pytest.mark.parametrize("x,m", [(0.3, 4), (1.5, 12), (4.0, 20)])
def test_truncation_bound_special_cases(x, m):
    """s = 1: the bound is R itself; s = 2: 2R(1 - 4R^2)/(1 - 2R) = 2R + 4R^2 >= the binomial sum 2R + R^2."""
    R1 = tail_remainder(x, m)
    assert truncation_bound(x, m, 1) == pytest.approx(R1, rel=1e-15)
    R2 = tail_remainder(x / 2, m)
    assert truncation_bound(x, m, 2) == pytest.approx(2 * R2 + 4 * R2 ** 2, rel=1e-12)
    assert truncation_bound(x, m, 2) >= 2 * R2 + R2 ** 2


def test_rounding_bound_equals_binomial_difference():
    """beta sum_l (alpha+beta)^{s-l-1} alpha^l == (alpha+beta)^s - alpha^s (Eq. (rouding)), checked in fractions."""
    x, m, s, sigma = 3.0, 9, 4, 5
    b = x / s
    alpha = Fraction(1) + Fraction(tail_remainder(b, m))
    beta = sum(Fraction(gamma(k * (sigma + 2) + m + 2)) * Fraction(b) ** k / math.factorial(k) for k in range(m + 1))
    exact = float((alpha + beta) ** s - alpha ** s)
    assert rounding_bound(x, m, s, sigma) == pytest.approx(exact, rel=1e-12)


def _rand_herm(d, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    return (a + a.conj().T) / 2


@pytest.mark.parametrize("xtarget,tau,seed", [(0.5, 1e-8, 1), (2.0, 1e-6, 2), (5.0, 1e-10, 3), (10.0, 1e-8, 4),
                                              (3.0, 1e-12, 5)])
def test_selected_pair_bounds_the_actual_error(xtarget, tau, seed):
    """eps_{A,Psi}(m,s) < E_A(m,s) <= tau (Eq. (accuracy inequality)) against the exact exponential."""
    d = 12
    H = _rand_herm(d, seed)
    dt = xtarget / one_norm(H)
    A = -1j * dt * H
    x = one_norm(A)
    sigma = d
    ms = select_ms(x, tau, sigma)
    assert ms is not None
    m, s = ms
    EA = error_bound(x, m, s, sigma)
    assert EA <= tau
    rng = np.random.default_rng(seed + 7)
    for _ in range(3):
        psi = rng.standard_normal(d) + 1j * rng.standard_normal(d)
        psi /= np.linalg.norm(psi)
        exact = sla.expm(A) @ psi
        approx = taylor_action(A, psi, m, s)
        err = np.linalg.norm(exact - approx) / np.linalg.norm(exact)
        assert err < EA
        # the rule is minimal: one fewer Taylor order at the chosen s violates tau
        if m > 1:
            assert error_bound(x, m - 1, s, sigma) > tau


def test_selection_rule_smallest_s_then_smallest_m():
    x, tau, sigma = 7.3, 1e-10, 9
    m, s = select_ms(x, tau, sigma)
    for s2 in range(1, s):
        assert all(error_bound(x, mm, s2, sigma) > tau for mm in range(1, 61))
    assert all(error_bound(x, mm, s, sigma) > tau for mm in range(1, m))
    assert error_bound(x, m, s, sigma) <= tau


def test_selection_monotone_in_norm_and_tolerance():
    sigma = 5
    prev = (0, 0)
    for x in np.linspace(0.05, 12.0, 40):
        m, s = select_ms(float(x), 1e-10, sigma)
        assert (s, m) >= prev
        prev = (s, m)
    mu = [np.prod(select_ms(4.0, tau, sigma)) for tau in (1e-6, 1e-8, 1e-10, 1e-12)]
    assert mu == sorted(mu)


def test_bound_infeasible_at_tiny_tau():
    """FP64 rounding alone exceeds tau = 1e-17 for every pair: the rule must report no solution."""
    assert select_ms(1.0, 1e-17, 5, s_max=64) is None
    assert math.isinf(error_bound(50.0, 5, 1, 5))


def test_unit_roundoff_is_fp64():
    assert U64 == 2.0 ** -53


@pytest.mark.parametrize("tau,expected", [(1e-8, (41, 3)), (1e-10, (32, 5)), (1e-12, (19, 22))])
def test_rule_reproduces_independent_probe_at_norm_30(tau, expected):
    """(m, s) at ||A||_1 = 30, sigma' = 9, m <= 60 (Sec. III.B rule on Eq. (overallupperbound)).

    The expected pairs were computed once, independently of this module, by a separate evaluation of
    the bound when the workloads were sized (the C3 transmon-cavity norm is about 30)."""
    assert select_ms(30.0, tau, 9) == expected


def _beta_decimal(b: float, indices):
    """sum_k gamma_{indices[k]} b^k / k! in 60-digit decimal arithmetic, gamma_n = n u'/(1 - n u'),
    u' = 2 sqrt(2) u / (1 - 2u), u = 2^-53 (App. C.2)."""
    getcontext().prec = 60
    u = Decimal(1) / Decimal(2 ** 53)
    up = 2 * Decimal(2).sqrt() * u / (1 - 2 * u)
    B = Decimal(repr(b))
    total = Decimal(0)
    for k, n in enumerate(indices):
        g = n * up / (1 - n * up)
        total += g * B ** k / math.factorial(k)
    return total


# The gamma indices of Eq. (B23), k (sigma' + 2) + m + 2 for k = 0..m, listed by hand for small cases.
@pytest.mark.parametrize("b,m,sigma,indices", [
    (0.7, 1, 1, [3, 6]),
    (1.3, 2, 3, [4, 9, 14]),
    (2.5, 3, 9, [5, 16, 27, 38]),
    (0.2, 4, 5, [6, 13, 20, 27, 34]),
])
def test_beta_matches_hand_listed_gamma_indices(b, m, sigma, indices):
    """With s = 1 the rounding bound of Eq. (rouding) is beta itself; beta must equal the hand-listed sum.

    A plausible slip in the index (sigma' + 1 instead of sigma' + 2, or m + 1 instead of m + 2)
    moves beta by far more than the tolerance, which the second assertion checks."""
    beta = float(_beta_decimal(b, indices))
    assert rounding_bound(b, m, 1, sigma) == pytest.approx(beta, rel=1e-13)
    slipped = float(_beta_decimal(b, [n - k for k, n in enumerate(indices)]))
    assert abs(slipped - beta) > 1e-4 * beta
    shifted = float(_beta_decimal(b, [n - 1 for n in indices]))
    assert abs(shifted - beta) > 1e-4 * beta


@pytest.mark.parametrize("x,seed", [(0.5, 11), (2.0, 12), (6.0, 13)])
def test_error_bound_holds_for_single_precision_arithmetic(x, seed):
    """E_A with u = 2^-24 bounds the error of the action actually evaluated in complex64 (App. C)."""
    from oracle.taylor_bound import U32

    d = 10
    H = _rand_herm(d, seed)
    A = -1j * (x / one_norm(H)) * H
    sigma = d
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    psi /= np.linalg.norm(psi)
    exact = sla.expm(A) @ psi
    for m, s in [(12, 1), (8, 2), (10, 4)]:
        EA = error_bound(one_norm(A), m, s, sigma, U32)
        if math.isinf(EA):
            continue
        Bf = (A / s).astype(np.complex64)
        c = psi.astype(np.complex64)
        for _ in range(s):
            term = c
            acc = c.copy()
            for j in range(1, m + 1):
                term = (Bf @ term) / np.float32(j)
                acc = acc + term
            c = acc
        err = np.linalg.norm(exact - c.astype(np.complex128))
        assert err <= EA, (m, s, err, EA)
