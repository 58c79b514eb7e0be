"""The paper's error bound E_A(m, s) and (m, s) rule for the scaled truncated-Taylor action.

TEST INFRASTRUCTURE ONLY.  Plain Python floats, written out term by term from
Sec. III.B and App. C of arXiv:2304.06200 so that a reader can check it against
the equations.  The CUDA library computes the same rule in its own C++ code;
tests compare the two.

Notation: x = ||A||_1 with A = -i H dt, b = ||B||_1 = x / s, sigma = sigma'
(the largest number of non-zeros in a row of H, Eq. (sigmapdef)), u = unit
roundoff (2^-53 for FP64).
"""

from __future__ import annotations

import math

import numpy as np

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def gamma(n: int, u: float = U64) -> float:
    """gamma_n = n u' / (1 - n u') with u' = 2 sqrt(2) u / (1 - 2u) (App. C.2, below Eqs. (operation error), (c7))."""
    up = 2.0 * math.sqrt(2.0) * u / (1.0 - 2.0 * u)
    if n * up >= 1.0:
        return math.inf
    return n * up / (1.0 - n * up)


def tail_remainder(b: float, m: int) -> float:
    """R_m(b) = sum_{q > m} b^q / q!  (App. C.1, below the first truncation equation).

    Summed forward from q = m + 1 (never as e^b minus the partial sum, which cancels).
    """
    if b <= 0.0:
        return 0.0
    logt = (m + 1) * math.log(b) - math.lgamma(m + 2)
    if logt > 700.0:
        return math.inf
    term = math.exp(logt)
    total = 0.0
    q = m + 1
    while True:
        total += term
        q += 1
        term *= b / q
        if q > b and term <= total * 1e-18:
            break
        if total > 1e300:
            return math.inf
    return total


def truncation_bound(x: float, m: int, s: int) -> float:
    """epsilon_t < s R (1 - (s R)^s) / (1 - s R), R = R_m(||B||_1)  (Eq. (truncation)); inf unless s R < 1."""
    R = tail_remainder(x / s, m)
    sR = s * R
    if not sR < 1.0:
        return math.inf
    return sR * (1.0 - sR ** s) / (1.0 - sR)


def rounding_bound(x: float, m: int, s: int, sigma: int, u: float = U64) -> float:
    """epsilon_r < beta sum_{l=0}^{s-1} (alpha+beta)^{s-l-1} alpha^l = (alpha+beta)^s - alpha^s  (Eq. (rouding)).

    alpha = 1 + R_m(||B||_1); beta = sum_{k=0}^m gamma_{k(sigma+2)+m+2} ||B||_1^k / k!  (Eq. (B23)).
    The sum form is used because its terms are all positive (no cancellation).
    """
    b = x / s
    alpha = 1.0 + tail_remainder(b, m)
    beta = 0.0
    for k in range(m + 1):
        beta += gamma(k * (sigma + 2) + m + 2, u) * b ** k / math.factorial(k)
    total = 0.0
    for l in range(s):
        total += (alpha + beta) ** (s - l - 1) * alpha ** l
    return beta * total


def error_bound(x: float, m: int, s: int, sigma: int, u: float = U64) -> float:
    """E_A(m, s) = truncation bound + rounding bound (Eq. (overallupperbound))."""
    t = truncation_bound(x, m, s)
    if math.isinf(t):
        return math.inf
    return t + rounding_bound(x, m, s, sigma, u)


def select_ms(x: float, tau: float, sigma: int, u: float = U64, m_max: int = 60, s_max: int = 4096):
    """The paper's rule (Sec. III.B, around Eq. (mudefnition)): among pairs with E_A(m, s) <= tau take the
    smallest s, then the smallest m.  Returns (m, s) or None if no pair with m <= m_max, s <= s_max qualifies.
    """
    for s in range(1, s_max + 1):
        for m in range(1, m_max + 1):
            if error_bound(x, m, s, sigma, u) <= tau:
                return m, s
    return None


def taylor_action(A: np.ndarray, psi: np.ndarray, m: int, s: int) -> np.ndarray:
    """(e^B_m)^s psi with B = A / s by repeated products (Eqs. (eBm), (eBmpsi), recursions (C13), (C20))."""
    B = np.asarray(A) / s
    c = np.asarray(psi, dtype=np.complex128)
    for _ in range(s):
        b = c
        acc = b.copy()
        for j in range(1, m + 1):
            b = (B @ b) / j
            acc = acc + b
        c = acc
    return c


def one_norm(H) -> float:
    """||H||_1 = max_j sum_i |H_ij| (equal to the infinity norm for Hermitian H, footnote to Eq. (norm inequality))."""
    Hd = H.toarray() if hasattr(H, "toarray") else np.asarray(H)
    return float(np.max(np.sum(np.abs(Hd), axis=0)))
