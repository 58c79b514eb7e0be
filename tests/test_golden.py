"""The oracle against tests/golden/rabi_closed_forms.txt (closed forms in 40-digit arithmetic).

The fixture is written by tests/golden/make_golden.py from the textbook two-level transition
probability; it shares nothing with the oracle.  Each row gives C1, C2, C3 (target |e>,
Omega = |e><e|) and their derivatives with respect to a constant drive, which equal the sums of
the per-step gradient entries.
"""

import os

import numpy as np
import pytest

from oracle import cost_and_grad
from workloads import two_level_rabi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rabi_closed_forms.txt")


def golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            rows.append((float(t[0]), float(t[1]), float(t[2]), int(t[3]), [float(x) for x in t[4:]]))
    return rows


def rabi_case(delta, u, dt, N, term):
    """The two-level problem with only one cost term switched on (term = 'C1' | 'C2' | 'C3')."""
    p = two_level_rabi(N, dt, delta=delta, target_excited=True)
    p.w_fid, p.w_forbid, p.w_amp, p.w_tint = (1.0, 0.0, 0.0, 0.0) if term == "C1" else \
        (0.0, 1.0, 0.0, 0.0) if term == "C2" else (0.0, 0.0, 0.0, 1.0)
    return p, np.full((1, N), u)


TERMS = {"C1": 0, "C2": 2, "C3": 4}


@pytest.mark.parametrize("row", golden_rows())
@pytest.mark.parametrize("term", list(TERMS))
def test_oracle_matches_closed_forms(row, term):
    delta, u, dt, N, vals = row
    p, uu = rabi_case(delta, u, dt, N, term)
    r = cost_and_grad(p, uu)
    c_ref, d_ref = vals[TERMS[term]], vals[TERMS[term] + 1]
    assert abs(r.cost - c_ref) <= 1e-13
    assert abs(np.sum(r.grad) - d_ref) <= 1e-12 * max(1.0, abs(d_ref))
