"""Writes rabi_closed_forms.txt: closed-form costs of a driven two-level system, in 40-digit arithmetic.

Independent of the oracle and of the CUDA path: the values come from the textbook transition
probability of H = (delta/2) sigma_z + u sigma_x (constant drive u, state |g> at t = 0),

    P_e(t) = (u / W)^2 sin^2(W t),   W = sqrt(u^2 + delta^2 / 4),

evaluated with mpmath.  For N steps of length dt (t_n = n dt) and target |e>:

    C1 = 1 - P_e(N dt)                              (Sec. III.A, Eq. (C1st), n = 1)
    C2 = (1/N) sum_{n=1..N} P_e(n dt)               (App. A, Eq. (c2st), Omega = |e><e|)
    C3 = 1 - (1/N) sum_{n=1..N} P_e(n dt)           (App. A, C3st)

and, for each, the derivative with respect to the constant drive u, which equals the sum over the
N per-step gradient entries dC/du_n (every step carries the same u).

Run:  python tests/golden/make_golden.py   (rewrites the fixture next to this script)
"""

import os

import mpmath as mp

mp.mp.dps = 40

CASES = [  # delta, u, dt, N
    ("0", "0.3", "0.37", 7),
    ("0.4", "0.45", "0.41", 9),
    ("1.7", "0.15", "0.41", 9),
    ("-0.8", "1.05", "0.2", 13),
    ("2.5", "0.9", "0.05", 40),
]


def p_exc(delta, u, t):
    w = mp.sqrt(u ** 2 + delta ** 2 / 4)
    return (u / w) ** 2 * mp.sin(w * t) ** 2


def costs(delta, u, dt, N):
    pe = [p_exc(delta, u, n * dt) for n in range(1, N + 1)]
    c1 = 1 - pe[-1]
    c2 = mp.fsum(pe) / N
    return c1, c2, 1 - c2


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rabi_closed_forms.txt")
    lines = ["# delta u dt N C1 dC1/du C2 dC2/du C3 dC3/du",
             "# H = (delta/2) sigma_z + u sigma_x, psi_0 = |g>, target |e>, Omega = |e><e|;",
             "# C1 Sec. III.A Eq. (C1st); C2 App. A Eq. (c2st); C3 App. A (C3st); written by make_golden.py"]
    for ds, us, dts, N in CASES:
        delta, u, dt = mp.mpf(ds), mp.mpf(us), mp.mpf(dts)
        c1, c2, c3 = costs(delta, u, dt, N)
        d1 = mp.diff(lambda x: costs(delta, x, dt, N)[0], u)
        d2 = mp.diff(lambda x: costs(delta, x, dt, N)[1], u)
        d3 = mp.diff(lambda x: costs(delta, x, dt, N)[2], u)
        vals = [mp.nstr(v, 25) for v in (c1, d1, c2, d2, c3, d3)]
        lines.append(" ".join([ds, us, dts, str(N)] + vals))
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
