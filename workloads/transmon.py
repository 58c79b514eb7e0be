"""Builders for the synthetic transmon/cavity GRAPE workloads.

Every builder returns a :class:`Problem` holding plain arrays.  Conventions:

* Product basis, transmon-major: ``|t, c>`` has index ``t * n_cav + c``; with two
  transmons ``|t1, t2, c>`` has index ``(t1 * n_t + t2) * n_cav + c``.
* ``b`` is the transmon lowering operator, ``a`` the cavity lowering operator
  (the paper writes ``c`` for the cavity, Eq. (fockH)).
* Drift ``H0 = sum_i [(alpha/2) n_i (n_i - 1) + chi n_a n_i] (+ J (b1^+ b2 + b1 b2^+))``
  in the frame rotating with the drives; controls are the x/y quadratures
  ``b + b^+`` and ``i (b - b^+)`` of every driven mode (both Hermitian).
* Controls ``u`` are real, shape ``(K, N)`` (Sec. II, Eq. (2) with one row per
  control channel), in rad/ns.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

TWO_PI = 2.0 * np.pi


@dataclass
class Problem:
    """One GRAPE cost+gradient problem: drift, controls, states, weights, u."""

    name: str
    dim: int
    dt: float
    n_steps: int
    H0: sp.csr_matrix
    Hk: list
    psi0: np.ndarray          # (dim, n_states) complex128, column h = |psi_0^h>
    target: np.ndarray        # (dim, n_states) complex128, column h = U_T |psi_0^h>
    omega: np.ndarray | None  # (dim,) float64 diagonal of the forbidden projector, or None
    w_fid: float = 1.0
    w_forbid: float = 0.0
    w_amp: float = 0.0
    w_tint: float = 0.0            # weight of the time-integrated infidelity C3 (App. A)
    u0: np.ndarray | None = None   # (K, N) float64 seeded controls
    tau: float = 1e-12
    meta: dict = field(default_factory=dict)

    @property
    def n_controls(self) -> int:
        return len(self.Hk)

    @property
    def n_states(self) -> int:
        return self.psi0.shape[1]

    def dense(self):
        """(H0, [H_k]) as dense complex128 arrays (small dims only)."""
        return self.H0.toarray(), [h.toarray() for h in self.Hk]

    def union_nnz(self) -> int:
        pat = abs(self.H0).astype(bool)
        for h in self.Hk:
            pat = pat + abs(h).astype(bool)
        return int(pat.nnz)


def _lower(n: int) -> sp.csr_matrix:
    """Truncated lowering operator on n levels."""
    return sp.diags([np.sqrt(np.arange(1, n, dtype=np.float64))], [1], shape=(n, n), format="csr").astype(np.complex128)


def _kron(*ops) -> sp.csr_matrix:
    out = ops[0]
    for o in ops[1:]:
        out = sp.kron(out, o, format="csr")
    return out.tocsr()


def _quadratures(op: sp.csr_matrix):
    """(op + op^+, i (op - op^+)): the x and y drive quadratures (both Hermitian)."""
    x = (op + op.getH()).tocsr()
    y = (1j * (op - op.getH())).tocsr()
    x.eliminate_zeros()
    y.eliminate_zeros()
    return x, y


def transmon_cavity(n_t: int, n_c: int, alpha_ghz: float = -0.225, chi_ghz: float = -0.002):
    """Drift and [b_x, b_y, a_x, a_y] controls for one transmon (n_t levels) x cavity (n_c levels)."""
    alpha = TWO_PI * alpha_ghz
    chi = TWO_PI * chi_ghz
    b1, a1 = _lower(n_t), _lower(n_c)
    It, Ic = sp.identity(n_t, format="csr", dtype=np.complex128), sp.identity(n_c, format="csr", dtype=np.complex128)
    nb1 = (b1.getH() @ b1).tocsr()
    na1 = (a1.getH() @ a1).tocsr()
    b = _kron(b1, Ic)
    a = _kron(It, a1)
    nb = _kron(nb1, Ic)
    na = _kron(It, na1)
    H0 = (0.5 * alpha) * (nb @ (nb - _kron(It, Ic))) + chi * (na @ nb)
    H0 = sp.csr_matrix(H0)
    H0.eliminate_zeros()
    bx, by = _quadratures(b)
    ax, ay = _quadratures(a)
    return H0.tocsr(), [bx, by, ax, ay]


def two_transmon_cavity(n_t: int, n_c: int, alpha_ghz: float = -0.225, chi_ghz: float = -0.002, j_ghz: float = 0.005):
    """Drift and [b1_x, b1_y, b2_x, b2_y, a_x, a_y] for two transmons (n_t levels each) x cavity (n_c)."""
    alpha = TWO_PI * alpha_ghz
    chi = TWO_PI * chi_ghz
    J = TWO_PI * j_ghz
    bt, ac = _lower(n_t), _lower(n_c)
    It = sp.identity(n_t, format="csr", dtype=np.complex128)
    Ic = sp.identity(n_c, format="csr", dtype=np.complex128)
    I_all = _kron(It, It, Ic)
    b1 = _kron(bt, It, Ic)
    b2 = _kron(It, bt, Ic)
    a = _kron(It, It, ac)
    n1 = (b1.getH() @ b1).tocsr()
    n2 = (b2.getH() @ b2).tocsr()
    na = (a.getH() @ a).tocsr()
    H0 = sp.csr_matrix((0.5 * alpha) * (n1 @ (n1 - I_all)) + (0.5 * alpha) * (n2 @ (n2 - I_all))
                       + chi * (na @ n1) + chi * (na @ n2) + J * (b1.getH() @ b2 + b1 @ b2.getH()))
    H0.eliminate_zeros()
    ctrls = []
    for op in (b1, b2, a):
        ctrls.extend(_quadratures(op))
    return H0.tocsr(), ctrls


def smooth_controls(n_controls: int, n_steps: int, dt: float, seed: int, rms_ghz: float = 0.01,
                    sigma_ns: float = 5.0) -> np.ndarray:
    """Seeded Gaussian-smoothed noise, one row per control, each row scaled to RMS 2 pi rms_ghz.

    White noise from ``default_rng(seed)`` is convolved along the time axis with a
    normalised Gaussian of width ``sigma_ns / dt`` steps, truncated at 4 sigma, with
    mirror-symmetric boundary extension.
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n_controls, n_steps))
    sig = sigma_ns / dt
    r = int(4.0 * sig + 0.5)
    x = np.arange(-r, r + 1, dtype=np.float64)
    ker = np.exp(-0.5 * (x / sig) ** 2)
    ker /= ker.sum()
    out = np.empty_like(w)
    for k in range(n_controls):
        padded = np.pad(w[k], r, mode="symmetric") if r < n_steps else np.pad(w[k], r, mode="wrap")
        out[k] = np.convolve(padded, ker, mode="valid")
    rms = np.sqrt(np.mean(out ** 2, axis=1, keepdims=True))
    rms[rms == 0] = 1.0
    return out * (TWO_PI * rms_ghz / rms)


def haar_unitary(n: int, seed: int) -> np.ndarray:
    """Haar-random n x n unitary: QR of a complex Gaussian with the R-diagonal phase fixed (Mezzadri)."""
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


def _basis_columns(dim: int, indices) -> np.ndarray:
    out = np.zeros((dim, len(indices)), dtype=np.complex128)
    for h, i in enumerate(indices):
        out[i, h] = 1.0
    return out


def _subspace_one(n_t, n_c, n_states, n_cav_levels=4):
    idx = [t * n_c + c for t in (0, 1) for c in range(min(n_cav_levels, n_c))]
    return idx[:n_states]


def _subspace_two(n_t, n_c, n_states, n_cav_levels):
    idx = [(t1 * n_t + t2) * n_c + c for t1 in (0, 1) for t2 in (0, 1) for c in range(min(n_cav_levels, n_c))]
    return idx[:n_states]


def _gate_problem(name, H0, Hk, dim, idx, dt, n_steps, seed, omega, w_fid, w_forbid, w_amp, tau, meta):
    psi0 = _basis_columns(dim, idx)
    UT = haar_unitary(len(idx), seed + 100000)
    target = psi0 @ UT            # phi_T^h = U_T psi_0^h restricted to the subspace
    u0 = smooth_controls(len(Hk), n_steps, dt, seed)
    return Problem(name=name, dim=dim, dt=dt, n_steps=n_steps, H0=H0, Hk=Hk, psi0=psi0, target=target,
                   omega=omega, w_fid=w_fid, w_forbid=w_forbid, w_amp=w_amp, u0=u0, tau=tau, meta=meta)


CONFIGS = {
    # name: description
    "c1_state_transfer_d30": "transmon 3 x cavity 10, 4 controls, N=200, dt=1 ns, |g,0> -> |g,1>",
    "c2_gate_d80": "transmon 4 x cavity 20, 4 controls, 8-state Haar gate, forbidden level 3, N=1000, dt=0.5 ns",
    "c3_gate_d4000": "transmons 4 x 4 x cavity 250, 6 controls, 4-state gate, N=2000, dt=1 ns",
    "c4_gate_d16000": "transmons 4 x 4 x cavity 1000, 6 controls, 16-state gate, N=4000, dt=0.5 ns",
}


def config_names():
    return list(CONFIGS)


def build_config(name: str, seed: int | None = None, n_steps: int | None = None, tau: float | None = None) -> Problem:
    """Build one of the named workloads; ``n_steps`` overrides N (for reduced-size checks)."""
    if name == "c1_state_transfer_d30":
        n_t, n_c, dt, N = 3, 10, 1.0, 200
        seed = 1 if seed is None else seed
        N = N if n_steps is None else n_steps
        H0, Hk = transmon_cavity(n_t, n_c)
        dim = n_t * n_c
        psi0 = _basis_columns(dim, [0 * n_c + 0])
        target = _basis_columns(dim, [0 * n_c + 1])
        u0 = smooth_controls(len(Hk), N, dt, seed)
        return Problem(name=name, dim=dim, dt=dt, n_steps=N, H0=H0, Hk=Hk, psi0=psi0, target=target, omega=None,
                       w_fid=1.0, w_forbid=0.0, w_amp=0.0, u0=u0, tau=1e-12 if tau is None else tau,
                       meta={"n_t": n_t, "n_c": n_c, "seed": seed})
    if name == "c2_gate_d80":
        n_t, n_c, dt, N = 4, 20, 0.5, 1000
        seed = 2 if seed is None else seed
        N = N if n_steps is None else n_steps
        H0, Hk = transmon_cavity(n_t, n_c)
        dim = n_t * n_c
        omega = np.array([1.0 if (i // n_c) == 3 else 0.0 for i in range(dim)])
        return _gate_problem(name, H0, Hk, dim, _subspace_one(n_t, n_c, 8), dt, N, seed, omega, 1.0, 1.0, 1e-2,
                             1e-12 if tau is None else tau, {"n_t": n_t, "n_c": n_c, "seed": seed})
    if name in ("c3_gate_d4000", "c4_gate_d16000"):
        big = name == "c4_gate_d16000"
        n_t, n_c = 4, (1000 if big else 250)
        dt, N = (0.5, 4000) if big else (1.0, 2000)
        n_states = 16 if big else 4
        seed = (4 if big else 3) if seed is None else seed
        N = N if n_steps is None else n_steps
        H0, Hk = two_transmon_cavity(n_t, n_c)
        dim = n_t * n_t * n_c
        t1 = np.arange(dim) // (n_t * n_c)
        t2 = (np.arange(dim) // n_c) % n_t
        omega = ((t1 == 3) | (t2 == 3)).astype(np.float64)
        idx = _subspace_two(n_t, n_c, n_states, 4 if big else 1)
        return _gate_problem(name, H0, Hk, dim, idx, dt, N, seed, omega, 1.0, 1.0, 1e-2,
                             (1e-10 if tau is None else tau), {"n_t": n_t, "n_c": n_c, "seed": seed})
    raise KeyError(f"unknown config {name!r}; known: {config_names()}")


def two_level_rabi(n_steps: int, dt: float, delta: float = 0.0, target_excited: bool = True) -> Problem:
    """Two-level system ``H = (delta/2) sigma_z + u_x sigma_x`` starting in |g> (index 0).

    With constant ``u_x`` the transfer probability has the textbook Rabi closed form,
    which pins the oracle's propagator, cost and gradient.
    """
    sz = sp.csr_matrix(np.array([[-1.0, 0.0], [0.0, 1.0]], dtype=np.complex128))  # |g>=0 has energy -1
    sx = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 0.0]], dtype=np.complex128))
    H0 = (0.5 * delta) * sz
    H0 = sp.csr_matrix(H0)
    psi0 = _basis_columns(2, [0])
    target = _basis_columns(2, [1 if target_excited else 0])
    omega = np.array([0.0, 1.0])
    return Problem(name="rabi", dim=2, dt=dt, n_steps=n_steps, H0=H0.tocsr(), Hk=[sx], psi0=psi0, target=target,
                   omega=omega, w_fid=1.0, w_forbid=0.0, w_amp=0.0,
                   u0=np.zeros((1, n_steps)), tau=1e-12, meta={"delta": delta})


def random_problem(dim: int, n_controls: int, n_states: int, n_steps: int, seed: int, dt: float = 0.3,
                   band: int = 3, density: float = 0.0, gate: bool = True, w_forbid: float = 0.5,
                   w_amp: float = 0.05, scale: float = 1.0, tau: float = 1e-12) -> Problem:
    """Random Hermitian banded (+ optional scattered) drift and controls, for ragged-size parity tests.

    The drift has a real random diagonal and complex off-diagonals within ``band``;
    each control is Hermitian with a random subset of the band plus, if
    ``density > 0``, scattered symmetric entries.  States are orthonormal columns
    of a seeded Haar unitary; the target applies a second Haar unitary inside
    the spanned subspace.
    """
    rng = np.random.default_rng(seed)

    def herm_band(p_keep, diag_scale):
        rows, cols, vals = [], [], []
        for i in range(dim):
            rows.append(i); cols.append(i); vals.append(diag_scale * rng.standard_normal())
            for off in range(1, band + 1):
                j = i + off
                if j < dim and rng.random() < p_keep:
                    v = (rng.standard_normal() + 1j * rng.standard_normal()) * 0.5
                    rows += [i, j]; cols += [j, i]; vals += [v, np.conj(v)]
        m = sp.csr_matrix((np.array(vals, dtype=np.complex128), (rows, cols)), shape=(dim, dim))
        if density > 0:
            nn = int(density * dim * dim / 2)
            ii = rng.integers(0, dim, nn)
            jj = rng.integers(0, dim, nn)
            vv = (rng.standard_normal(nn) + 1j * rng.standard_normal(nn)) * 0.3
            s = sp.csr_matrix((vv, (ii, jj)), shape=(dim, dim))
            m = m + s + s.getH()
        m.sum_duplicates()
        return (scale * m).tocsr()

    H0 = herm_band(0.9, 1.0)
    Hk = []
    for _ in range(n_controls):
        h = herm_band(0.5, 0.0)
        h.setdiag(0.2 * rng.standard_normal(dim))
        h.eliminate_zeros()
        Hk.append(h.tocsr())
    V = haar_unitary(dim, seed + 1)
    psi0 = V[:, :n_states].copy()
    if gate:
        target = psi0 @ haar_unitary(n_states, seed + 2)
    else:
        target = V[:, n_states:n_states + n_states].copy() if 2 * n_states <= dim else V[:, ::-1][:, :n_states].copy()
    omega = (rng.random(dim) < 0.2).astype(np.float64)
    u0 = 0.5 * rng.standard_normal((n_controls, n_steps))
    return Problem(name=f"random_d{dim}_k{n_controls}_n{n_states}_N{n_steps}", dim=dim, dt=dt, n_steps=n_steps,
                   H0=H0, Hk=Hk, psi0=psi0, target=target, omega=omega, w_fid=1.0, w_forbid=w_forbid, w_amp=w_amp,
                   u0=u0, tau=tau, meta={"seed": seed})


def batch_instances(seed: int = 5, count: int = 64):
    """64 independent GRAPE instances of uneven size (dims 30/80/240/1000/4000), seeded.

    Per instance i: N ~ U[200, 2000], K ~ U{2..6} (clamped to the number of
    available controls, first K of the ordered list), n ~ U{1..8}; controls and
    targets use seed 5000 + i.
    """
    rng = np.random.default_rng(seed)
    systems = [("t3c10", 30), ("t4c20", 80), ("t4c60", 240), ("t4c250", 1000), ("tt4c250", 4000)]
    counts = rng.multinomial(count, [0.2] * 5)
    out = []
    i = 0
    for (sysname, dim), cnt in zip(systems, counts):
        for _ in range(cnt):
            N = int(rng.integers(200, 2001))
            K = int(rng.integers(2, 7))
            n = int(rng.integers(1, 9))
            s = 5000 + i
            if sysname == "tt4c250":
                H0, Hk = two_transmon_cavity(4, 250)
                idx = _subspace_two(4, 250, n, 2)
                t1 = np.arange(dim) // 1000
                t2 = (np.arange(dim) // 250) % 4
                omega = ((t1 == 3) | (t2 == 3)).astype(np.float64)
            else:
                n_t = 3 if sysname == "t3c10" else 4
                n_c = dim // n_t
                H0, Hk = transmon_cavity(n_t, n_c)
                idx = _subspace_one(n_t, n_c, n)
                omega = np.array([1.0 if (j // n_c) == n_t - 1 else 0.0 for j in range(dim)])
            Hk = Hk[:min(K, len(Hk))]
            p = _gate_problem(f"batch{i}_{sysname}", H0, Hk, dim, idx, 1.0, N, s, omega, 1.0, 1.0, 1e-2, 1e-10,
                              {"system": sysname, "seed": s})
            out.append(p)
            i += 1
    return out
