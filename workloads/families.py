"""Further Hamiltonian families of the paper, as GRAPE workloads.

* ``three_transmons``: three resonantly driven transmons with nearest-neighbour
  exchange, Eq. (gateH) (H_2), target: a Hadamard on every transmon's {0, 1}
  subspace (Sec. IV.B, gate benchmark).
* ``qubit_chain``: N_q qubits with x/y drives and nearest-neighbour sigma_z sigma_z
  coupling (H_3, App. on the scaling of mu); the union pattern grows like d log d.
* ``fluxonium_pair``: two capacitively coupled fluxonium qubits controlled through
  their external fluxes, Eq. (fluxonium) (H_4), in the harmonic-oscillator basis,
  where cos(phi) is a dense operator (the row count of nonzeros grows with the
  cutoff).

The paper states no parameter values for these systems; the values below are
typical circuit-QED numbers in GHz (converted to rad/ns), documented per builder.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .transmon import TWO_PI, Problem, _basis_columns, _kron, _lower, haar_unitary, smooth_controls


def _eye(n: int) -> sp.csr_matrix:
    return sp.identity(n, format="csr", dtype=np.complex128)


def three_transmons(n_t: int, alpha_ghz: float = -0.225, g_ghz: float = 0.005):
    """H_2 (Eq. (gateH)): drift sum_nu (alpha/2) n_nu (n_nu - 1) + g (b1 b2^+ + b2 b3^+ + h.c.) and the
    three drive operators b_nu + b_nu^+ (one real control a^(nu) per transmon)."""
    alpha = TWO_PI * alpha_ghz
    g = TWO_PI * g_ghz
    b1 = _lower(n_t)
    It = _eye(n_t)
    b = [_kron(b1, It, It), _kron(It, b1, It), _kron(It, It, b1)]
    I_all = _kron(It, It, It)
    H0 = sp.csr_matrix((n_t ** 3, n_t ** 3), dtype=np.complex128)
    for bv in b:
        nv = (bv.getH() @ bv).tocsr()
        H0 = H0 + (0.5 * alpha) * (nv @ (nv - I_all))
    exch = b[0] @ b[1].getH() + b[1] @ b[2].getH()
    H0 = sp.csr_matrix(H0 + g * (exch + exch.getH()))
    H0.eliminate_zeros()
    Hk = []
    for bv in b:
        x = (bv + bv.getH()).tocsr()
        x.eliminate_zeros()
        Hk.append(x)
    return H0.tocsr(), Hk


def hadamard3_problem(n_t: int, n_steps: int, dt: float, seed: int, tau: float = 1e-10,
                      w_forbid: float = 1.0, w_amp: float = 1e-2) -> Problem:
    """Simultaneous Hadamard on the {0,1} subspace of each of three transmons (8 columns; C1 gate form).

    Index convention |t1, t2, t3> -> (t1 n_t + t2) n_t + t3.  The forbidden projector Omega
    marks every basis state with some transmon in its highest kept level.
    """
    H0, Hk = three_transmons(n_t)
    dim = n_t ** 3
    comp = [(t1 * n_t + t2) * n_t + t3 for t1 in (0, 1) for t2 in (0, 1) for t3 in (0, 1)]
    psi0 = _basis_columns(dim, comp)
    h = np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)
    UT = np.kron(np.kron(h, h), h).astype(np.complex128)
    target = psi0 @ UT
    levels = np.array([[(i // (n_t * n_t)), (i // n_t) % n_t, i % n_t] for i in range(dim)])
    omega = (levels == n_t - 1).any(axis=1).astype(np.float64)
    u0 = smooth_controls(len(Hk), n_steps, dt, seed, rms_ghz=0.02)
    return Problem(name=f"h2_hadamard3_d{dim}", dim=dim, dt=dt, n_steps=n_steps, H0=H0, Hk=Hk, psi0=psi0,
                   target=target, omega=omega, w_fid=1.0, w_forbid=w_forbid, w_amp=w_amp, u0=u0, tau=tau,
                   meta={"family": "H_2", "n_t": n_t, "seed": seed})


def qubit_chain(n_q: int, g_ghz: float = 0.01):
    """H_3: drift g sum_nu sigma_z^nu sigma_z^{nu+1}; controls [sigma_x^1, sigma_y^1, sigma_x^2, ...] (K = 2 N_q).

    Qubit 1 is the most significant bit of the basis index."""
    g = TWO_PI * g_ghz
    sx = sp.csr_matrix(np.array([[0, 1], [1, 0]], dtype=np.complex128))
    sy = sp.csr_matrix(np.array([[0, -1j], [1j, 0]], dtype=np.complex128))
    sz = sp.csr_matrix(np.array([[1, 0], [0, -1]], dtype=np.complex128))
    I2 = _eye(2)

    def site(op, nu):
        return _kron(*[op if j == nu else I2 for j in range(n_q)])

    dim = 2 ** n_q
    H0 = sp.csr_matrix((dim, dim), dtype=np.complex128)
    for nu in range(n_q - 1):
        H0 = H0 + g * (site(sz, nu) @ site(sz, nu + 1))
    H0 = sp.csr_matrix(H0)
    H0.eliminate_zeros()
    Hk = []
    for nu in range(n_q):
        Hk.append(site(sx, nu).tocsr())
        Hk.append(site(sy, nu).tocsr())
    return H0.tocsr(), Hk


def qubit_chain_problem(n_q: int, n_steps: int, dt: float, seed: int, n_states: int = 4, tau: float = 1e-10,
                        w_amp: float = 1e-2) -> Problem:
    """A Haar-random gate on the span of the first ``n_states`` computational basis states (C1 gate form)."""
    H0, Hk = qubit_chain(n_q)
    dim = 2 ** n_q
    idx = list(range(n_states))
    psi0 = _basis_columns(dim, idx)
    target = psi0 @ haar_unitary(n_states, seed + 100000)
    u0 = smooth_controls(len(Hk), n_steps, dt, seed, rms_ghz=0.02)
    return Problem(name=f"h3_qubit_chain_d{dim}", dim=dim, dt=dt, n_steps=n_steps, H0=H0, Hk=Hk, psi0=psi0,
                   target=target, omega=None, w_fid=1.0, w_forbid=0.0, w_amp=w_amp, u0=u0, tau=tau,
                   meta={"family": "H_3", "n_q": n_q, "seed": seed})


def _fluxonium_ops(n_cut: int, ec: float, ej: float, el: float, pad: int = 40):
    """(H_single, phi, n) of one fluxonium truncated to ``n_cut`` oscillator levels.

    phi = phi_zpf (b + b^+), n = i n_zpf (b^+ - b) with phi_zpf = (2 E_C / E_L)^(1/4) and
    n_zpf = (E_L / (32 E_C))^(1/4) (so that [phi, n] = i); 4 E_C n^2 + (E_L/2) phi^2 and cos(phi)
    are formed in a basis ``pad`` levels larger and then truncated, so that the kept block does
    not carry the truncation error of the operator products.
    """
    M = n_cut + pad
    b = _lower(M).toarray()
    phi_zpf = (2.0 * ec / el) ** 0.25
    n_zpf = (el / (32.0 * ec)) ** 0.25
    phi = phi_zpf * (b + b.conj().T)
    nop = 1j * n_zpf * (b.conj().T - b)
    lam, V = np.linalg.eigh(phi)
    cosphi = (V * np.cos(lam)[None, :]) @ V.conj().T
    H = 4.0 * ec * (nop @ nop) + 0.5 * el * (phi @ phi) - ej * cosphi
    k = slice(0, n_cut)
    return H[k, k], phi[k, k], nop[k, k]


def fluxonium_pair(n_cut: int, ec_ghz=(1.0, 1.1), ej_ghz=(4.0, 4.2), el_ghz=(1.0, 0.9), g_ghz: float = 0.02,
                   drop: float = 1e-12):
    """H_4 (Eq. (fluxonium)) without the control-squared identity term.

    Expanding (E_L/2)(phi - phi_ext)^2 gives (E_L/2) phi^2 - E_L phi_ext phi + (E_L/2) phi_ext^2; the
    last term is a multiple of the identity (a global phase, invisible to every cost term), so it is
    left out and H is linear in the controls u_i = phi_ext,i with H_i = -E_L,i phi_i.  Entries below
    ``drop`` times the largest are removed (cos(phi) is dense in the oscillator basis), and the drift
    is shifted by a multiple of the identity so that its diagonal range is centred on zero (again a
    global phase) to keep ||A||_1 small.
    """
    ops = [_fluxonium_ops(n_cut, TWO_PI * ec_ghz[i], TWO_PI * ej_ghz[i], TWO_PI * el_ghz[i]) for i in (0, 1)]
    I = np.eye(n_cut)
    g = TWO_PI * g_ghz
    H0 = np.kron(ops[0][0], I) + np.kron(I, ops[1][0]) + g * np.kron(ops[0][2], ops[1][2])
    diag = np.real(np.diag(H0))
    H0 = H0 - 0.5 * (diag.max() + diag.min()) * np.eye(n_cut * n_cut)
    el = [TWO_PI * el_ghz[i] for i in (0, 1)]
    Hk = [-el[0] * np.kron(ops[0][1], I), -el[1] * np.kron(I, ops[1][1])]

    def sparse(m):
        m = np.where(np.abs(m) > drop * np.abs(m).max(), m, 0.0)
        m = 0.5 * (m + m.conj().T)
        out = sp.csr_matrix(m.astype(np.complex128))
        out.eliminate_zeros()
        return out

    return sparse(H0), [sparse(h) for h in Hk]


def fluxonium_problem(n_cut: int, n_steps: int, dt: float, seed: int, n_states: int = 4, tau: float = 1e-10,
                      w_amp: float = 1e-2) -> Problem:
    """A Haar-random gate on the span of the ``n_states`` lowest eigenstates of the drift (C1 gate form)."""
    H0, Hk = fluxonium_pair(n_cut)
    dim = n_cut * n_cut
    lam, V = np.linalg.eigh(H0.toarray())
    psi0 = np.ascontiguousarray(V[:, :n_states]).astype(np.complex128)
    target = psi0 @ haar_unitary(n_states, seed + 100000)
    u0 = smooth_controls(len(Hk), n_steps, dt, seed, rms_ghz=0.01)
    return Problem(name=f"h4_fluxonium_pair_d{dim}", dim=dim, dt=dt, n_steps=n_steps, H0=H0, Hk=Hk, psi0=psi0,
                   target=target, omega=None, w_fid=1.0, w_forbid=0.0, w_amp=w_amp, u0=u0, tau=tau,
                   meta={"family": "H_4", "n_cut": n_cut, "seed": seed})
