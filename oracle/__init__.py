"""CPU FP64 oracle for the hard-coded-gradient (HG) GRAPE cost and gradient.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may use it.  It shares no code with the CUDA path.

Contents
--------
``grape_oracle``   exact-exponential cost and gradient (dense ``eigh`` propagators,
                   stored states, divided-difference propagator derivative).
``taylor_bound``   the paper's error bound E_A(m, s) and the (m, s) selection rule
                   (App. C), plus a plain truncated-Taylor action for pins.
``fullad_torch``   a second reference: CPU complex128 torch full automatic
                   differentiation through ``torch.linalg.matrix_exp`` per step.
``sparse_reference`` the same exact-exponential cost and gradient for large sparse
                   problems: exponential actions by ``scipy.sparse.linalg.expm_multiply``
                   and the auxiliary block-matrix derivative (Sec. III.B), pinned to
                   ``grape_oracle`` on small problems.

Every function cites the passage of arXiv:2304.06200 it follows.
"""

from .grape_oracle import (  # noqa: F401
    OracleResult,
    cost_and_grad,
    cost_only,
    step_hamiltonians,
    propagator,
    propagator_derivative,
    forward_states,
)
from .taylor_bound import (  # noqa: F401
    tail_remainder,
    error_bound,
    select_ms,
    taylor_action,
    gamma,
)
