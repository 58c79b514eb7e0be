"""Seeded synthetic GRAPE problems shaped like the paper's transmon-cavity workloads.

This module only *builds inputs*: Hamiltonian matrices (as scipy CSR), initial
states, targets, forbidden-state projectors and seeded control amplitudes.  It
holds none of the method's arithmetic (no propagation, no cost, no gradient),
so that both the CPU oracle (``oracle/``) and the CUDA path
(``paper_2304_06200_gb300``) can be fed the same problems without sharing code.

Physical model (Sec. II; benchmark Hamiltonian Eq. (fockH) in Sec. IV.B): in
the frame rotating with the drives, a transmon ``b`` (anharmonicity alpha) is
dispersively coupled to a cavity ``a`` (shift chi) and both are driven by
x/y quadrature controls.  Units: angular frequency in rad/ns (``X/2pi = v GHz``
means ``X = 2 pi v``), time in ns.  ``families`` adds the paper's other
Hamiltonians: three coupled transmons (H_2), a qubit chain (H_3) and a coupled
fluxonium pair (H_4).
"""

from .transmon import (  # noqa: F401
    Problem,
    build_config,
    config_names,
    smooth_controls,
    haar_unitary,
    transmon_cavity,
    two_transmon_cavity,
    two_level_rabi,
    random_problem,
    batch_instances,
)
from .families import (  # noqa: F401
    three_transmons,
    hadamard3_problem,
    qubit_chain,
    qubit_chain_problem,
    fluxonium_pair,
    fluxonium_problem,
)
from .dense import dense_register_gate, gue_drift, qubit0_drives  # noqa: F401
