"""Oracle: a plain, slow, FP64 CPU restatement of the superconducting-circuit
evolution that the CUDA library computes.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path (no kernels, headers, helpers, tables or constants); the two meet
only in the seeded input dictionaries of ``paper_2406_18155_gb300.workloads``,
which carry parameters and random draws but none of the method's arithmetic.

What it computes (paper sections in brackets):

* subsystem Hamiltonians, diagonalisation and truncation        [Sec. 2.1, Eq. 8]
* the composite Hamiltonian as an explicit sum of Kronecker
  products of local operators, dense (np.kron) or matrix-free    [Eq. 1, App. B]
* fixed-step classic RK4 time evolution of a batch of columns   (solver reading R1)
* Suzuki-Trotter evolution Q2, Q4, Q4j (the paper's solvers)    [Sec. 2.3, App. A]
  and its discrete adjoint for the pulse parameters              [Sec. 2.5]
* virtual-Z compensation of the gate fidelity and the dressed
  (idle-Hamiltonian eigen-) basis of the gate metric              [App. C]
* the vectorised Lindblad master equation (density matrices)     [App. C]
* the composite state-transfer cost and the average gate
  fidelity                                                      [Eq. 13, Eq. D2]
* the exact discrete adjoint of RK4 (the discretise-then-
  differentiate gradient that the local continuous adjoint
  method computes)                                              [Sec. 2.5, Eqs. 7-12]
* an independent tangent-linear RK4 and central finite
  differences through the whole pipeline, eigendecomposition
  included.

Every floating-point quantity is numpy float64 / complex128.
"""
from .subsystems import (transmon, fluxonium, diagonalise, build_mode,
                         mathieu_transmon_levels)
from .system import OracleSystem
from .evolve import (rk4_evolve, rk4_evolve_matrix_free, frame_epilogue,
                     fidelities, fidelity_and_costate, evolve_and_fidelity,
                     adjoint_gradient, tangent_linear_derivative,
                     finite_difference_gradient, param_vector, set_param_vector)
from .trotter import q2_evolve, q2_evolve_and_fidelity

__all__ = [
    "transmon", "fluxonium", "diagonalise", "build_mode", "mathieu_transmon_levels",
    "OracleSystem", "rk4_evolve", "rk4_evolve_matrix_free", "frame_epilogue",
    "fidelities", "fidelity_and_costate", "evolve_and_fidelity",
    "adjoint_gradient", "tangent_linear_derivative", "finite_difference_gradient",
    "param_vector", "set_param_vector", "q2_evolve", "q2_evolve_and_fidelity",
]
