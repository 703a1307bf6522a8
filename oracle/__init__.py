"""Plain FP64 CPU oracle of one time step of the operator-splitting, fully
decoupled, matrix-based solidification scheme (Algorithm 1, Sec. 4).

TEST INFRASTRUCTURE ONLY. This package exists to check the CUDA path. Only
the tests, the smoke check and the CPU-baseline leg of the benchmark may
import it. The product path never calls it, and it shares no code with the
CUDA library: both sides read the same plain case dictionaries and seeded
initial fields, nothing else.

Contents
--------
scheme   grid conventions, vectorised term-wise assembly (Sec. 4, Eq. 4.3-4.4),
         pressure projection (Eq. 3.4-3.5), quadratic lever-rule update
         (Eq. 3.13-3.19) and the Algorithm 1 step.
forward  forward (equation-based, residual-probing) assembly (Sec. 4, Eq. 4.5-4.7),
         used only to cross-check the vectorised assembly.
solve    linear solves: sparse direct (SuperLU) for small systems, CG /
         BiCGSTAB for large ones.

Pins: every function here is pinned by a ``-m "not gpu"`` test in ``tests/``
against something other than itself (closed forms, the paper's Table 1,
conservation laws, forward-vs-vectorised assembly, brute-force dense solves).
The whole-step field values at the benchmark workloads have no closed form:
the paper prints no numbers for them, so beyond the invariants the step
itself is "parity unpinned" at those sizes.
"""
from .scheme import (Grid, State, initial_state, step, run, assemble_momentum, assemble_solute,
                     assemble_temperature, assemble_scalar, poisson_matrix, poisson_rhs, project,
                     lever_update, inverse_permeability, liquidus, equilibrium_fraction, thermal_walls,
                     divergence, sparse_from_planes, PLANES)
from .forward import forward_assemble
from .solve import solve_system, solve_poisson

__all__ = [
    "Grid", "State", "initial_state", "step", "run", "assemble_momentum", "assemble_solute",
    "assemble_temperature", "assemble_scalar", "poisson_matrix", "poisson_rhs", "project",
    "lever_update", "inverse_permeability", "liquidus", "equilibrium_fraction", "thermal_walls", "divergence",
    "sparse_from_planes", "PLANES", "forward_assemble", "solve_system", "solve_poisson",
]
