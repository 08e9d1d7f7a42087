"""FP64 CPU oracle of the three-species Keldysh-lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by the
CPU-baseline leg of ``bench.py``.  The product library never imports it, and it
imports nothing from the product package.

Parity status per function is listed in ``oracle.oracle`` (module docstring).
"""
from .oracle import (  # noqa: F401
    Oracle, build_oracle, cross_section, observables_from_fields,
    slip_poiseuille_slab, slip_poiseuille_pipe,
)
