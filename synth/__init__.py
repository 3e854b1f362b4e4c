"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only draws random numbers and places atoms: it holds none of the
method's arithmetic (no integrals, no Fock build, no multipole parameters, no
density matrices).  Both the CPU oracle and the CUDA library receive what it
produces as plain inputs:

* ``params.synthetic_table(seed)`` -- raw per-element NDDO parameters (H, C, N,
  O) drawn inside physically sensible ranges.  No published parameter value is
  reproduced; the ranges only fix signs and orders of magnitude.
* ``geometry.*`` -- seeded molecular geometries for the five workloads.
* ``velocities.maxwell_boltzmann`` -- seeded initial velocities.
"""
from .params import synthetic_table, FIELDS, ELEMENTS, table_to_array  # noqa: F401
from .geometry import (  # noqa: F401
    c4h6, carbon_packing, carbon_fragments, organic_molecule, molecule_batch,
    serving_requests, fullerene_c60, Molecule,
)
from .velocities import maxwell_boltzmann, MASS  # noqa: F401
