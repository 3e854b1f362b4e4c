"""FP64 CPU oracle of the KSA-XL-BOMD per-step electronic update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code, header, table or constant with it; both
receive the same seeded inputs from ``synth``.

The oracle follows the paper (arXiv 2303.00689, "Semi-Empirical Shadow
Molecular Dynamics: A PyTorch implementation") in its own notation:

* ``nddo``        -- NDDO (MNDO/AM1 form) pair integrals, overlaps, core-core
                     terms and their derivatives (the paper cites these
                     Hamiltonians in the Introduction and states NDDO => S = I
                     under eq. 6; the formulas themselves are not printed).
* ``hamiltonian`` -- h, F = h + G(P) (eqs. 3, 6, 17), shadow energy (eq. 13)
                     and forces (eqs. 22, 37-41).
* ``electronic``  -- eigendecomposition, Fermi occupations and mu (eqs. 7, 8,
                     19), entropy (eq. 4), canonical DMPT (eq. 36), Krylov
                     kernel (eqs. 31-35).
* ``dynamics``    -- SCF start (Results, "SCF Optimization"), modified Verlet
                     with damping (eqs. 27-30, 35), constant of motion (eq. 26).

Parity status of each function is stated in its module header.  Parity with
PySeQM/MOPAC numbers is unpinned: the paper prints no worked example and the
parameter tables are synthetic.
"""
