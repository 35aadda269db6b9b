"""Plain FP64 CPU oracle for the AMOEBA induced-dipole polarization solve.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it. It shares no code with the CUDA library; the only
common input is the seeded generator, which holds none of the arithmetic.

What it computes (the paper names the quantities and routines but prints no
formulas; the formulas come from the works it cites for AMOEBA and from the
standard Ewald / smooth-PME literature):

* the right-hand side of the polarization equation, the permanent-multipole
  field E0 (paper, Section "Hotspots": ``efld0_direct2``);
* the matrix-vector product T*mu applied at each iteration of the
  polarization solver (paper, Section "Hotspots": ``tmatxb_pme2``), as
  real-space Ewald + smooth-PME reciprocal + self terms;
* the iterative solve of (alpha^-1 - T) mu = E0 (paper, Section "Hotspots"
  and Section "Sequential performance": the solver calls the product about
  nine times per step), here preconditioned conjugate gradients;
* the polarization energy and its gradients (paper, Section "Hotspots":
  ``epolar1``);
* the permanent-multipole energy and its gradients (paper, Section
  "Hotspots": ``empole1``);
* the TCG-1 energy (one truncated conjugate-gradient step) and its exact
  gradients, and divide-and-conquer Jacobi iterations (paper, Section
  "Perspectives on Tinker-HP 1.2 performance");
* local-frame multipoles and the forces their frames add, and the
  two-field (direct / polarization scaled) solve with its energy and
  gradients (paper, Section "Polarizable AMOEBA force field").

Modules:
  ewald      screened Coulomb kernels B_n and Thole damping
  pairs      periodic / cluster pair enumeration
  realspace  real-space permanent field and dipole field (pair sums)
  pme        smooth particle-mesh Ewald for multipoles and dipoles
  ewald_exact direct lattice + k-space Ewald sums for tiny boxes
  solver     operator assembly, PCG, dense Cholesky solve
  energy     polarization energy
  forces     gradients of the polarization energy (positions, multipoles)
  multipole  permanent-multipole energy and gradients (derivative tensors)
  tcg        TCG-1 energy and gradients; d(c.E)/dx and d(a.T b)/dx
  dcji       divide-and-conquer (block) Jacobi iterations on the dense operator
  frames     local frames (Z-then-X, bisector), global moments, frame forces
  two_rhs    direct- and polarization-scaled fields, two solves, energy, gradients

Every function works in float64 numpy. Pins that tie it to the physics
(closed forms, brute force, invariants) live in ``tests/test_oracle_*.py``.
"""
from .setup import Setup  # noqa: F401
