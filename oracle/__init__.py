"""CPU FP64 oracle for the stochastic-LapH quark-line path (test infrastructure).

This package is a plain, slow, obviously-correct restatement of what the path
computes, written from the paper (Morningstar et al., "Improved stochastic
estimation of quark propagation with Laplacian Heaviside smearing in lattice
QCD", arXiv:1104.3870).  It exists to check the CUDA library: only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  The product path never calls into it, and it shares no code with
the CUDA side (only the seeded input generators in ``synth`` feed both).

Every function cites the passage it follows.  Where the paper is silent the
reading taken is stated in the docstring.  All arithmetic is numpy complex128
(FP64); library primitives (``numpy.linalg``, ``scipy.sparse.linalg.eigsh``,
``scipy.linalg.lu_factor``) serve as single steps where a definition needs a
dense eigen- or linear solve.

Modules:
  lattice    site indexing and shifts
  gamma      Dirac matrices (chiral basis), sigma_{mu nu}
  gauge      stout smearing, clover field strength
  laplacian  3D gauge-covariant Laplacian, its lowest eigenpairs, phase rule
  noise      Philox4x32-10 counter generator and Z4 LapH noise
  dilution   time/spin/LapH dilution projectors
  dirac      anisotropic Wilson-clover matrix K, BiCGStab, dense solves
  laph       sources, sinks, meson functions and correlators (momentum, same-time lines)
  displacement  gauge-covariant displacements, displaced LapH overlaps and meson functions
  baryon     baryon functions and correlators (three-quark elementals, LapH tensor)
  wick       Wick's theorem for products of LapH bilinears (brute-force correlators)
  precond    gauge-covariant learned preconditioner (forward/backward)
"""
