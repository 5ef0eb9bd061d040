"""CPU FP64 oracle for KLE-PCGC (arXiv 2510.26180).  TEST INFRASTRUCTURE ONLY.

This package is the slow, plain, obviously-correct reference that the CUDA
path is checked against.  It is not part of the product: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with
``paper_2510_26180_gb300`` (neither imports the other); the only common input
is the seeded xi draws of the ``synth`` package.

Modules
  kl_input    exponential-covariance KL of the input field (1D and separable 2D)
  gpc         total-degree Hermite gPC basis (Section 2.2, eq. complete)
  heat1d      1D finite-difference operator and backward-Euler propagators
  pcgc        Algorithms 1 and 2: parareal with sequential and with
              diagonalized (alpha-circulant) coarse grid correction
  surrogate   Algorithm 3 offline part: snapshot KL + gPC least squares
  contraction convergence factors K_cla(z,J), K(z,J,alpha) (Theorem linearthm)
  klecgc      end-to-end driver: setup + batch solve, plus error metrics

Readings of passages where the paper is silent or garbled are listed at the
top of each module that takes them.  Parity status: every function is pinned
by ``tests/test_oracle_*.py`` except where a module header says
"parity unpinned".
"""
