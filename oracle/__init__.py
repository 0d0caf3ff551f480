"""CPU FP64 oracle for the NEDNER-NUFFT planar photoacoustic reconstruction.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or constant generator with the CUDA library.

Modules
  window  Kaiser-Bessel window and its analytic Fourier transform (Sec. 3).
  ndft    O1: the discrete reconstruction formula eq:disc_rec evaluated
          directly, its exact transpose and its sensor-position gradient.
  nufft   O2: the NEDNER-NUFFT algorithm in the paper's order (NED, NER,
          inverse FFT; Sec. 3), in FP64 with a wide window, and its transpose.
  metrics the appendix's quality measures: correlation coefficient and the
          normalised Tenenbaum (Sobel) sharpness.
  voronoi detector weights as periodic Voronoi cell sizes and their gradient.

Parity status: every function here is pinned by tests under
``tests/test_oracle_pins.py`` (closed forms, lattice special cases, integer
frequency special cases, exact invariants, dot-product and finite-difference
checks); nothing is "parity unpinned" except the absolute amplitude of the
uniform-ball physics check, which limited view makes only loosely determined.
"""
from . import window, ndft, nufft, metrics, voronoi  # noqa: F401
