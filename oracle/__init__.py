"""FP64 CPU oracle for SOCS aerial imaging, the Gaussian resist and the ILT gradient.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or
executes anything in this package: only the tests, `__graft_entry__.smoke()`
and the CPU-baseline leg of `bench.py` use it.  It shares no code with the CUDA
library (which has its own optics builder, FFTs and eigensolver); the two
meet only through the seeded inputs of `synth`.

Everything is plain numpy in float64 (complex128), written to be checked by
eye against the paper's equations:

* `optics`  - source sampling, pupil, band crop, Eq. (2) TCC and its Eq. (3)
  eigen-decomposition (numpy's Hermitian eigensolver as a library step).
* `imaging` - mask spectrum, Abbe imaging (Eq. (1) with Eq. (2) substituted),
  SOCS imaging from given kernels (Eq. (4)), row-sampled SOCS for large clips.
* `resist`  - periodic Gaussian resist blur and threshold (Eq. (5)), contour
  crossings used for the edge-placement difference.
* `ilt`     - the ILT loss over focus planes and its adjoint gradient,
  plus central finite differences.
* `ai`      - the AI initialiser's input channels (Eq. (9)) and the
  print-consistency images and loss (Eqs. (15)-(17)).
* `raster`  - exact area coverage of rectangle masks (the grey-level m of
  Eq. (1) for shapes that do not fall on pixel boundaries).
* `contour` - marching-squares contours of the resist image (section II.D)
  and the edge-placement error at control points with its through-focus
  average and effective value (Eqs. (6)-(8)).

Parity status: every function here is pinned by tests under `tests/` against
closed forms, brute-force direct DFTs on 16x16 grids, invariants and finite
differences (see `tests/test_oracle_*.py`).  The paper prints no worked
numerical example, so no pin comes from a printed value.
"""
