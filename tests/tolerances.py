"""Tolerances of the GPU parity tests, in one place.

* FP64 results against the FP64 oracle: 1e-12 relative (inf-norm over all components) after
  up to 1000 steps; the kernels and the oracle differ by rounding order and FMA contraction only.
* FP32 state with the Kahan-compensated update against the FP64 oracle started from the same
  FP32 values: 1e-6 relative.  The compensated update keeps the accumulation error of y at
  the level of one rounding of the increments, so what remains is the FP32 rounding of the
  slope and stage-state arithmetic (unit roundoff 6e-8 per operation) carried along the
  trajectory; measured 2e-7 for the chaotic Roessler chain after 1000 steps of dt = 0.01.
"""
FP64_TOL = 1e-12
FP32_KAHAN_TOL = 1e-6
