"""FP64 NumPy oracle of the IRLS structured-low-rank reconstruction (TEST INFRASTRUCTURE).

This package is a plain, slow, obviously-correct CPU restatement of the paper's method, written
for checking the CUDA path. Only the test-suite, the smoke check and the benchmark's CPU-baseline
leg may import it; the library in `paper_1704_04511_gb300` never does, and shares no code with it.

Modules:
  slr     -- forward model, explicit lifting, Gram, weight, sum-of-squares operator, CG, IRLS
  t2fit   -- mono-exponential T2 fitting of a recovered series (Sec. IV-A)

Parity status: every function in `slr` is pinned by a test against brute force, a closed form or a
special case (see tests/test_oracle_*.py) except the complete IRLS trajectory, which the paper gives
no worked example for: "parity unpinned" for `slr.irls` as a whole (its individual steps are
pinned). `t2fit` is pinned on noise-free mono-exponential data.
"""
