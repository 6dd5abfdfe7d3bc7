"""FP64 CPU oracle for the TensorNet energy-and-force path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
the benchmark's CPU-baseline / reference leg may import this package.  The
product path (the C-ABI library and its Python binding) never calls it and
fails loudly when its CUDA extension is missing.

Modules:
  neighbors  brute-force O(N^2) minimum-image pair search (Sec. 2.5.1)
  tensornet  TensorNet forward and an analytic reverse pass (forces and
             weight gradients) in float64, written with full 3x3 matrices

Parity status of each function is stated in its module header.
"""
