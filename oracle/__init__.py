"""FP64 CPU oracle for LR-spline volume ray casting.

Test infrastructure only: the test suite, the smoke check and the benchmark's
CPU-baseline leg may use it; the CUDA library never does.
"""
