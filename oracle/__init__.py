"""Plain FP64 CPU oracle of the deflated block-Jacobi CG solver.

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and
by the CPU-baseline leg of the benchmark, never by the GPU library.
"""
