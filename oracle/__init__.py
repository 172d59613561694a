"""CPU oracle for the LHDM nonnegative least-squares method.

TEST INFRASTRUCTURE ONLY.  Plain, slow FP64 implementations that the test
suite, the smoke check and the benchmark's CPU-baseline leg use to check and
time the CUDA path.  Nothing in the product package imports this package, and
this package imports nothing from the product package.
"""
