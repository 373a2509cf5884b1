"""FP64 CPU oracle of AccAltProj.  TEST INFRASTRUCTURE: only the tests, the smoke check and
the CPU-baseline leg of the benchmark may import this package; the CUDA library never does."""
