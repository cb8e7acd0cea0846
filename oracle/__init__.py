"""FP64 CPU oracle of the Reg-FLBM D3Q27 step (test infrastructure only: the tests, the
smoke check and the benchmark's CPU-baseline leg use it; the library never does)."""
