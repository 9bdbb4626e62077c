"""Plain FP64 CPU oracle of the relativistic multigroup SHDOM step.

Test infrastructure only: the test-suite, the smoke check and the CPU-baseline
leg of the benchmark import it; the CUDA library and its binding never do.
"""
