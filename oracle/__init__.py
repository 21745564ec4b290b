"""Plain FP64 CPU oracle of the D2Q37 time step: test infrastructure only.

Only tests/, the package smoke check and the benchmark's CPU-baseline leg may import it.
"""
