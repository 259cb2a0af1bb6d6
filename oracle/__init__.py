"""FP64 CPU oracle of the LxW-DG time step (test infrastructure only).

Importable only by the tests, the smoke check and the benchmark's
CPU-baseline leg; the GPU library never loads it.
"""
