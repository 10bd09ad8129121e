"""CPU FP64 oracle for the DFT+U (ACBN0) Hubbard projector -- test infrastructure only.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark use this package.
It shares no code with the GPU library and never imports it.
"""
