"""GB300-native Hubbard projector of self-consistent DFT+U (ACBN0) on a real-space grid.

The compute path is libdftu.so (CUDA, sm_103a) behind the C ABI of include/dftu.h;
paper_1711_08935_gb300.dftu is its thin Python binding.
"""
