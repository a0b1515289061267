"""GB300-native MPMI-SC tick engine: a C-ABI CUDA library (csrc/, include/mpmi.h)
with a thin ctypes binding (mpmi.py).  Import ``paper_1906_02318_gb300.mpmi``
for the API; ``paper_1906_02318_gb300.build`` compiles the library in-tree."""
