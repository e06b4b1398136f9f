"""GB300-native Adaptive Banded Event Alignment (ABEA).

The alignment runs in hand-written CUDA kernels behind the C ABI declared in
include/abea.h; `binding` is the Python marshalling layer over that library.
Importing the package loads nothing; `binding.load()` opens the library.
"""
