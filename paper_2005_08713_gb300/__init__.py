"""GB300-native codec of Hulsken, "Fast Compression Method for Medical Images on the Web" (2020).

The compute path is the CUDA library in ``csrc/`` behind the C ABI of
``include/isx.h``; ``isx`` is its thin ctypes binding.  ``synth`` holds the
seeded input generators.  Importing the package loads nothing.
"""
