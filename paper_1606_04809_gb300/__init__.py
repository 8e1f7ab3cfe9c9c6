"""GB300-native asynchronous Sparse SAGA (ASAGA, arXiv:1606.04809).

The solver lives in a C-ABI CUDA library (``include/asaga.h``); the
``asaga`` module is its ctypes binding, ``synth`` makes seeded inputs.
Importing the package loads nothing native; ``asaga.load()`` does.
"""
