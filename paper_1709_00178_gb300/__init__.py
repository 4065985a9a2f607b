"""GB300-native PYRIT erasure codec (polynomial ring transform coding over GF(2^w)).

The compute path lives in the CUDA library ``csrc/`` builds (``libpyrit.so``) behind the C ABI
declared in ``include/pyrit.h``; ``pyrit`` is its thin ctypes binding. Importing this package
loads nothing: ``from paper_1709_00178_gb300 import pyrit`` loads the library and fails loudly
if it has not been built.
"""
