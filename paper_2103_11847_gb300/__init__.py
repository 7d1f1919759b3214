"""GB300 (sm_103a) library for the cosine-product Krylov solvers of arXiv 2103.11847.

The compute path lives in the C-ABI shared library built from ``csrc/`` (see
``include/tcprod.h``); ``tcprod`` is its thin ctypes binding. Importing this
package does not load the library; ``tcprod.lib()`` does, and fails loudly if
it has not been built.
"""
