"""CPU FP64 oracle for the APFC semi-implicit amplitude step.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path (the CUDA library and its Python binding) never
imports, links or calls anything here, and this package never imports the
product.

Everything is plain numpy in float64 / complex128. Library primitives used as
steps: ``numpy.fft`` (diagonalising the periodic constant-coefficient
operators), ``numpy.linalg`` (dense solves and 2x2 eigenvalues).

Parity status per function is listed in the module docstring of
``oracle.apfc``.
"""
from .apfc import *  # noqa: F401,F403
from .adjoint import *  # noqa: F401,F403
