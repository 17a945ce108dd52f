"""FP64 CPU oracle for the decomposed-kernel Gaussian process.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg, never by the library. It shares no
code with the CUDA path. Every function is pinned by a CPU test against the
mathematics (Mercer convergence, Gauss-Hermite orthonormality, closed forms
and brute-force routes to the same posterior); see ``oracle/fagp.py``.
"""
from .fagp import *  # noqa: F401,F403
from . import fagp  # noqa: F401
