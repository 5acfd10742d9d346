"""Plain, slow FP64 CPU oracle for Randomized Householder QR (Grigori & Timsit 2024).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs
of ``bench.py`` use it.  It shares no code, constants, tables or helpers with the
CUDA library under ``paper_2405_10923_gb300/``; the only module both sides use is
``rhqr_inputs`` (seeded input matrices, no method arithmetic).

Every routine follows one passage of the paper and cites it by section,
algorithm or equation.  The routines are written with plain numpy array
arithmetic (``+ - * / @``, slicing, ``sqrt``) so that they also run on numpy
object arrays of ``decimal.Decimal``: the tests use that to run the very same
code in 60-digit arithmetic and check the exact-arithmetic identities of
Section 3.

Modules
-------
rng      counter-based random operators (signs, row samples, Gaussian entries)
sketch   Walsh-Hadamard transform, SRHT and Gaussian sketches, RHSketch (Alg. 1)
rhqr     RHVector (Alg. 2), right/left-looking RHQR (Alg. 3/4), Q formation,
         Householder QR, recRHQR (Alg. 6), refinement passes, LU reconstruction
         (eq. lufact), RHQR-Arnoldi (Alg. 7) and RHQR-GMRES (Alg. 8)
metrics  orthogonality, residual and condition-number measures

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
except the absolute entries of Q and R for inputs whose condition number
exceeds the inverse unit roundoff (only invariants are meaningful there).
"""

from . import rng, sketch, rhqr, metrics  # noqa: F401
