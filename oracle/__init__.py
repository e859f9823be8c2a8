"""CPU oracle for sketched FGMRES (FGMRES wrapped around a sketched-GMRES preconditioner).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of the method, written to be checked
against the paper by eye.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference
arm may import it.  The CUDA library never imports, links or calls it, and it imports nothing from the CUDA
library; the two share only the seeded problem generators in ``workloads/``, which hold none of the method's
arithmetic.

Contents (each function cites the passage it follows):

* ``oracle.sketch``  -- the sparse-sign subspace embedding ``S`` (Eq. 1; Section 4.1 uses the Clarkson-Woodruff
  case with one nonzero per column) drawn from SplitMix64.
* ``oracle.sgmres``  -- one sketched-GMRES cycle used as the variable preconditioner (Eq. 3, Section 3:
  truncated-Arnoldi basis, sketched least squares by Gram-Schmidt QR with reorthogonalisation, stop rules C1-C3).
* ``oracle.fgmres``  -- Algorithm 1 (FGMRES, and FFOM), the FFOM residual of Eq. 4, Algorithm 2 (restarting with a
  variable preconditioner).
* ``oracle.gmres``   -- textbook GMRES used only as a pin (brute-force Krylov least squares, restarted GMRES(m)).
* ``oracle.lowprec`` -- explicit FP32 / BF16 rounding helpers for the precision-matched inner cycle.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against closed forms, brute-force dense solves,
library routines and the identities of Sections 2-3 (see those files).  No stored value in ``tests/golden`` comes
from the CUDA path.
"""
from . import sketch, sgmres, fgmres, gmres, lowprec  # noqa: F401
