"""CPU FP64 oracle for the time-parallel inexact Uzawa solver.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never calls it, and it shares no code with the
CUDA path; the only common module is ``synthetic`` (seeded inputs).

Contents
--------
``_native``   C (gcc, OpenMP) sequential implicit Euler with a banded Cholesky
              (or CG) solve per step, on uniform or given time steps, and the action
              of the time-global matrix B (§2, eq. 2.1 and 2.3).  This is the plain definition the solver must
              reproduce: the saddle-point system (eq. 2.7) has u as its second
              component, which is exactly the implicit-Euler solution.
``spacetime`` NumPy/SciPy statement of K, B, S, the DST change of basis Phi,
              mu_k, the preconditioner H and the inexact Uzawa iteration (§2-§4).
``mg``        The multigrid V-cycle reading used for the spatial solves.

Pins (tests that tie these functions to something other than themselves) live
in ``tests/test_oracle_*.py``; the printed values they use are under
``tests/golden/``.  Parity unpinned: none of the functions above.
"""
from . import _native, mg, spacetime  # noqa: F401
from ._native import apply_A, apply_B, build, implicit_euler, max_threads  # noqa: F401
