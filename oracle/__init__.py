"""CPU oracle for the shifted-solve path of projection MOR with reused SPAI
preconditioners (Singh & Ahuja, "Reusing Preconditioners in Projection based
Model Order Reduction Algorithms").

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check
and the CPU-baseline leg of the benchmark may import it.  The CUDA library
never calls it, and it shares no code with the CUDA library: it is a plain,
slow, FP64 restatement of what the paper defines, written so that a reader can
check each function against the paper by eye.

Modules
  operator  -- the shifted operator sigma E - A (and the second-order
               sigma^2 M + sigma D + K), transfer functions          (Sec. II)
  spai      -- SPAI columns, the reuse update Q, the preconditioner chain
                                                   (Sec. III.A-C, Table II)
  krylov    -- right-preconditioned BiCGSTAB and GMRES(m), dense LU
                                                         (Sec. III.A, IV)
  irka      -- Gram-Schmidt, Petrov-Galerkin projection, reduced poles,
               IRKA (Algorithm 2 with N_j = 0) with the reuse schedule of
               Algorithm 4 mapped onto IRKA shifts x iterations

Parity status of every function is stated in its docstring; all are pinned
by tests in tests/test_oracle_*.py except where the docstring says
"parity unpinned".
"""
from . import operator, spai, krylov, irka  # noqa: F401
