"""Plain FP64 CPU oracle for the PGD-TO optimizer step (arXiv 2511.13905).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its CPU-baseline leg and ``--impl reference`` arm) may import it.
The CUDA library never calls it, and it imports nothing from the CUDA path.

Every function here is written to be read against the paper, not to be fast:
NumPy FP64 vector operations and, for tiny inputs, plain Python loops.

Notation (paper -> code):
  rho_t -> x,  rho_tilde -> z,  grad g_j(rho_t) -> row a_j of A (m x n),
  paper dual y <= 0 -> lam = -y >= 0,  l, u -> lo, hi,
  b_j = G_j - g_j(rho_t) + a_j^T rho_t  (linearisation about rho_t, Sec. 3.2, eq. linearized).

With that notation the regularised projection (Sec. 3.2.3 / App. A.3, eq. h and
eq. reg_jacobian) is the unique solution of

    min_x ||x - z||^2 + (C/2)||s||^2   s.t.  lo <= x <= hi,  A x - s <= b,  s >= 0,

whose dual form is  x(lam) = clip(z - A^T lam, lo, hi),
r_j(lam) = a_j^T x(lam) - b_j - 2 lam_j / C,  lam >= 0,  r <= 0,  lam_j r_j = 0.

Modules:
  projection  -- solution form, residual, exact solvers, Alg. 1, Alg. 2
  bruteforce  -- KKT active-pattern enumeration for tiny n (a pin, not a solver)
  checks      -- KKT residuals and tolerance metrics used by the parity tests
  step        -- one iteration of Alg. 3 (step size, PR+ direction, projection)

Functions whose result no independent pin fixes say "parity unpinned" in their
docstring; at present there are none.
"""

from .projection import (  # noqa: F401
    primal_from_dual,
    residual,
    jacobian_h,
    phi,
    solve_single_exact,
    solve_single_bisect,
    solve_independent_exact,
    solve_independent_bisect,
    solve_coupled_exact,
    alg2_general_projection,
)
from .bruteforce import project_bruteforce  # noqa: F401
from .checks import kkt_report, parity_errors  # noqa: F401
from .step import step_scalars, oracle_step, StepParams  # noqa: F401
