"""Plain FP64 CPU oracle of the shifted-system TEM hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline arm of ``bench.py`` may import or run anything in this package.
It shares no code with the GPU library: it assembles its own Whitney-edge
matrices, builds its own source vectors and observation operator, solves the
shifted systems with its own plain up-looking sparse LDL^T (ldlt.c, under a
coordinate-bisection ordering in sparse_ldlt.py) and forms the response
and the Jacobian products straight from their definitions in the paper
(Section 2.3 eq. for u(t_j); Section 3.1 for J and J^T).

Modules
  fem       Kuhn-mesh edges, PEC mask, Whitney element matrices, K and M(sigma)
  survey    source vectors f (loop line integrals) and observation operator Q
  tem       shifted solves, residue sums, J.v, J^T.w
  rational  pole/coefficient fit of exp(-t z), its seed poles, objective and error
  inversion RT0 two-point regulariser and LSQR (Paige-Saunders)
  gn        Gauss-Newton loop (Armijo backtracking, lambda cooling) on the oracle's products
  fit_poles script writing the stored pole / residue tables (calls rational only)
  halfspace closed-form step-off dB_z/dt of a loop on a half-space
"""
