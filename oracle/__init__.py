"""Plain FP64 CPU oracle for the unfitted DG (SIPG + Nitsche + face ghost penalty) Poisson operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``
may use it.  It shares no code with the CUDA library (``paper_2404_07911_gb300``) and does not
import it.

What it computes (paper: arXiv 2404.07911):
  * ``basis``    1D Gauss-Legendre rules, Gauss-Lobatto nodes, Lagrange polynomials and their
                 derivatives of every order (Sec. 3.2, tensor-product shape functions).
  * ``mesh``     Cartesian background grid, inside / cut / outside classification against a
                 sphere level set, lexicographic numbering of active cells, interior face typing
                 (Sec. 2.3, quadrature classification).
  * ``saye``     dimension-reduction quadrature (the method of Saye 2015 that Sec. 1 and Sec. 2.3
                 use for cut cells and cut faces), restated for sphere level sets with closed-form
                 roots.
  * ``forms``    the bilinear forms of Eq. bilinear_cg (CG + Nitsche) and Eq. bilinear_dg (SIPG), Sec. 2.1, plus the
                 face-based ghost penalty on normal-derivative jumps of orders 1..J, assembled by
                 brute-force quadrature with the naive full-basis evaluation of Eq. naive_evaluation (Sec. 3.2) (no sum
                 factorisation), and applied as y = A x.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
library routines, paper-printed DoF counts or brute force, except the exact placement of the
dimension-reduction quadrature points, whose *integrals* are pinned but whose point positions are
"parity unpinned" (no independent source fixes them).
"""
