"""FP64 CPU oracle for the local-smoothing geometric multigrid method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the smoke check and the bench's CPU
baseline leg use it.  It is a plain, slow, readable restatement of the method
of Clevenger, Heister, Kanschat and Kronbichler (ACM TOMS 2021, arXiv
1904.03317) with assembled sparse matrices:

* ``mesh``  -- forest of a Cartesian brick, isotropic refinement, and the
  vertex 2:1 closure (Sec. 2.3, Sec. 3.5: leaves sharing a degree of freedom
  differ by at most one level), computed by a plain fixed-point iteration.
* ``fem``   -- Q_k Lagrange elements (Sec. 2.1), element matrices by
  Gauss-Legendre quadrature, hanging-node elimination on the leaf mesh
  (Sec. 1), level spaces V_l = V_l^S + V_l^I on the cells of level l
  (Sec. 2.3, Fig. 1), transfer by embedding with R = P^T (Sec. 2.2).
* ``gmg``   -- Chebyshev-Jacobi smoother (Sec. 4.1), eigenvalue estimate by
  10 CG steps from the (-5.5 .. 5.5) pattern (Sec. 4.1), the V-cycle of
  Algorithm 2 in local-smoothing form (Sec. 2.3), dense Cholesky coarse solve,
  and the outer preconditioned CG.

Parity status of each function is stated in its docstring; every function is
pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` except
where a docstring says "parity unpinned".
"""
