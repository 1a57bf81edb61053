"""Plain, slow FP64 CPU oracle for the Lippmann-Schwinger Nystrom hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from this
package.  It shares no code with the CUDA library (``paper_2608_17615_b300``);
the two meet only through the seeded inputs of ``lsinput``.

Every function follows a passage of the paper (arXiv 2608.17615, "Fast
high-order solvers for the Lippmann-Schwinger equation in piecewise-smooth
heterogeneous media") or a textbook definition, cited in its docstring:

* ``bessel``   J0, J1, Y0, Y1, H0^(1), H1^(1) from textbook series/expansions
* ``nystrom``  naive Nystrom pair sum (Eq. linear_system without correction)
* ``vdim``     VDIM near/self correction (Eq. DIM_decomp, local-patch reading)
* ``operator`` L = I + k^2 V M (Eq. linear_system_matrix) and its transpose
* ``precond``  Cartesian grid, transfer operators (Approach II), sparsifying
               preconditioner, P = I + T_C^Q (S - I) T_Q^C (Eq. preconditioner_factored)
* ``gmres``    left-preconditioned unrestarted GMRES (modified Gram-Schmidt)
* ``farfield`` far-field pattern and the Mie series of a constant disk

Parity pins (tests/test_oracle_*.py) tie each function to something other
than itself: scipy, closed forms, brute-force quadrature, the Mie series,
invariants stated in the paper.  Functions without such a pin say
"parity unpinned" in their docstring.
"""
