"""FP64 CPU oracle for the preconditioned all-at-once solve of the regularised
time-space fractional inverse source problem (arXiv 2507.02809).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library (no kernels, headers, tables or helpers) and never imports it.

Modules
-------
coefficients  L1 weights b_m, e_m, eta (Sec. 4, Eq. 5 and the e_m definition),
              fractional centred-difference coefficients a_l (Eq. 8, Eq. 9, Lemma 1).
system        grid, problem container, dense A and P (Sec. 5, Eq. 11 and the
              preconditioner definition of Sec. 5.1), right-hand side z, structured matvec
              (Sec. 5 "Implementation"), forward substitution for P (Sec. 5.1).
gmres         restarted / unrestarted GMRES with left or right preconditioning.
adjoint       A^T lam = ybar, backward substitution for P^T, and the gradients of a misfit of
              f with respect to alpha, mu and gamma2 (from the block structure of Eq. 11).

Parity status of each function is written in its docstring; the only
"parity unpinned" item is the multi-dimensional coefficient table (the paper
says only that it is computed "through the FFT", Sec. 4 after Lemma 1), which
is pinned by invariants and an independent quadrature instead of paper values.
"""
