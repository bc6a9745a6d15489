"""FP64 CPU oracle of the GMG-preconditioned CG solver -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously correct restatement of what the
CUDA path computes, written from the paper ("A Matrix-Free Galerkin Multigrid
Solver and Failure-Mode Screen for Single-GPU 3D SIMP Linear Systems").  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` may import it.  The product library never calls it, links
it, or falls back to it; it shares no code, table or helper with the CUDA
sources.  Random inputs come from ``paper_2604_26441_b300.inputs``, which holds
none of the method's arithmetic.

Modules:

* ``fem``       -- hex8 element stiffness, grid numbering, SIMP moduli, global
                   assembly and the element-sum (matrix-free) operator;
* ``hierarchy`` -- 2:1 trilinear transfer operators, Dirichlet inheritance by
                   injection, Galerkin coarse operators (explicit sparse triple
                   products and the element-wise level-1 formula), diagonals,
                   power iteration and the regularised coarsest Cholesky;
* ``solver``    -- damped Jacobi, Chebyshev-Jacobi, the V-cycle and PCG with
                   true-residual acceptance.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
brute force on tiny inputs, library routines for special cases, or values the
paper prints.  Functions without such a pin say "parity unpinned" in their
docstring.
"""
