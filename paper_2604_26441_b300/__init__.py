"""B300-native (sm_103a) matrix-free Galerkin geometric-multigrid PCG solver for
frozen-density 3D SIMP elasticity on structured hex8 grids.

``paper_2604_26441_b300.gmg`` is the binding of the C ABI (include/gmg.h);
``paper_2604_26441_b300.inputs`` builds the seeded synthetic workloads;
``paper_2604_26441_b300.build`` compiles the CUDA library in-tree.  Importing
the package itself loads nothing.
"""
