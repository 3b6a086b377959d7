"""CPU FP64 oracle for the Q1 hexahedral matrix-free operators and their Krylov solvers.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may use it.  It shares no
code with the CUDA library (``paper_2308_09839_gb300/csrc``); both sides only read the same seeded
inputs from ``paper_2308_09839_gb300.inputs``.

The oracle is the plain definition of what the method computes (Sec. 2, Eqs. 1-6; Sec. 3): build
every element matrix A^e with 2x2x2 Gauss quadrature, multiply it by the gathered element vector,
and sum the results into the global vector.  The matrix-free kernels only reorder that arithmetic,
so they must agree with it up to rounding.

Modules:
  fem      reference element, element matrices, element-wise apply, CSR assembly, load vectors and
           error norms (Eqs. 1-6, Algorithm 1, Sec. 3)
  solvers  textbook CG (the operations of Table 4), Jacobi-PCG, flexible CG, iterative refinement
  conv     plain 3D convolution forward/backward for the learned preconditioner's network
  net      the network's forward and backward composed from ``conv``
  optim    its training step: Adam (Kingma & Ba 2015) and the library's gradient-norm clip
"""
