"""Oracle: a plain, slow, FP64 CPU implementation of what the ChFSI path computes.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import or run anything in this package.  It shares no
code with the CUDA library (``paper_1305_5120_gb300``) and imports nothing from it; the
two meet only in the seeded input generator ``paper_1305_5120_gb300.synth``, which holds
none of the method's arithmetic.

Two parts:

* ``oracle.direct`` (O1): the plain definition of the result -- the nev smallest
  eigenpairs of the Hermitian-definite pencil (H, S) -- by Cholesky reduction to standard
  form, Householder tridiagonalisation and the implicit tridiagonal QR iteration (C code in
  ``tridiag.c``), with cyclic Jacobi as an independent cross-check.
* ``oracle.chfsi`` (O2): Algorithm 1 of the paper (Chebyshev filtered subspace iteration
  with locking) written step by step in the paper's order and notation.

Every function names the passage of the paper it follows.  Parity status of each function
is stated in its docstring ("pinned by ..." or "parity unpinned").
"""
