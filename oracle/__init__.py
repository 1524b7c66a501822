"""CPU oracle for packed small-prime-field arithmetic (test infrastructure only).

This package is a plain, slow, obviously correct CPU restatement of what the packed F_p hot
path computes, written from Dumas, Fousse and Salvy, "Simultaneous Modular Reduction and
Kronecker Substitution for Small Finite Fields".  It exists to check the CUDA library, and
nothing else may depend on it: only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run it.  It shares no code with the CUDA
path and never imports the product package.

Modules
  field   plain definitions: polynomial product, dot product and matrix product with every
          coefficient reduced by %, GF(p^k) by explicit remainder, irreducibility brute force
  dqt     Discrete Q-adic Transform (Eq. dqt), its inverse by radix conversion
          (the inverse in Algorithm 1), REDQ (Algorithm 2) and its correction matrix/tables (Sec. 3),
          right, middle-product and full (Q, Theta) compression (Sec. 7)
  fdiv    exact software floating point with a parametric mantissa, FDIV (Algorithm 3),
          AFDIV (Algorithm 4) and the rounding-mode table (Table "fdiv", Sec. 4)
  bounds  exactness bounds (Eq. bounds, Eq. delayed, Eq. lower, Eq. upper), compression
          factor e (Sec. 7.6.1) and the operation-count model (Table "mulpol")
  gfpk    Algorithm FGDP's tables built from the plain field definition (Sec. 6); the plain
          GF(p^k) dot and matrix products, the generator and the discrete-log form live in field

Parity status: every function here is pinned by tests under tests/ (paper examples,
closed forms, brute force); none is "parity unpinned".
"""
