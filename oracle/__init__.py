"""CPU oracle for the Monte Carlo exp(tA)v estimator — TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import, call, link or execute anything in this package.  The
product library never routes through it, and it shares no code with the CUDA
path (no kernels, headers, helpers, tables or constants); the only thing both
sides consume is the seeded input generator module ``workloads``.

Contents
--------
``dense``   deterministic FP64 references for x = exp(tA) v:
            dense scaling-and-squaring Taylor expm (Moler & Van Loan's
            method 3), the Kronecker / discrete-sine closed form for grid
            Laplacians, truncated Taylor with scaling for large sparse A,
            uniformization for CTMC generators, the Lie and Strang split
            products (Eqs. deff and eq_general1), and power iteration for
            lambda_max (Sec. 6).
``walker``  a plain C implementation of the paper's path sampler (Sec. 3,
            Eq. paths) and Algorithms 1-2 under Theorems 1-2, with the same
            counter-based Philox4x32-10 draws the library uses, compiled with
            gcc and called through ctypes.
"""
