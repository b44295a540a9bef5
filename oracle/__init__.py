"""CPU oracle for the multi-source Helmholtz solve (test infrastructure).

This package is a plain, slow, FP64 (complex128) restatement of what the GPU
path computes, written from the paper (Treister & Haber, "Full waveform
inversion guided by travel time tomography", Sec. 2.1, 2.4, 4 and 5.3).  It
exists only to check the GPU path: the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library itself never
does, and it shares no code with the CUDA kernels or their host driver.

Modules
-------
``helmholtz``  operator, grid transfers, Galerkin hierarchy, damped Jacobi,
               V-cycle, dense LU and block flexible GMRES (Sec. 2.4, Sec. 4,
               Alg. "Two-grid cycle", Sec. 5.3).
``conv``       direct-summation 3x3 convolutions and their gradients for the
               learned preconditioning stage (not in the paper; checked by
               finite differences).

Parity status of each function is stated in its docstring; every function
here is pinned by a ``-m "not gpu"`` test against closed forms, brute force
or library routines (see ``tests/test_oracle_*.py``).
"""
