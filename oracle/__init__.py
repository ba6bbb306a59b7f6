"""CPU oracle for the LGF fast multipole method (Liska & Colonius, "A parallel
fast multipole method for elliptic difference equations").

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link
or execute anything in this package: only the tests, the smoke check and the
benchmark's CPU-baseline leg use it.  It shares no code with the CUDA library
(no kernels, headers, tables or helpers); the only code both sides use is the
seeded input generator module ``workloads``.

Contents
  lgf.py     the lattice Green's function G(n) of the 7-point Laplacian from the
             1D Bessel-integral form (App. A, Eq. lgf3), FP64
  direct.py  + direct.c: the exact O(N^2) sum u = G * f (Eq. dpoissonsoln), C/OpenMP
  fmm.py     the FLGF method step by step (Sec. 3.1, Steps 0-3), NumPy FP64
  select.py  the two-step choice of n_max and the interval size for a target
             error (Sec. 2.5), NumPy FP64

Parity status of each function is stated in its module header.
"""
