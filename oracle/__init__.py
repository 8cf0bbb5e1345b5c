"""FP64 CPU oracle of the Liouville-Lanczos method (test infrastructure only).

This package is the reference the CUDA path is checked against.  It is plain NumPy/SciPy
in float64/complex128: full-grid FFTs, explicit loops over k-points and bands, LAPACK for
the tridiagonal solve.  It shares no code with the CUDA path; the only thing both consume
is the ground-state bundle written by the seeded input generator in `workloads/`.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import
it.  The product path never calls it.

Modules
  basis       G-sphere <-> FFT-grid maps, the k -> k+Q intersection map    (Sec. 2.3)
  xc          Slater + Perdew-Zunger 1981 LDA: e_xc, v_xc, f_xc           (Sec. 5; Eq. 12)
  liouvillian D, K, P_c, response density, Hartree+XC response            (Eqs. 12-13, 16, 24-28)
  lanczos     pseudo-Hermitian and non-Hermitian recursions               (Sec. 2.5)
  spectrum    (omega - T) x = e_1, chi = (z, x), eps^-1, eps              (Eqs. 5, 30-33)
  casida      brute-force diagonalisation of the full Liouvillian         (pin)
"""
