"""FP64 CPU oracle for the fast direct Helmholtz / Laplace / Stokes inverses.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the solver computes, written from the paper (Vitoshkin &
Gelfgat, "On direct inverse of Stokes, Helmholtz and Laplacian operators ...",
arXiv:1107.2461) in NumPy/SciPy, FP64 throughout.  Only the test-suite,
``__graft_entry__.smoke()`` and the CPU-baseline arm of ``bench.py`` may import
it.  The CUDA library never imports, links or calls anything here, and nothing
here imports the CUDA library.

Modules
  operators1d   1D finite-volume operators on a stretched grid (Sec. 3, Eq. 23;
                staggered first derivatives of Eq. 30-31)
  assembled     the assembled 3D operator I*sigma - lambda*(Dxx(+)Dyy(+)Dzz)
                (Eq. 23, 27) and its direct sparse solve -- the plain definition
  decomposition the Lynch eigenvalue decomposition solvers TPF (Eq. 25, 29) and
                TPT (Thomas in one direction, Sec. 3), done naively
  stokes        the staggered (MAC) Stokes system (Eq. 8), its direct solve, the
                three-step semi-direct inverse (Sec. 2) and BiCGstab, BiCGstab(2)
                or volume-weighted CG on the pressure matrix C (Eq. 9)
  cylindrical   the Helmholtz operator in cylindrical coordinates and its TPT
                (Eq. 44) and TPF (Eq. 45-46) inverses (Sec. 6)

Every function names the passage it follows.  Parity: every function is
pinned by a -m "not gpu" test against a closed form, an invariant, a brute-force
dense inverse or an independently assembled operator (tests/test_oracle_*.py).
"""
