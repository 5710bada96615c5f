"""FP64 CPU oracle for the VFISV per-pixel Milne-Eddington inversion.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, calls or links anything here; only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` do.  It
shares no code with the CUDA path: its Voigt/Faraday function is the library
Faddeeva function (``scipy.special.wofz``), its Stokes vector is the
Milne-Eddington solution obtained by solving the 4x4 propagation-matrix
system, and its Jacobian is the derivative of that inverse.  The CUDA path
uses a Weideman rational approximation and the closed-form (Cramer)
solution instead.

Modules
-------
``me``   synthesis: Zeeman pattern (Eq. 7), Voigt/Faraday functions and their
         derivatives (Eqs. 8-9), absorption matrix, Unno-Rachkovsky solution,
         filter convolution and the analytic Jacobian.
``lm``   inversion: chi-square (Eq. 1), normal equations (Eqs. 2-4, read as
         Gauss-Newton), damped SVD solve (Eqs. 5-6), epsilon rule (Table 2),
         derivatives only after a successful step (Fig. 6), covariance.
``mlp``  the initial-guess network (24 -> 256 -> 256 -> 256 -> 11, GELU):
         forward, backward, loss and Adam in FP64.
``init`` initial models from the filtergrams (Sec. 5): weak-field B,
         gamma, the azimuth from Q and U, the polarisation level, and the
         paper's combination with the network.

Parity status: every function is pinned by the tests under ``tests/``
(closed forms, brute-force quadrature, invariants, finite differences,
noise-free round trips).  The sign convention of the magneto-optical
(rho) terms is fixed by the propagation matrix used here and is checked
only for self-consistency (closed form vs 4x4 solve): parity unpinned for
that sign beyond self-consistency, as the paper does not print the matrix.
"""
from . import me, lm, mlp, init  # noqa: F401
