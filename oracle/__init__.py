"""Plain FP64 CPU oracle for the multi-sphere T-matrix method (CELES, JQSRT 2017).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call or link anything in this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` use it.  It shares no code, header, table or constant
generator with the GPU path.

Every function follows the paper's definitions written out plainly, in FP64,
with NumPy / SciPy primitives (special functions, dense LU) as single steps:

* ``special``      spherical Bessel/Hankel functions, normalised associated
                   Legendre functions and the angular functions pi, tau
                   (App. A.1), exact Wigner-3j symbols (App. A.2).
* ``svwf``         spherical and plane vector wave functions (App. A.1).
* ``translation``  a5/b5 coefficients, the translation operator A and the
                   coupling matrix W (Sec. 2.2, App. A.2).
* ``mie``          the sphere T-matrix Q_{tau l} (App. B).
* ``incident``     plane-wave and Gaussian-beam initial-field coefficients
                   (App. A.2 PVWF->SVWF transform, App. C).
* ``solve``        master-equation assembly and dense LU solve (Eqs. for M and
                   the master equation, Sec. 2.2), on-the-fly matvec rows,
                   GMRES, cross sections.
* ``precond``      cuboid partition and block-diagonal LU preconditioner
                   (Sec. 3.2.1).
* ``farfield``     plane-wave amplitude g_j of the scattered field (App. D).

Coefficient order (fixed by this project; the paper does not fix one):
``n = (tau-1)*L*(L+2) + l*(l+1) - 1 + m`` (0-based), tau in {1, 2},
l = 1..L, m = -l..l.
"""

from . import special, svwf, translation, mie, incident, solve, precond, farfield  # noqa: F401
