"""GB300-native multi-sphere T-matrix solver (the hot path of CELES, JQSRT 2017).

The compute lives in ``_lib/libceles_gb300.so`` (CUDA, sm_103a) behind the C
ABI of ``include/celes.h``; ``binding`` mirrors that ABI function by function
(argument marshalling only) and ``Simulation`` is a small convenience wrapper
that owns one context.
"""

from . import binding  # noqa: F401
from .binding import (CELES_FP32, CELES_FP64, CELES_SOLVE_FP64, CELES_SOLVE_MIXED, CELES_X0_TA,  # noqa: F401
                      CELES_X0_USER, CELES_X0_ZERO, CelesError, make_incident)


class Simulation:
    """One scattering problem on one GPU (owns a celes context).

    positions (N, 3), radii (N,), n_sphere (N,) complex refractive indices,
    n0 background index, wavelength (vacuum, same length unit), lmax.
    """

    def __init__(self, positions, radii, n_sphere, n0, wavelength, lmax, device=0, check_overlap=True, chunks=0):
        import numpy as np
        self.k0 = 2.0 * np.pi / wavelength
        self.ctx = binding.celes_create(positions, radii, n_sphere, n0, self.k0, lmax, device=device,
                                        check_overlap=check_overlap, chunks=chunks)
        self.lmax = lmax
        self.N = binding.celes_num_spheres(self.ctx)
        self.nmax = binding.celes_nmax(self.ctx)

    @classmethod
    def from_scene(cls, scene, **kw):
        return cls(scene.positions, scene.radii, scene.n_sphere, scene.n0, scene.wavelength, scene.lmax, **kw)

    def set_incident(self, incidents):
        descs = []
        for inc in incidents:
            if hasattr(inc, "kind"):
                descs.append(make_incident(inc.kind, inc.beta, inc.alpha, inc.pol, inc.E0, inc.waist, inc.focus,
                                           inc.alpha_G))
            else:
                descs.append(inc)
        binding.celes_set_incident(self.ctx, descs)

    def solve(self, tol=1e-6, **kw):
        return binding.celes_solve(self.ctx, tol, **kw)

    def coefficients(self):
        return binding.celes_get_coefficients(self.ctx)

    def incident_coefficients(self):
        return binding.celes_get_incident_coefficients(self.ctx)

    def tmatrix(self):
        return binding.celes_get_tmatrix(self.ctx)

    def farfield(self, dirs, rhs=0):
        return binding.celes_farfield(self.ctx, dirs, rhs)

    def precond_build(self, edge):
        binding.celes_precond_build(self.ctx, edge)

    def close(self):
        if self.ctx:
            binding.celes_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
