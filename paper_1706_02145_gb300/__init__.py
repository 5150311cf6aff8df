"""GB300-native multi-sphere T-matrix solver (the hot path of CELES, JQSRT 2017).

The compute lives in ``_lib/libceles_gb300.so`` (CUDA, sm_103a) behind the C
ABI of ``include/celes.h``; ``binding`` mirrors that ABI function by function
(argument marshalling only).  The classes below own library handles:

* ``Simulation``: one sphere cluster (positions and radii in nm, complex
  refractive indices, vacuum wavelength, lmax) with its incident fields,
  solve of (I - T W) b = T a_in, and the derived quantities.
* ``BatchSolver``: every RHS of several Simulations (any lmax and size) in one
  lockstep solve on the GPU.
* ``LearnedGuess``: the graph network that predicts a first iterate.

Typical use::

    import paper_1706_02145_gb300 as celes
    sim = celes.Simulation(positions, radii, n_sphere, 1.0, 550.0, lmax=4)
    sim.set_incident([celes.make_incident("gaussian", waist=2000.0)])
    sim.precond_build(900.0)                 # optional block preconditioner
    info = sim.solve(1e-6)                   # FP32 GMRES, FP64 refinement
    b = sim.coefficients()                   # [rhs][sphere][n] complex
    g = sim.farfield(dirs)                   # (beta, alpha) directions
    E = sim.nearfield(points)                # NaN inside spheres
    sim.close()

Every call runs on the GPU; there is no CPU fallback, and a missing or
unloadable library raises.
"""

from . import binding  # noqa: F401
from .binding import (CELES_FP32, CELES_FP64, CELES_SOLVE_FP64, CELES_SOLVE_MIXED, CELES_SOLVER_BICGSTAB,  # noqa: F401
                      CELES_SOLVER_GMRES, CELES_X0_LEARNED, CELES_X0_TA, CELES_X0_USER, CELES_X0_ZERO, CelesError,
                      make_incident)


class Simulation:
    """One scattering problem on one GPU (owns a celes context).

    positions (N, 3), radii (N,), n_sphere (N,) complex refractive indices,
    n0 background index, wavelength (vacuum, same length unit), lmax.
    autotune / variant: the coupling kernel's launch shape (celes_options);
    autotune=False gives bit-reproducible FP32 products.
    """

    def __init__(self, positions, radii, n_sphere, n0, wavelength, lmax, device=0, check_overlap=True, chunks=0,
                 autotune=True, variant=-1):
        import numpy as np
        self.k0 = 2.0 * np.pi / wavelength
        self.ctx = binding.celes_create(positions, radii, n_sphere, n0, self.k0, lmax, device=device,
                                        check_overlap=check_overlap, chunks=chunks, autotune=autotune,
                                        variant=variant)
        self.lmax = lmax
        self.N = binding.celes_num_spheres(self.ctx)
        self.nmax = binding.celes_nmax(self.ctx)

    @classmethod
    def from_scene(cls, scene, **kw):
        return cls(scene.positions, scene.radii, scene.n_sphere, scene.n0, scene.wavelength, scene.lmax, **kw)

    def set_incident(self, incidents, n_beta=0):
        """incidents: synth.Incident-like objects or binding.make_incident descriptors."""
        descs = []
        for inc in incidents:
            if hasattr(inc, "kind"):
                descs.append(make_incident(inc.kind, inc.beta, inc.alpha, inc.pol, inc.E0, inc.waist, inc.focus,
                                           inc.alpha_G, n_beta))
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

    def nearfield(self, points, rhs=0, what=2):
        """E at points (Np, 3): what 0 scattered, 1 incident, 2 total (NaN inside spheres)."""
        return binding.celes_nearfield(self.ctx, points, rhs, what)

    def power(self, rhs=0, n_beta=128, n_alpha=128):
        """(R, T) reflected and transmitted power fractions of a Gaussian-beam RHS."""
        return binding.celes_power(self.ctx, rhs, n_beta, n_alpha)

    def s11(self, betas, rhs_a=0, rhs_b=1, n_alpha=64):
        """Unnormalised S11 at polar angles betas (TE/TM average of the azimuthal mean intensity)."""
        return binding.celes_s11(self.ctx, betas, rhs_a, rhs_b, n_alpha)

    def predict_guess(self, gnn):
        """Store a LearnedGuess network's first iterate for solve(x0=CELES_X0_LEARNED)."""
        binding.celes_gnn_predict(gnn.g, self.ctx)

    def close(self):
        if self.ctx:
            binding.celes_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Lockstep solve of every RHS of several Simulations (any lmax and size) on one GPU."""

    def __init__(self, simulations, restart=30):
        self.sims = list(simulations)
        self.b = binding.celes_batch_create([s.ctx for s in self.sims], restart=restart)

    def solve(self, tol=1e-6, mode=CELES_SOLVE_MIXED, restart=30, **kw):
        """Returns (status, per-simulation info dicts); coefficients land in each Simulation."""
        return binding.celes_batch_solve(self.b, len(self.sims), tol, mode=mode, restart=restart, **kw)

    def close(self):
        if self.b:
            binding.celes_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LearnedGuess:
    """Graph-network first iterate (16-NN message passing on the tcgen05 BF16 GEMM)."""

    def __init__(self, lmax, width=128, layers=3, seed=0, device=0):
        self.g = binding.celes_gnn_create(lmax, width=width, layers=layers, seed=seed, device=device)

    def train(self, sim, steps=1, lr=1e-3, rhs=0):
        """Adam steps on one solved Simulation; returns the loss."""
        return binding.celes_gnn_train(self.g, sim.ctx, rhs=rhs, steps=steps, lr=lr)

    def close(self):
        if self.g:
            binding.celes_gnn_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
