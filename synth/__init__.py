"""Seeded synthetic sphere packings and illumination settings.

This module is shared by the tests, the benchmark, the oracle checks and the
CUDA path.  It produces INPUTS only (sphere centres, radii, refractive
indices, wavelength, truncation degree and incident-field parameters); it holds
none of the scattering method's arithmetic.

Lengths are in nanometres.  Seeds follow ``seed = 1000 * config + index`` with
NumPy's PCG64 generator.

Workload shapes (all "synthetic stand-ins" for the paper's Lubachevsky-
Stillinger and MSTM packings, which are not available here):

* ``config1``  50 spheres, R = 100 nm, n = 1.52, lambda = 550 nm, lmax = 3, in a
  cube at fill 0.2 (uniform centres, rejection of overlaps), x-polarised plane
  wave along +z.
* ``config2``  N spheres (default 10 000), lognormal radii (E[R] = 150 nm,
  sigma of ln R = 0.1), n = 1.5 + 0.001i, lambda = 550 nm, lmax = 4, random
  sequential addition in a cylindrical slab of thickness 2 um at fill 0.3 (the
  cylinder radius follows from N and the fill), Gaussian beam w = 2 um focused
  at the centre of the illuminated (z = z_min) face, x-polarised.
* ``config3``  ensemble ``index`` of 64: N ~ U[200, 3000], lmax ~ U{2..5},
  lambda ~ U[400, 800] nm, R ~ U[80, 200] nm (one radius per ensemble), real
  n ~ U[1.45, 2.0], fill ~ U[0.1, 0.35] in a cube (FCC lattice plus hard-
  sphere Monte Carlo above 0.3), 8 plane waves with directions on a Fibonacci
  lattice of the cap beta <= 60 deg, polarisation 2.
* ``config5``  N spheres (default 100 000), R = 130 nm, n = 1.52, lambda =
  550 nm, lmax = 3, slab of thickness 4 um at fill 0.25 (square footprint from
  N and the fill), Gaussian beam w = 5 um.
"""

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Incident:
    kind: str                 # "plane" or "gaussian"
    beta: float = 0.0         # plane wave: polar angle of k
    alpha: float = 0.0        # plane wave: azimuth of k
    pol: int = 2              # plane wave: 1 = TE (e_alpha), 2 = TM (e_beta)
    waist: float = 0.0        # gaussian: beam waist w
    focus: tuple = (0.0, 0.0, 0.0)
    alpha_G: float = -np.pi / 2   # gaussian: E0 = -sin(aG) e_x + cos(aG) e_y
    E0: float = 1.0


@dataclass
class Scene:
    positions: np.ndarray     # (N, 3) float64, nm
    radii: np.ndarray         # (N,) float64, nm
    n_sphere: np.ndarray      # (N,) complex128 refractive index of each sphere
    n0: float                 # background refractive index
    wavelength: float         # vacuum wavelength, nm
    lmax: int
    incidents: List[Incident] = field(default_factory=list)
    name: str = ""

    @property
    def N(self):
        return self.positions.shape[0]

    @property
    def k0(self):
        return 2.0 * np.pi / self.wavelength

    @property
    def k(self):
        return self.n0 * self.k0

    @property
    def n_rel(self):
        return self.n_sphere / self.n0

    @property
    def nmax(self):
        return 2 * self.lmax * (self.lmax + 2)


def rng_for(config: int, index: int = 0):
    return np.random.Generator(np.random.PCG64(1000 * config + index))


# ----------------------------------------------------------------------------
# packings
# ----------------------------------------------------------------------------

class _Grid:
    """Uniform cell grid for overlap queries during sequential addition."""

    def __init__(self, lo, hi, cell):
        self.lo = np.asarray(lo, float)
        self.cell = float(cell)
        self.shape = np.maximum(1, np.ceil((np.asarray(hi, float) - self.lo) / cell).astype(int))
        self.cells = {}

    def key(self, p):
        c = np.floor((p - self.lo) / self.cell).astype(int)
        return tuple(np.clip(c, 0, self.shape - 1))

    def neighbours(self, p):
        cx, cy, cz = self.key(p)
        out = []
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    out.extend(self.cells.get((cx + dx, cy + dy, cz + dz), ()))
        return out

    def add(self, p, idx):
        self.cells.setdefault(self.key(p), []).append(idx)


def random_sequential_addition(rng, radii, sampler, lo, hi, gap=1e-3, max_tries=2_000_000):
    """Place spheres of the given radii one by one at positions drawn by
    ``sampler(rng, R, m)`` (m candidates at a time), rejecting overlaps
    (|r_i - r_j| < R_i + R_j + gap)."""
    radii = np.asarray(radii, float)
    N = radii.size
    pos = np.zeros((N, 3))
    grid = _Grid(lo, hi, 2.0 * radii.max() + gap)
    tries = 0
    for i in range(N):
        R = radii[i]
        placed = False
        while not placed:
            cand = sampler(rng, R, 64)
            for c in cand:
                tries += 1
                if tries > max_tries:
                    raise RuntimeError("random sequential addition did not converge (fill too high?)")
                nb = grid.neighbours(c)
                if nb:
                    q = pos[nb]
                    dd = np.sum((q - c) ** 2, axis=1)
                    lim = (radii[nb] + R + gap) ** 2
                    if np.any(dd < lim):
                        continue
                pos[i] = c
                grid.add(c, i)
                placed = True
                break
    return pos


def config1(seed_index: int = 0, N: int = 50) -> Scene:
    rng = rng_for(1, seed_index)
    R = 100.0
    side = (N * 4.0 / 3.0 * np.pi * R ** 3 / 0.2) ** (1.0 / 3.0)
    radii = np.full(N, R)

    def sampler(rng, r, m):
        return rng.uniform(r, side - r, size=(m, 3))

    pos = random_sequential_addition(rng, radii, sampler, (0, 0, 0), (side, side, side), gap=0.0)
    return Scene(pos, radii, np.full(N, 1.52 + 0j), 1.0, 550.0, 3,
                 [Incident("plane", beta=0.0, alpha=0.0, pol=2)], name=f"plane-wave cube N={N} L=3")


def lognormal_radii(rng, N, mean=150.0, sigma=0.1):
    mu = np.log(mean) - sigma ** 2 / 2.0
    return np.exp(rng.normal(mu, sigma, size=N))


def config2(seed_index: int = 0, N: int = 10_000, lmax: int = 4) -> Scene:
    rng = rng_for(2, seed_index)
    radii = lognormal_radii(rng, N)
    # largest first packs more easily; the order is then shuffled
    order = np.argsort(-radii)
    radii = radii[order]
    thick = 2000.0
    vol = np.sum(4.0 / 3.0 * np.pi * radii ** 3)
    rc = np.sqrt(vol / 0.3 / (np.pi * thick))

    def sampler(rng, r, m):
        rr = (rc - r) * np.sqrt(rng.uniform(0, 1, m))
        ph = rng.uniform(0, 2 * np.pi, m)
        z = rng.uniform(r, thick - r, m)
        return np.stack([rr * np.cos(ph), rr * np.sin(ph), z], axis=1)

    pos = random_sequential_addition(rng, radii, sampler, (-rc, -rc, 0.0), (rc, rc, thick))
    perm = rng.permutation(N)
    pos, radii = pos[perm], radii[perm]
    inc = Incident("gaussian", waist=2000.0, focus=(0.0, 0.0, 0.0), alpha_G=-np.pi / 2)
    return Scene(pos, radii, np.full(N, 1.5 + 0.001j), 1.0, 550.0, lmax, [inc],
                 name=f"polydisperse cylinder slab N={N} L={lmax} Gaussian w=2um")


def fibonacci_cap(n, beta_max):
    """n directions (beta, alpha) on a Fibonacci lattice of the cap beta <= beta_max."""
    golden = np.pi * (3.0 - np.sqrt(5.0))
    i = np.arange(n) + 0.5
    cosb = 1.0 - i / n * (1.0 - np.cos(beta_max))
    return np.arccos(cosb), np.mod(golden * i, 2 * np.pi)


def _config3_draw(rng):
    N_ = int(rng.integers(200, 3001))
    L_ = int(rng.integers(2, 6))
    lam = float(rng.uniform(400.0, 800.0))
    R = float(rng.uniform(80.0, 200.0))
    n = float(rng.uniform(1.45, 2.0))
    fill = float(rng.uniform(0.1, 0.35))
    return N_, L_, lam, R, n, fill


def config3_size(index: int) -> int:
    """Number of spheres of multi-ensemble ``index`` (no packing)."""
    return _config3_draw(rng_for(3, index))[0]


def config3(index: int, n_rhs: int = 8, N: Optional[int] = None, lmax: Optional[int] = None,
            max_tries: int = 2_000_000, sweeps: int = 200) -> Scene:
    """Multi-ensemble ``index``: N ~ U[200, 3000], lmax ~ U{2..5}, lambda, R, n
    and fill drawn per ensemble; monodisperse spheres in a cube; ``n_rhs``
    plane waves on a Fibonacci cap beta <= 60 deg.  Fills above 0.3 use an FCC
    lattice with hard-sphere Monte-Carlo sweeps (``fcc_shaken_cube``; random
    sequential addition slows sharply on its way to jamming), others random
    sequential addition.  Should addition give up (its try budget), the cube
    grows in 3 % steps (a new pass from the same seed each time) until the
    spheres fit, and that ensemble's fill is lower than drawn."""
    sides = []
    for grow in range(60):
        rng = rng_for(3, index)
        N_, L_, lam, R, n, fill = _config3_draw(rng)
        N = N_ if N is None else N
        L = L_ if lmax is None else lmax
        side = (N * 4.0 / 3.0 * np.pi * R ** 3 / fill) ** (1.0 / 3.0) * 1.03 ** grow
        radii = np.full(N, R)

        def sampler(rng, r, m, side=side):
            return rng.uniform(r, side - r, size=(m, 3))

        if fill > 0.3 and grow == 0:
            pos = fcc_shaken_cube(rng, N, R, side, sweeps=sweeps)
        else:
            try:
                pos = random_sequential_addition(rng, radii, sampler, (0, 0, 0), (side, side, side),
                                                 max_tries=max_tries if grow == 0 else 400 * N)
            except RuntimeError:
                sides.append(side)
                continue
        betas, alphas = fibonacci_cap(n_rhs, np.deg2rad(60.0))
        incs = [Incident("plane", beta=float(b), alpha=float(a), pol=2) for b, a in zip(betas, alphas)]
        fill_eff = N * 4.0 / 3.0 * np.pi * R ** 3 / side ** 3
        return Scene(pos, radii, np.full(N, n + 0j), 1.0, lam, L, incs,
                     name=f"ensemble {index}: N={N} L={L} lambda={lam:.0f} fill={fill_eff:.2f}")
    raise RuntimeError(f"config3({index}): no packing found up to side {sides[-1]:.0f} nm")


def fcc_shaken_cube(rng, N, R, side, sweeps=200, gap=1e-3, step=None):
    """N spheres of radius R in the cube [0, side]^3 from an FCC lattice and a
    hard-sphere Monte-Carlo shake (for fills above the random-sequential-
    addition jamming limit, about 0.38 in bulk).

    The FCC lattice constant is the largest one whose sites inside
    [R, side - R]^3 number at least N; N sites are drawn at random (the rest
    stay vacant).  Each sweep then proposes a uniform displacement of up to
    ``step`` (default a quarter of the nearest-neighbour clearance, at least
    R / 20) for every sphere, in ten random batches; a proposal is accepted
    when it stays inside the walls, clears every current sphere and every
    other proposal of its batch (so accepted moves never overlap)."""
    from scipy.spatial import cKDTree
    lo, hi = R, side - R
    inner = hi - lo
    # largest lattice constant a with at least N sites of the FCC lattice in the inner cube
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])

    def sites(a):
        n = int(np.floor(inner / a)) + 1
        g = np.arange(n)
        cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
        pts = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
        return pts[np.all(pts <= inner + 1e-9, axis=1)] + lo

    a_hi = inner
    a_lo = 2.0 * R * np.sqrt(2.0)  # nearest-neighbour distance a / sqrt(2) = 2R
    if sites(a_lo).shape[0] < N:
        raise RuntimeError("fcc_shaken_cube: the cube cannot hold N spheres on an FCC lattice")
    for _ in range(60):
        a_mid = 0.5 * (a_lo + a_hi)
        if sites(a_mid).shape[0] >= N:
            a_lo = a_mid
        else:
            a_hi = a_mid
    pts = sites(a_lo)
    pos = pts[rng.choice(pts.shape[0], N, replace=False)]
    if step is None:
        step = max(0.25 * (a_lo / np.sqrt(2.0) - 2.0 * R), R / 20.0)
    dmin = 2.0 * R + gap
    for _ in range(sweeps):
        order = rng.permutation(N)
        for batch in np.array_split(order, 10):
            prop = pos[batch] + rng.uniform(-step, step, size=(batch.size, 3))
            ok = np.all((prop >= lo) & (prop <= hi), axis=1)
            tree = cKDTree(pos)
            hits = tree.query_ball_point(prop, dmin)
            for q, h in enumerate(hits):
                if ok[q] and any(j != batch[q] for j in h):
                    ok[q] = False
            if ok.any():
                ptree = cKDTree(prop[ok])
                clash = ptree.query_pairs(dmin, output_type="ndarray")
                idx = np.flatnonzero(ok)
                if len(clash):
                    ok[idx[np.unique(clash.ravel())]] = False
            pos[batch[ok]] = prop[ok]
    return pos


def config4(index: int, N: Optional[int] = None, fill: Optional[float] = None, max_tries: int = 2_000_000,
            sweeps: int = 200) -> Scene:
    """Learned-guess ensembles: R = 100 nm, n = 1.52, lambda = 550 nm, L = 3,
    x-polarised plane wave along +z, in a cube; N ~ U[1000, 5000] and fill ~
    U[0.2, 0.4] unless given.  Fills up to 0.3 use random sequential
    addition; above 0.3 (or when addition stalls) an FCC lattice with
    ``sweeps`` hard-sphere Monte-Carlo sweeps (``fcc_shaken_cube``): addition
    slows sharply on its way to jamming (about a minute per 4000-sphere cube
    at fill 0.34), the lattice start does not.  The ensemble has exactly the
    drawn fill."""
    rng = rng_for(4, index)
    N_ = int(rng.integers(1000, 5001))
    fill_ = float(rng.uniform(0.2, 0.4))
    N = N_ if N is None else N
    fill = fill_ if fill is None else fill
    R = 100.0
    side = (N * 4.0 / 3.0 * np.pi * R ** 3 / fill) ** (1.0 / 3.0)
    radii = np.full(N, R)
    pos = None
    if fill <= 0.3:
        def sampler(rng, r, m, side=side):
            return rng.uniform(r, side - r, size=(m, 3))

        try:
            pos = random_sequential_addition(rng, radii, sampler, (0, 0, 0), (side, side, side),
                                             max_tries=max_tries)
        except RuntimeError:
            pos = None
    if pos is None:
        pos = fcc_shaken_cube(rng, N, R, side, sweeps=sweeps)
    return Scene(pos, radii, np.full(N, 1.52 + 0j), 1.0, 550.0, 3,
                 [Incident("plane", beta=0.0, alpha=0.0, pol=2)], name=f"learned-guess cube N={N} fill={fill:.3f}")


def config5(seed_index: int = 0, N: int = 100_000) -> Scene:
    rng = rng_for(5, seed_index)
    R = 130.0
    thick = 4000.0
    vol = N * 4.0 / 3.0 * np.pi * R ** 3
    side = np.sqrt(vol / 0.25 / thick)
    radii = np.full(N, R)

    def sampler(rng, r, m):
        xy = rng.uniform(-side / 2 + r, side / 2 - r, size=(m, 2))
        z = rng.uniform(r, thick - r, size=(m, 1))
        return np.concatenate([xy, z], axis=1)

    pos = random_sequential_addition(rng, radii, sampler, (-side / 2, -side / 2, 0), (side / 2, side / 2, thick))
    inc = Incident("gaussian", waist=5000.0, focus=(0.0, 0.0, 0.0), alpha_G=-np.pi / 2)
    return Scene(pos, radii, np.full(N, 1.52 + 0j), 1.0, 550.0, 3, [inc],
                 name=f"monodisperse slab N={N} L=3 Gaussian w=5um")


def random_cluster(config: int, index: int, N: int, lmax: int, radius=100.0, fill=0.2,
                   n=1.52 + 0j, wavelength=550.0, polydisperse=False) -> Scene:
    """Small seeded cube cluster used by parity tests (sizes the oracle
    finishes in seconds)."""
    rng = rng_for(config, index)
    radii = lognormal_radii(rng, N, radius, 0.1) if polydisperse else np.full(N, float(radius))
    # the centres fill a cube of the nominal volume; the box grows by one
    # diameter so that small clusters stay placeable
    rmax = radii.max()
    side = (np.sum(4.0 / 3.0 * np.pi * radii ** 3) / fill) ** (1.0 / 3.0) + 2.0 * rmax

    def sampler(rng, r, m):
        return rng.uniform(r, side - r, size=(m, 3))

    pos = random_sequential_addition(rng, radii, sampler, (0, 0, 0), (side, side, side))
    return Scene(pos, radii, np.full(N, n, dtype=complex), 1.0, wavelength, lmax,
                 [Incident("plane", beta=0.0, alpha=0.0, pol=2)], name=f"cluster N={N} L={lmax}")


def random_vector(config: int, index: int, shape, dtype=np.complex128):
    """Seeded complex test vector with unit-variance real and imaginary parts."""
    rng = rng_for(config, index)
    v = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    return v.astype(dtype)
