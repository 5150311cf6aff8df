"""The seeded synthetic inputs follow their stated recipes: sizes, radius
distribution, material, container, fill fraction, incident fields, disjoint
spheres (the method requires non-overlapping spheres) and determinism."""

import numpy as np
import pytest
from scipy.spatial import cKDTree

import synth


def _disjoint(sc):
    tree = cKDTree(sc.positions)
    pairs = tree.query_pairs(2.0 * sc.radii.max(), output_type="ndarray")
    if len(pairs) == 0:
        return True
    d = np.linalg.norm(sc.positions[pairs[:, 0]] - sc.positions[pairs[:, 1]], axis=1)
    return bool(np.all(d >= sc.radii[pairs[:, 0]] + sc.radii[pairs[:, 1]]))


def _volume(sc):
    return float(np.sum(4.0 / 3.0 * np.pi * sc.radii ** 3))


def test_config1_cube():
    sc = synth.config1(0)
    assert sc.N == 50 and sc.lmax == 3 and sc.wavelength == 550.0
    assert np.all(sc.radii == 100.0) and np.all(sc.n_sphere == 1.52)
    side = (_volume(sc) / 0.2) ** (1.0 / 3.0)
    assert np.all(sc.positions >= 100.0 - 1e-9) and np.all(sc.positions <= side - 100.0 + 1e-9)
    assert _disjoint(sc)
    inc = sc.incidents[0]
    assert inc.kind == "plane" and inc.beta == 0.0 and inc.pol == 2


def test_config2_polydisperse_cylinder_slab():
    sc = synth.config2(0, N=2000)
    assert sc.lmax == 4 and np.all(sc.n_sphere == 1.5 + 0.001j)
    ln = np.log(sc.radii)
    assert abs(np.mean(sc.radii) - 150.0) < 2.0 and abs(np.std(ln) - 0.1) < 0.01
    z = sc.positions[:, 2]
    assert np.all(z - sc.radii >= -1e-9) and np.all(z + sc.radii <= 2000.0 + 1e-9)
    rho = np.hypot(sc.positions[:, 0], sc.positions[:, 1])
    rc = np.sqrt(_volume(sc) / 0.3 / (np.pi * 2000.0))
    assert np.all(rho + sc.radii <= rc + 1e-9)
    assert abs(_volume(sc) / (np.pi * rc ** 2 * 2000.0) - 0.3) < 1e-12
    assert _disjoint(sc)
    inc = sc.incidents[0]
    assert inc.kind == "gaussian" and inc.waist == 2000.0 and inc.alpha_G == -np.pi / 2


def test_config2_full_size_radius_of_the_slab():
    """The bench workload: 10 000 spheres give a cylinder radius near 8.7 um."""
    rng = synth.rng_for(2, 0)
    radii = synth.lognormal_radii(rng, 10_000)
    rc = np.sqrt(np.sum(4.0 / 3.0 * np.pi * radii ** 3) / 0.3 / (np.pi * 2000.0))
    assert 8500.0 < rc < 8900.0


@pytest.mark.parametrize("index", [0, 3])
def test_config3_ensembles(index):
    sc = synth.config3(index, N=300)
    assert 2 <= sc.lmax <= 5 and 400.0 <= sc.wavelength <= 800.0
    assert 80.0 <= sc.radii[0] <= 200.0 and np.all(sc.radii == sc.radii[0])
    assert 1.45 <= sc.n_sphere[0].real <= 2.0
    assert len(sc.incidents) == 8
    assert all(i.kind == "plane" and 0.0 <= i.beta <= np.deg2rad(60.0) + 1e-12 for i in sc.incidents)
    assert _disjoint(sc)


def test_config3_sizes_of_all_64_ensembles():
    sizes = [synth.config3_size(i) for i in range(64)]
    assert all(200 <= n <= 3000 for n in sizes) and len(set(sizes)) > 50


def test_config3_dense_ensembles_keep_their_drawn_fill():
    """Ensemble 17 draws fill 0.34: it is packed from an FCC lattice shaken by
    hard-sphere Monte Carlo, inside the walls of the cube of exactly that
    fill, disjoint and reproducible."""
    sc = synth.config3(17, N=300, sweeps=30)
    drawn = synth._config3_draw(synth.rng_for(3, 17))[5]
    assert drawn > 0.3
    side = (np.sum(4.0 / 3.0 * np.pi * sc.radii ** 3) / drawn) ** (1.0 / 3.0)
    assert np.all(sc.positions >= sc.radii[0] - 1e-9) and np.all(sc.positions <= side - sc.radii[0] + 1e-9)
    assert sc.N == 300 and _disjoint(sc)
    again = synth.config3(17, N=300, sweeps=30)
    assert np.array_equal(sc.positions, again.positions)


def test_config3_grows_the_cube_when_addition_gives_up():
    """With a try budget too small for random sequential addition, the cube
    grows (from the same seed) until the spheres fit: the fill is lower."""
    sc = synth.config3(12, N=300, max_tries=300)
    drawn = synth._config3_draw(synth.rng_for(3, 12))[5]
    assert drawn <= 0.3
    side = sc.positions.max() + sc.radii[0]
    assert sc.N == 300 and _disjoint(sc)
    assert np.sum(4.0 / 3.0 * np.pi * sc.radii ** 3) / side ** 3 < drawn


@pytest.mark.parametrize("fill", [0.25, 0.38, 0.4])
def test_config4_cube_at_its_drawn_fill(fill):
    # fills above 0.3 come from an FCC lattice shaken by hard-sphere Monte
    # Carlo; every ensemble holds exactly its fill, inside the walls, disjoint
    sc = synth.config4(5, N=1200, fill=fill, sweeps=40)
    assert sc.N == 1200 and sc.lmax == 3 and np.all(sc.radii == 100.0) and np.all(sc.n_sphere == 1.52)
    side = (_volume(sc) / fill) ** (1.0 / 3.0)
    assert np.all(sc.positions >= 100.0 - 1e-9) and np.all(sc.positions <= side - 100.0 + 1e-9)
    assert _disjoint(sc)
    assert sc.incidents[0].kind == "plane" and sc.incidents[0].pol == 2


def test_config4_shake_moves_the_lattice():
    # the Monte-Carlo sweeps displace the spheres from their lattice sites
    rng = synth.rng_for(4, 99)
    side = (1000 * 4.0 / 3.0 * np.pi * 100.0 ** 3 / 0.38) ** (1.0 / 3.0)
    p0 = synth.fcc_shaken_cube(synth.rng_for(4, 99), 1000, 100.0, side, sweeps=0)
    p1 = synth.fcc_shaken_cube(rng, 1000, 100.0, side, sweeps=30)
    moved = np.linalg.norm(p1 - p0, axis=1)
    assert np.median(moved) > 5.0


def test_config4_fill_draws_span_the_recipe():
    def draw(i):
        rng = synth.rng_for(4, i)
        return int(rng.integers(1000, 5001)), float(rng.uniform(0.2, 0.4))
    sizes, fills = zip(*[draw(i) for i in range(200)])
    assert min(fills) < 0.22 and max(fills) > 0.38
    assert min(sizes) < 1200 and max(sizes) > 4800
    assert synth.config4(7, N=1000, sweeps=5).name.endswith(f"fill={draw(7)[1]:.3f}")


def test_config5_slab_at_reduced_size():
    sc = synth.config5(0, N=4000)
    assert sc.lmax == 3 and np.all(sc.radii == 130.0)
    z = sc.positions[:, 2]
    assert np.all(z >= 130.0 - 1e-9) and np.all(z <= 4000.0 - 130.0 + 1e-9)
    side = np.sqrt(_volume(sc) / 0.25 / 4000.0)
    assert np.all(np.abs(sc.positions[:, :2]) <= side / 2 - 130.0 + 1e-9)
    assert _disjoint(sc)
    assert sc.incidents[0].kind == "gaussian" and sc.incidents[0].waist == 5000.0


def test_seeded_and_independent():
    a, b = synth.config2(1, N=500), synth.config2(1, N=500)
    c = synth.config2(2, N=500)
    assert np.array_equal(a.positions, b.positions) and np.array_equal(a.radii, b.radii)
    assert not np.allclose(a.positions, c.positions)
    v1 = synth.random_vector(2, 77, (10, 4))
    assert np.array_equal(v1, synth.random_vector(2, 77, (10, 4)))
