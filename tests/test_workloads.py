"""The seeded input recipe (workloads.py) against the recipe it states: atom
counts, species, layer spacing and stagger, jitter, wrapping, Gaussian widths,
and MD frames whose velocity scale is checked against SI constants."""
import math

import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("name", sorted(W.WORKLOADS))
def test_workload_slab_follows_the_recipe(name):
    w = W.WORKLOADS[name]
    at = W.workload_atoms(w)
    n, layers = w.n, w.layers
    assert len(at.Z) == 2 * n * n * layers == w.n_atoms
    cell = np.asarray(w.cell)
    assert np.all(at.pos >= 0.0) and np.all(at.pos < cell)
    ti = np.array([s == "Ti" for s in at.species])
    assert np.all(at.Z[ti] == 4.0) and np.all(at.Z[~ti] == 6.0) and ti.sum() == n * n * layers
    # each atom within the jitter of its lattice site (periodic distance)
    a, b = cell[0] / n, cell[1] / n
    k = 0
    for l in range(layers):
        z = cell[2] / 2 + (l - (layers - 1) / 2) * 1.0
        sx = 0.5 if l % 2 else 0.0
        for i in range(n):
            for j in range(n):
                for bx, by in ((0.0, 0.0), (0.5, 0.5)):
                    site = np.array([(i + bx + sx) * a, (j + by) * b, z])
                    d = at.pos[k] - site
                    d -= cell * np.round(d / cell)
                    assert np.all(np.abs(d) <= 0.05 + 1e-12), (k, d)
                    k += 1
    if w.sigma_core is None:
        for s in (at.sigma_core, at.sigma_cloud):
            assert np.all((s >= 0.3) & (s <= 1.0)) and np.std(s) > 0.1
    else:
        assert np.all(at.sigma_core == 0.3) and np.all(at.sigma_cloud == 0.8)


def test_recipe_is_seeded():
    w = W.WORKLOADS["mixed_192x192x384"]
    a1, a2, a3 = W.workload_atoms(w, seed=0), W.workload_atoms(w, seed=0), W.workload_atoms(w, seed=1)
    assert np.array_equal(a1.pos, a2.pos) and np.array_equal(a1.sigma_core, a2.sigma_core)
    assert not np.array_equal(a1.pos, a3.pos)


def test_maxwell_velocity_scale_from_si_constants():
    """sqrt(kT/m) per component at 300 K, from CODATA k_B and the atomic mass
    unit in SI, converted to Angstrom/fs (1 m/s = 1e-5 A/fs)."""
    kB, amu = 1.380649e-23, 1.66053906660e-27
    mass = np.full(40000, 15.999)
    v = W.maxwell_velocities(mass, temperature=300.0, seed=3)
    sd = math.sqrt(kB * 300.0 / (15.999 * amu)) * 1e-5
    assert abs(np.std(v) / sd - 1.0) < 0.01
    assert abs(np.mean(v)) < 0.02 * sd


def test_md_frames_are_ballistic_and_wrapped():
    w = W.WORKLOADS["md_128x128x256"]
    at = W.workload_atoms(w)
    tr = W.md_frames(at, w.cell, 5, dt_fs=0.5, temperature=300.0, seed=0)
    cell = np.asarray(w.cell)
    assert tr.shape == (5, len(at.Z), 3)
    assert np.allclose(tr[0], at.pos)
    assert np.all(tr >= 0.0) and np.all(tr < cell)
    step = tr[1:] - tr[:-1]
    step -= cell * np.round(step / cell)
    assert np.allclose(step, step[0][None], atol=1e-12)       # constant velocity
    v = W.maxwell_velocities(at.mass, 300.0, 1)
    assert np.allclose(step[0], 0.5 * v, atol=1e-12)
