"""Seeded synthetic inputs for the generalized-Poisson solver.

This module draws the random numbers and lays out the atom geometry that both
the CPU oracle and the CUDA path consume. It holds none of the solver's
arithmetic: no dielectric, no charge density, no operator. Both sides build
those themselves from the atoms returned here.

Geometry stands in for the paper's TiO2 anatase (101) slab in water (Sec. II.A,
Sec. III): a compact, staggered two-species slab centred in an orthorhombic
periodic cell, with the solvent filling the rest of the box.

Slab recipe (the paper prints no structure file, so this is a reading):
  * ``layers`` planes spaced ``spacing`` (1.0 A) apart, centred at Lz/2;
  * each plane an n x n square lattice, a = Lx/n, with a two-atom basis:
    "Ti" (Z=4) at (0,0) and "O" (Z=6) at (1/2,1/2);
  * alternate planes shifted by (1/2, 0) a;
  * every coordinate jittered uniformly by +-0.05 A with
    ``numpy.random.default_rng(seed)``; positions wrapped into [0, L).
"""
from __future__ import annotations

import dataclasses
import numpy as np

# valence charges used for the Gaussian pseudo-ions (Sec. II.A, the ionic
# densities integrate to Z_I); atomic masses in amu for the Maxwell draw
SPECIES = {"Ti": dict(Z=4.0, mass=47.867), "O": dict(Z=6.0, mass=15.999)}
KB_EV = 8.617333262e-5          # Boltzmann constant, eV/K
EV_PER_AMU_TO_A2_FS2 = 9.648533212e-3   # 1 eV/amu expressed in A^2/fs^2


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    grid: tuple            # (nx, ny, nz)
    cell: tuple            # (lx, ly, lz) in Angstrom
    n: int                 # in-plane lattice repeats
    layers: int
    sigma_core: float | None = 0.3     # None -> drawn per Gaussian
    sigma_cloud: float | None = 0.8
    sigma_range: tuple = (0.3, 1.0)
    tol: float = 1e-10
    levels: int = 0        # 0 -> solver default
    frames: int = 1
    dt_fs: float = 0.5
    temperature: float = 300.0
    description: str = ""

    @property
    def n_atoms(self):
        return 2 * self.n * self.n * self.layers

    @property
    def n_points(self):
        return int(np.prod(self.grid))


WORKLOADS = {
    "fp64_fullbox_32x32x64": Workload(
        "fp64_fullbox_32x32x64", (32, 32, 64), (10.0, 10.0, 20.0), 2, 3,
        description="plain FP64 full-box multigrid, 24-atom slab, tol 1e-10"),
    "split_96x96x192": Workload(
        "split_96x96x192", (96, 96, 192), (13.0, 13.0, 40.0), 3, 4, levels=5,
        description="FP64 dry/wet split, 72-atom slab, 5 levels, tol 1e-10"),
    "adjoint_64x64x128": Workload(
        "adjoint_64x64x128", (64, 64, 128), (10.0, 10.0, 20.0), 2, 6,
        description="FP64 energy, dE/drho and forces, 48-atom slab"),
    "mixed_192x192x384": Workload(
        "mixed_192x192x384", (192, 192, 384), (26.0, 26.0, 52.0), 6, 4,
        sigma_core=None, sigma_cloud=None,
        description="mixed precision, 288-atom slab, sigma ~ U[0.3,1.0] A"),
    "md_128x128x256": Workload(
        "md_128x128x256", (128, 128, 256), (13.0, 13.0, 26.0), 3, 8, frames=100,
        description="100 warm-started MD frames, 144-atom slab, 300 K, dt 0.5 fs"),
}


@dataclasses.dataclass
class Atoms:
    pos: np.ndarray        # (n, 3) float64, Angstrom, wrapped into [0, L)
    Z: np.ndarray          # (n,) float64 valence charge
    sigma_core: np.ndarray   # (n,) float64, std. dev. of the +Z core Gaussian
    sigma_cloud: np.ndarray  # (n,) float64, std. dev. of the -Z cloud Gaussian
    mass: np.ndarray       # (n,) float64 amu
    species: list


def slab_atoms(cell, n, layers, seed=0, spacing=1.0, jitter=0.05,
               sigma_core=0.3, sigma_cloud=0.8, sigma_range=(0.3, 1.0)) -> Atoms:
    """Compact staggered slab (recipe in the module docstring)."""
    cell = np.asarray(cell, dtype=np.float64)
    rng = np.random.default_rng(seed)
    a = cell[0] / n
    b = cell[1] / n
    pos, species = [], []
    for l in range(layers):
        z = cell[2] / 2 + (l - (layers - 1) / 2) * spacing
        sx = 0.5 if l % 2 else 0.0
        for i in range(n):
            for j in range(n):
                for sp, (bx, by) in (("Ti", (0.0, 0.0)), ("O", (0.5, 0.5))):
                    pos.append([((i + bx + sx) % n) * a, ((j + by) % n) * b, z])
                    species.append(sp)
    pos = np.asarray(pos, dtype=np.float64)
    pos += rng.uniform(-jitter, jitter, pos.shape)
    pos = np.mod(pos, cell)
    nat = len(species)
    if sigma_core is None:
        sc = rng.uniform(sigma_range[0], sigma_range[1], nat)
        se = rng.uniform(sigma_range[0], sigma_range[1], nat)
    else:
        sc = np.full(nat, float(sigma_core))
        se = np.full(nat, float(sigma_cloud))
    Z = np.array([SPECIES[s]["Z"] for s in species], dtype=np.float64)
    m = np.array([SPECIES[s]["mass"] for s in species], dtype=np.float64)
    return Atoms(pos, Z, sc, se, m, species)


def workload_atoms(w: Workload, seed=0) -> Atoms:
    return slab_atoms(w.cell, w.n, w.layers, seed=seed, sigma_core=w.sigma_core,
                      sigma_cloud=w.sigma_cloud, sigma_range=w.sigma_range)


def maxwell_velocities(mass, temperature=300.0, seed=0):
    """Per-component N(0, kT/m) velocities in A/fs (no centre-of-mass removal)."""
    rng = np.random.default_rng(seed)
    sd = np.sqrt(KB_EV * temperature / np.asarray(mass) * EV_PER_AMU_TO_A2_FS2)
    return rng.standard_normal((len(mass), 3)) * sd[:, None]


def md_frames(atoms: Atoms, cell, frames, dt_fs=0.5, temperature=300.0, seed=0):
    """Ballistic trajectory x_t = x_0 + t*dt*v, wrapped into the cell.

    Returns an array (frames, n_atoms, 3). Frame 0 is the input geometry.
    """
    v = maxwell_velocities(atoms.mass, temperature, seed + 1)
    cell = np.asarray(cell, dtype=np.float64)
    t = np.arange(frames, dtype=np.float64)[:, None, None] * dt_fs
    return np.mod(atoms.pos[None] + t * v[None], cell)


def fd_atom_indices(n_atoms, count=6, seed=0):
    """Seeded choice of the atoms whose forces are checked by finite differences."""
    rng = np.random.default_rng(seed + 7)
    return np.sort(rng.choice(n_atoms, size=min(count, n_atoms), replace=False))


def random_field(shape, seed=0, mean_zero=True):
    """A seeded smooth-ish random field (used as a generic right-hand side)."""
    rng = np.random.default_rng(seed + 11)
    f = rng.standard_normal(shape)
    if mean_zero:
        f -= f.mean()
    return f


def vdw_radii(Z):
    """Synthetic van der Waals radii (Angstrom) per species for the Eq. 9-10
    dielectric: "O" (Z = 6) 1.52, "Ti" (Z = 4) 2.0."""
    return np.where(np.asarray(Z) == 6, 1.52, 2.0)


def lower_layer_zlim(at, w):
    """z_lim of Eq. 19 between the lowest layer of the slab and the next one (in
    the cell), so that the lowest layer excludes the solvent below it."""
    zs = np.sort(np.mod(at.pos[:, 2], w.cell[2]))
    per = len(zs) // w.layers
    return float(0.5 * (zs[per - 1] + zs[per]))
