"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Small cases compare element by element; the full-size workloads compare
sampled outputs the oracle computes one by one, and properties that hold at
any size (the FP64 residual measured by the oracle's own operator, the energy
identity). Tolerances: FP64 path 1e-10 relative for phi and E; mixed precision
1e-8 for E and phi, 1e-6 for forces.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import gp_oracle as O

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0904_4887_gb300 import GPSolver
    return GPSolver


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _gauss(at):
    return np.stack([at.Z, at.sigma_core, at.sigma_cloud], axis=1)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _case(grid, cell, n, layers, seed=0):
    at = W.slab_atoms(cell, n, layers, seed=seed)
    h = O.spacing(grid, cell)
    eps = O.dielectric(grid, cell, at.pos)
    rho = O.charge_density(grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    return at, h, eps, rho


SMALL = [((32, 32, 64), (10.0, 10.0, 20.0), 2, 3),       # the 32x32x64 full-box workload
         ((24, 24, 48), (10.0, 10.0, 20.0), 2, 3),       # 3 * 2^k extents, ragged 32-wide tiles
         ((16, 8, 24), (7.0, 6.5, 12.0), 1, 2)]          # anisotropic, tiny


@pytest.fixture(scope="module")
def small_cases():
    return [(_case(g, c, n, l), g, c) for g, c, n, l in SMALL]


# ------------------------------------------------------------------ fields

@pytest.mark.parametrize("k", range(len(SMALL)))
def test_dielectric_matches_oracle(small_cases, k):
    GPSolver = _gpu()
    (at, h, eps, rho), grid, cell = small_cases[k]
    s = GPSolver(grid, cell)
    s.set_atoms(_t(at.pos))
    e = s.eps().cpu().numpy()
    assert _rel(e, eps) < 1e-13
    pm = s.plane_max()
    assert np.array_equal(pm < 1e-3, O.dry_planes(eps))


@pytest.mark.parametrize("k", range(len(SMALL)))
def test_charge_density_matches_oracle(small_cases, k):
    GPSolver = _gpu()
    (at, h, eps, rho), grid, cell = small_cases[k]
    s = GPSolver(grid, cell)
    r = s.build_rho(_t(at.pos), _t(_gauss(at))).cpu().numpy()
    assert np.max(np.abs(r - rho)) < 1e-12 * np.max(np.abs(rho))


def test_empty_atom_list_gives_uniform_eps():
    GPSolver = _gpu()
    s = GPSolver((16, 16, 16), (8.0, 8.0, 8.0))
    s.set_atoms(torch.zeros((0, 3), dtype=torch.float64, device=DEV))
    assert torch.all(s.eps() == 78.36)


# ------------------------------------------------------------------ operators

@pytest.mark.parametrize("k", range(len(SMALL)))
def test_fft_poisson_matches_oracle(small_cases, k):
    GPSolver = _gpu()
    (at, h, eps, rho), grid, cell = small_cases[k]
    s = GPSolver(grid, cell)
    src = W.random_field(eps.shape, seed=k)
    got = s.fft_poisson(_t(src)).cpu().numpy()
    ref = O.fft_poisson(src, h)
    assert _rel(got, ref) < 1e-12


@pytest.mark.parametrize("k", range(len(SMALL)))
def test_fp64_residual_matches_oracle(small_cases, k):
    GPSolver = _gpu()
    (at, h, eps, rho), grid, cell = small_cases[k]
    s = GPSolver(grid, cell)
    s.set_atoms(_t(at.pos))
    phi = W.random_field(eps.shape, seed=10 + k)
    r, rel = s.residual(_t(rho), _t(phi))
    ref = -4 * math.pi * rho - O.apply_A(phi, eps, h)
    assert _rel(r.cpu().numpy(), ref) < 1e-13
    assert abs(rel - np.linalg.norm(ref) / np.linalg.norm(4 * math.pi * rho)) < 1e-12 * rel


# ------------------------------------------------------------------ solves

def _solve_case(small_cases, k, **params):
    GPSolver = _gpu()
    (at, h, eps, rho), grid, cell = small_cases[k]
    s = GPSolver(grid, cell, **params)
    s.set_atoms(_t(at.pos))
    rho_t = _t(rho)
    phi = s.solve(rho_t, tol=1e-13 if params.get("precision", 1) == 0 else 1e-12)
    ref, info = O.solve(rho, eps, h, tol=1e-14)
    return s, phi.cpu().numpy(), ref, rho, grid, cell, eps


@pytest.mark.parametrize("k", range(len(SMALL)))
@pytest.mark.parametrize("split,accel", [(0, 1), (1, 1), (1, 0)])
def test_fp64_solve_matches_oracle(small_cases, k, split, accel):
    s, phi, ref, rho, grid, cell, eps = _solve_case(small_cases, k, precision=0, split=split, inner=6, accel=accel)
    assert _rel(phi, ref) < 1e-10
    E = O.energy(rho, phi, grid, cell)
    E0 = O.energy(rho, ref, grid, cell)
    assert abs(E - E0) < 1e-10 * abs(E0)
    st = s.stats()
    assert st.residual < 1e-13


@pytest.mark.parametrize("k", range(len(SMALL)))
@pytest.mark.parametrize("split,accel", [(0, 1), (1, 1), (1, 0)])
def test_mixed_solve_matches_oracle(small_cases, k, split, accel):
    s, phi, ref, rho, grid, cell, eps = _solve_case(small_cases, k, precision=1, split=split, accel=accel)
    assert _rel(phi, ref) < 1e-8
    E = O.energy(rho, phi, grid, cell)
    E0 = O.energy(rho, ref, grid, cell)
    assert abs(E - E0) < 1e-8 * abs(E0)


ROWCASE = ((64, 48, 48), (10.0, 7.5, 12.0), 2, 2)   # nx = 64: the row-tile smoothers apply; 6 rows ragged


@pytest.fixture(scope="module")
def row_case():
    g, c, n, l = ROWCASE
    at, h, eps, rho = _case(g, c, n, l)
    ref, info = O.solve(rho, eps, h, tol=1e-14)
    return (at, h, eps, rho), g, c, ref


@pytest.mark.parametrize("shape", range(15))
@pytest.mark.parametrize("split", [0, 1])
def test_every_sweep_shape_converges_to_oracle(row_case, shape, split):
    """Each finest-level smoother tile (x-y tiles, whole-row tiles with 4, 6, 8
    rows, warp-specialised whole-row tiles), on the periodic box and on the Dirichlet wet band, inside the mixed
    solve, gives the oracle's solution."""
    GPSolver = _gpu()
    (at, h, eps, rho), grid, cell, ref = row_case
    s = GPSolver(grid, cell, precision=1, split=split, sweep_shape=shape)
    s.set_atoms(_t(at.pos))
    assert s.stats().sweep_shape == shape
    assert s.stats().split_active == split
    phi = s.solve(_t(rho), tol=1e-12).cpu().numpy()
    assert _rel(phi, ref) < 1e-8
    assert s.stats().residual < 1e-12


ROWLEN = {96: ((96, 24, 48), (15.0, 7.5, 12.0)), 128: ((128, 24, 48), (20.0, 7.5, 12.0)),
          256: ((256, 32, 48), (40.0, 10.0, 12.0))}


@pytest.fixture(scope="module")
def rowlen_cases():
    out = {}
    for nx, (g, c) in ROWLEN.items():
        at, h, eps, rho = _case(g, c, 2, 2, seed=3)
        ref, _ = O.solve(rho, eps, h, tol=1e-14)
        out[nx] = (at, rho, ref, g, c)
    return out


@pytest.mark.parametrize("nx", sorted(ROWLEN))
@pytest.mark.parametrize("shape", range(4, 15))
def test_row_tiles_on_other_row_lengths(rowlen_cases, nx, shape):
    """The whole-row tiles (48, 64 and 128 pairs per row; 24 or 32 rows, so
    the 14- and 12-row tiles are ragged), forced through sweep_shape, give the
    oracle's solution; a tile that does not fit a row length resolves to shape 0."""
    GPSolver = _gpu()
    at, rho, ref, grid, cell = rowlen_cases[nx]
    s = GPSolver(grid, cell, precision=1, sweep_shape=shape)
    s.set_atoms(_t(at.pos))
    assert s.stats().sweep_shape in (shape, 0)
    phi = s.solve(_t(rho), tol=1e-12).cpu().numpy()
    assert _rel(phi, ref) < 1e-8
    assert s.stats().residual < 1e-12


@pytest.mark.parametrize("k", range(len(SMALL)))
@pytest.mark.parametrize("graph_outer", [0, 2])
def test_mixed_df64_residual_path(small_cases, k, graph_outer):
    """Mixed precision at tol 1e-9 runs its outer residual in df64: the residual it
    reports is the FP64 residual of the phi it returns (checked by the oracle) and
    the energy is within 1e-8 of the oracle's."""
    GPSolver = _gpu()
    (at, h, eps, rho), grid, cell = small_cases[k]
    s = GPSolver(grid, cell, precision=1, split=0, graph_outer=graph_outer)
    s.set_atoms(_t(at.pos))
    phi = s.solve(_t(rho), tol=1e-9).cpu().numpy()
    st = s.stats()
    true_res = O.residual_norm(phi, rho, eps, h)
    assert st.residual <= 1e-9 and true_res <= 2e-9
    assert abs(true_res - st.residual) <= 1e-11 + 0.01 * true_res
    ref, _ = O.solve(rho, eps, h, tol=1e-14)
    E, E0 = O.energy(rho, phi, grid, cell), O.energy(rho, ref, grid, cell)
    assert abs(E - E0) < 1e-8 * abs(E0)


@pytest.mark.parametrize("nu_coarse", [0, 1, 3])
@pytest.mark.parametrize("split", [0, 1])
def test_coarse_sweep_count_converges_to_oracle(small_cases, nu_coarse, split):
    """Other sweep counts on the levels below the finest (nu_coarse; 0 = nu1, nu2; the shared-
    memory bottom of the V-cycle and the band levels included) give the oracle's
    solution; a count outside 0 .. 8 is refused."""
    GPSolver = _gpu()
    from paper_0904_4887_gb300 import GPError
    (at, h, eps, rho), grid, cell = small_cases[0]
    s = GPSolver(grid, cell, precision=1, split=split, nu_coarse=nu_coarse)
    s.set_atoms(_t(at.pos))
    phi = s.solve(_t(rho), tol=1e-12).cpu().numpy()
    ref, _ = O.solve(rho, eps, h, tol=1e-14)
    assert _rel(phi, ref) < 1e-8
    assert s.stats().residual < 1e-12
    with pytest.raises(GPError) as e:
        GPSolver(grid, cell, precision=1, nu_coarse=9).set_atoms(_t(at.pos))
    assert e.value.status == 1                      # GP_ERR_INVALID_ARG


def test_split_band_matches_oracle_planner(small_cases):
    GPSolver = _gpu()
    (at, h, eps, rho), grid, cell = small_cases[0]
    s = GPSolver(grid, cell, split=1, precision=0)
    s.set_atoms(_t(at.pos))
    st = s.stats()
    levels = st.levels
    expect = O.plan_band(O.dry_planes(eps), levels, 1)
    assert expect is not None and st.split_active == 1
    assert (st.band_first, st.band_dirichlet) == expect
    assert st.dry_planes == int(O.dry_planes(eps).sum())


def test_uniform_eps_is_vacuum_over_eps0():
    """No atoms: eps = eps0 everywhere and phi = phi_vac / eps0 (a closed form)."""
    GPSolver = _gpu()
    grid, cell = (32, 32, 32), (10.0, 10.0, 10.0)
    h = O.spacing(grid, cell)
    rho = W.random_field((32, 32, 32), seed=3)
    s = GPSolver(grid, cell, precision=0)
    s.set_atoms(torch.zeros((0, 3), dtype=torch.float64, device=DEV))
    phi = s.solve(_t(rho), tol=1e-13).cpu().numpy()
    ref = O.vacuum_potential(rho, h) / 78.36
    assert _rel(phi, ref) < 1e-10


# ------------------------------------------------------------------ energy, forces

def test_energy_and_forces_match_oracle():
    GPSolver = _gpu()
    grid, cell = (32, 32, 48), (10.0, 10.0, 15.0)
    at, h, eps, rho = _case(grid, cell, 2, 3, seed=2)
    s = GPSolver(grid, cell, precision=0)
    pos = _t(at.pos)
    s.set_atoms(pos)
    phi = s.solve(_t(rho), tol=1e-13)
    E, E2, F = s.energy_forces(phi, _t(rho), _t(_gauss(at)))
    p = phi.cpu().numpy()
    Ge, Gr = O.energy_gradient(p, grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    Fo = -(Ge + Gr)
    assert _rel(F.cpu().numpy(), Fo) < 1e-10
    Eo = O.energy(rho, p, grid, cell)
    assert abs(E - Eo) < 1e-12 * abs(Eo)
    assert abs(E2 - O.field_energy(p, eps, grid, cell)) < 1e-12 * abs(Eo)
    assert abs(E - E2) < 1e-10 * abs(E)          # Eq. 4 identity at convergence
    # solvent (eps) part alone
    _, _, Fe = s.energy_forces(phi, _t(rho), None)
    assert _rel(Fe.cpu().numpy(), -Ge) < 1e-10


# ------------------------------------------------------------------ Eq. 9-10 dielectric (kind 1)

def _radii(Z):
    return W.vdw_radii(Z)


@pytest.mark.parametrize("k", range(len(SMALL)))
def test_gamma_dielectric_matches_oracle(small_cases, k):
    """Eq. 9-10 over every image within the tail-bounded radius (several cells
    wide on these grids): the library picks the oracle's radius and matches its
    eps element by element."""
    GPSolver = _gpu()
    (at, h, eps, rho), grid, cell = small_cases[k]
    p = O.GammaParams()
    rv = _radii(at.Z)
    ref = O.dielectric_gamma(grid, cell, at.pos, rv, p)
    s = GPSolver(grid, cell, precision=0, kind=1, beta=p.beta)
    s.set_atoms(_t(at.pos), radii=_t(rv))
    assert abs(s.stats().gamma_cutoff - O.gamma_cutoff(cell, rv, p.tail)) < 1e-5
    assert s.stats().gamma_cutoff > 2.0 * max(cell)
    assert _rel(s.eps().cpu().numpy(), ref) < 1e-13


def test_gamma_tail_parameter_moves_the_radius():
    """A looser tail bound shortens the radius the way the oracle's bound says,
    and eps follows the oracle at that radius too."""
    GPSolver = _gpu()
    grid, cell = (16, 8, 24), (7.0, 6.5, 12.0)
    at = W.slab_atoms(cell, 1, 2, seed=0)
    rv = _radii(at.Z)
    p = O.GammaParams(tail=1e-6)
    s = GPSolver(grid, cell, precision=0, kind=1, beta=p.beta, gamma_tail=p.tail)
    s.set_atoms(_t(at.pos), radii=_t(rv))
    rc = O.gamma_cutoff(cell, rv, p.tail)
    assert abs(s.stats().gamma_cutoff - rc) < 1e-5 and rc < O.gamma_cutoff(cell, rv, 1e-13) - 5.0
    assert _rel(s.eps().cpu().numpy(), O.dielectric_gamma(grid, cell, at.pos, rv, p)) < 1e-13


def test_gamma_fp64_kernels_beyond_the_staged_rows():
    """A tail bound so small that the radius passes the rows the df64 kernels
    stage (54 A) takes the FP64 kernels; eps and both force terms still follow
    the oracle at that radius."""
    GPSolver = _gpu()
    grid, cell = (16, 8, 24), (7.0, 6.5, 12.0)
    at = W.slab_atoms(cell, 1, 2, seed=0)
    rv = _radii(at.Z)
    p = O.GammaParams(tail=1e-30)
    s = GPSolver(grid, cell, precision=0, kind=1, beta=p.beta, gamma_tail=p.tail)
    s.set_atoms(_t(at.pos), radii=_t(rv))
    assert s.stats().gamma_cutoff > 60.0
    assert _rel(s.eps().cpu().numpy(), O.dielectric_gamma(grid, cell, at.pos, rv, p)) < 1e-13


def test_gamma_dielectric_is_reproducible():
    """The df64 kernels sum each point's terms in a fixed order (the tile's image
    list is built by a scan, not by atomics): building eps twice gives the same bits."""
    GPSolver = _gpu()
    grid, cell = (32, 32, 48), (10.0, 10.0, 15.0)
    at, _, _, _ = _case(grid, cell, 2, 3, seed=2)
    rv = _t(_radii(at.Z))
    s = GPSolver(grid, cell, precision=0, kind=1)
    s.set_atoms(_t(at.pos), radii=rv)
    e1 = s.eps().clone()
    s.set_atoms(_t(at.pos), radii=rv)
    assert torch.equal(e1, s.eps())


def test_gamma_image_lists_longer_than_a_tile_holds():
    """A 10 x 10 x 15 A cell with 54 atoms: 847 images per atom within the 41.7 A
    radius, about 11,000 reaching each tile, more than the image list of either
    df64 kernel holds, so both take their candidates in windows. eps and both force
    terms still follow the oracle."""
    GPSolver = _gpu()
    grid, cell = (16, 16, 24), (10.0, 10.0, 15.0)
    at = W.slab_atoms(cell, 3, 3, seed=4)
    rv = _radii(at.Z)
    p = O.GammaParams()
    eps = O.dielectric_gamma(grid, cell, at.pos, rv, p)
    s = GPSolver(grid, cell, precision=0, kind=1, beta=p.beta)
    s.set_atoms(_t(at.pos), radii=_t(rv))
    assert _rel(s.eps().cpu().numpy(), eps) < 1e-13
    rho = O.charge_density(grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    phi = s.solve(_t(rho), tol=1e-13)
    pn = phi.cpu().numpy()
    _, _, F = s.energy_forces(phi, _t(rho), _t(_gauss(at)))
    Ge, Gr = O.energy_gradient(pn, grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud, p=p, rvdw=rv)
    assert _rel(F.cpu().numpy(), -(Ge + Gr)) < 1e-10


def test_gamma_energy_and_forces_match_oracle():
    """Eq. 9-10 dielectric: solve, energy and both force terms against the oracle (Eq. 11 with
    the derived Eq. 12 sign)."""
    GPSolver = _gpu()
    grid, cell = (32, 32, 48), (10.0, 10.0, 15.0)
    at, h, _, rho = _case(grid, cell, 2, 3, seed=2)
    p = O.GammaParams()
    rv = _radii(at.Z)
    eps = O.dielectric_gamma(grid, cell, at.pos, rv, p)
    s = GPSolver(grid, cell, precision=0, kind=1, beta=p.beta)
    s.set_atoms(_t(at.pos), radii=_t(rv))
    phi = s.solve(_t(rho), tol=1e-13)
    ref, _ = O.solve(rho, eps, h, tol=1e-14)
    pn = phi.cpu().numpy()
    assert _rel(pn, ref) < 1e-10
    E, E2, F = s.energy_forces(phi, _t(rho), _t(_gauss(at)))
    Ge, Gr = O.energy_gradient(pn, grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud, p=p, rvdw=rv)
    assert _rel(F.cpu().numpy(), -(Ge + Gr)) < 1e-10
    _, _, Fe = s.energy_forces(phi, _t(rho), None)
    assert _rel(Fe.cpu().numpy(), -Ge) < 1e-10
    assert abs(E - E2) < 1e-10 * abs(E)


def test_gamma_forces_match_central_differences_on_the_gpu():
    """Eq. 9-10 forces of the library against central differences (h = 1e-4 A)
    of its own energy, every step on the GPU: the solvent term with rho frozen,
    on 4 seeded atoms, to 1e-6 of the largest component."""
    GPSolver = _gpu()
    grid, cell = (32, 32, 48), (10.0, 10.0, 15.0)
    at, h, _, rho = _case(grid, cell, 2, 3, seed=2)
    rv = _t(_radii(at.Z))
    s = GPSolver(grid, cell, precision=0, kind=1)
    rho_t = _t(rho)

    def J(q):
        s.set_atoms(_t(q), radii=rv)
        phi = s.solve(rho_t, tol=1e-13)
        E, E2, _ = s.energy_forces(phi, rho_t, None, forces=False)
        return 2.0 * E - E2            # the variational energy: second order in phi's error

    s.set_atoms(_t(at.pos), radii=rv)
    phi = s.solve(rho_t, tol=1e-13)
    _, _, F = s.energy_forces(phi, rho_t, None)
    F = F.cpu().numpy()
    sel = np.random.default_rng(11).choice(len(at.pos), 4, replace=False)
    d = 1e-4
    fd = np.zeros((len(sel), 3))
    for t_, a in enumerate(sel):
        for c in range(3):
            pp = at.pos.copy(); pp[a, c] += d
            pm = at.pos.copy(); pm[a, c] -= d
            fd[t_, c] = -(J(pp) - J(pm)) / (2 * d)
    scale = np.max(np.abs(fd))
    assert scale > 1e-3
    assert np.max(np.abs(fd - F[sel])) < 1e-6 * scale


def _eq19_setup(grid, cell, n, layers, seed=0):
    at = W.slab_atoms(cell, n, layers, seed=seed)
    zs = np.sort(at.pos[:, 2])
    per = len(zs) // layers
    zlim = 0.5 * (zs[per - 1] + zs[per])                  # the lowest layer excludes the solvent below it
    return at, W.vdw_radii(at.Z), zlim


@pytest.mark.parametrize("grid,cell,n,layers", [((32, 32, 64), (10.0, 10.0, 20.0), 2, 3),
                                                ((24, 24, 48), (10.0, 10.0, 20.0), 2, 3)])
def test_eq19_dielectric_matches_oracle(grid, cell, n, layers):
    GPSolver = _gpu()
    at, rv, zlim = _eq19_setup(grid, cell, n, layers)
    p = O.GammaParams()
    ref = O.dielectric_eq19(grid, cell, at.pos, rv, zlim, p)
    s = GPSolver(grid, cell, precision=0, kind=2, beta=p.beta, zlim=zlim)
    s.set_atoms(_t(at.pos), radii=_t(rv))
    assert _rel(s.eps().cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("split,precision", [(0, 0), (1, 0), (1, 1)])
def test_eq19_solve_and_forces_match_oracle(split, precision):
    """Eq. 19 makes the region below the slab dry, so the split's band (with the whole
    dry run as Dirichlet planes) is about half the box; the solve (full box or split)
    and the forces match the oracle."""
    GPSolver = _gpu()
    grid, cell = (32, 32, 64), (10.0, 10.0, 20.0)
    at, rv, zlim = _eq19_setup(grid, cell, 2, 3, seed=1)
    p = O.GammaParams()
    h = O.spacing(grid, cell)
    eps = O.dielectric_eq19(grid, cell, at.pos, rv, zlim, p)
    rho = O.charge_density(grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    ref, _ = O.solve(rho, eps, h, tol=1e-14)
    s = GPSolver(grid, cell, precision=precision, split=split, kind=2, beta=p.beta, zlim=zlim,
                 n_dirichlet=0)
    s.set_atoms(_t(at.pos), radii=_t(rv))
    st = s.stats()
    if split:
        assert st.split_active == 1 and st.wet_fraction < 0.8
    phi = s.solve(_t(rho), tol=1e-13 if precision == 0 else 1e-12)
    pn = phi.cpu().numpy()
    assert _rel(pn, ref) < (1e-10 if precision == 0 else 1e-8)
    if precision == 0:
        E, E2, F = s.energy_forces(phi, _t(rho), _t(_gauss(at)))
        Ge, Gr = O.energy_gradient(pn, grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud, p=p, rvdw=rv,
                                   zlim=zlim)
        assert _rel(F.cpu().numpy(), -(Ge + Gr)) < 1e-10
        assert abs(E - E2) < 1e-10 * abs(E)


def test_gamma_needs_radii():
    GPSolver = _gpu()
    from paper_0904_4887_gb300.gp import GPError
    grid, cell = (16, 8, 24), (7.0, 6.5, 12.0)
    at = W.slab_atoms(cell, 1, 2, seed=0)
    s = GPSolver(grid, cell, kind=1)
    with pytest.raises(GPError):
        s.set_atoms(_t(at.pos))
    with pytest.raises(GPError):
        s.set_atoms(_t(at.pos), radii=_t(-np.ones(len(at.Z))))


def test_autograd_forces_match_central_differences():
    """dE/dR from the hand-written backward against central differences of E
    (h = 1e-4 A) on 6 seeded atoms, rho moving with its atoms."""
    GPSolver = _gpu()
    from paper_0904_4887_gb300 import poisson_energy
    grid, cell = (32, 32, 64), (10.0, 10.0, 20.0)
    at = W.slab_atoms(cell, 2, 3, seed=4)
    s = GPSolver(grid, cell, precision=0)
    gauss = _t(_gauss(at))

    def energy(p):
        pt = _t(p)
        rho = s.build_rho(pt, gauss)
        E, _ = poisson_energy(pt, rho, s, tol=1e-13, gauss=gauss)
        return float(E)

    pos = _t(at.pos).requires_grad_(True)
    rho = s.build_rho(pos.detach(), gauss)
    E, phi = poisson_energy(pos, rho, s, tol=1e-13, gauss=gauss)
    E.backward()
    G = pos.grad.cpu().numpy()
    idx = W.fd_atom_indices(len(at.Z), 6, seed=0)
    d = 1e-4
    fd = np.zeros((len(idx), 3))
    for t, a in enumerate(idx):
        for c in range(3):
            pp = at.pos.copy(); pp[a, c] += d
            pm = at.pos.copy(); pm[a, c] -= d
            fd[t, c] = (energy(pp) - energy(pm)) / (2 * d)
    err = np.max(np.abs(fd - G[idx])) / np.max(np.abs(fd))
    assert err < 1e-6, err


def test_grad_rho_is_h3_phi():
    GPSolver = _gpu()
    from paper_0904_4887_gb300 import poisson_energy
    grid, cell = (16, 16, 32), (10.0, 10.0, 20.0)
    at, h, eps, rho = _case(grid, cell, 2, 2)
    s = GPSolver(grid, cell, precision=0)
    rho_t = _t(rho).requires_grad_(True)
    E, phi = poisson_energy(_t(at.pos), rho_t, s, tol=1e-13)
    E.backward()
    assert torch.allclose(rho_t.grad, phi * s.dv, rtol=0, atol=0)


# ------------------------------------------------------------------ errors

def test_error_paths():
    GPSolver = _gpu()
    from paper_0904_4887_gb300 import GPError
    grid, cell = (16, 16, 16), (8.0, 8.0, 8.0)
    s = GPSolver(grid, cell)
    rho = torch.ones((16, 16, 16), dtype=torch.float64, device=DEV)
    with pytest.raises(GPError) as e:
        s.solve(rho - rho.mean(), tol=1e-8)
    assert e.value.status == 8                      # no dielectric yet
    s.set_atoms(torch.zeros((0, 3), dtype=torch.float64, device=DEV))
    with pytest.raises(GPError) as e:
        s.solve(rho, tol=1e-8)                      # not neutral
    assert e.value.status == 2
    with pytest.raises(GPError) as e:
        s.solve(rho - rho.mean(), tol=0.0)
    assert e.value.status == 1
    z = s.solve(torch.zeros_like(rho), tol=1e-8)
    assert torch.count_nonzero(z) == 0
    with pytest.raises(GPError):
        GPSolver((10, 16, 16), cell)                # 10 is not 2^a 3^b


def test_graph_captured_warm_start_frames():
    """Consecutive frames warm-started from the previous phi with the fixed-count
    graph-captured solve reach the tolerance and agree with the oracle."""
    GPSolver = _gpu()
    grid, cell = (32, 32, 64), (10.0, 10.0, 20.0)
    at = W.slab_atoms(cell, 2, 3, seed=0)
    traj = W.md_frames(at, cell, 4, dt_fs=0.5, temperature=300.0, seed=0)
    gauss = _t(_gauss(at))
    s = GPSolver(grid, cell, precision=1, graph_outer=2)
    phi = s.zeros()
    for f in range(4):
        pos = _t(traj[f])
        s.set_atoms(pos)
        rho = s.build_rho(pos, gauss)
        s.solve(rho, phi, tol=1e-10)
        assert s.stats().residual <= 1e-10
    h = O.spacing(grid, cell)
    eps = O.dielectric(grid, cell, traj[3])
    rho_o = O.charge_density(grid, cell, traj[3], at.Z, at.sigma_core, at.sigma_cloud)
    ref, _ = O.solve(rho_o, eps, h, tol=1e-14)
    assert _rel(phi.cpu().numpy(), ref) < 1e-7


def test_checked_loop_starts_from_the_callers_phi(small_cases):
    """The outer loop of the mixed solve starts from the phi it is given. From
    zero its first residual is b itself (recorded as 1, not evaluated); from a
    nonzero phi (the answer to a looser tolerance) the first residual is
    evaluated, equals the residual that solve ended with, and the solve goes on
    to the oracle's answer."""
    GPSolver = _gpu()
    (at, h, eps, rho), grid, cell = small_cases[0]
    s = GPSolver(grid, cell, precision=1)
    s.set_atoms(_t(at.pos))
    rho_t = _t(rho)
    phi = s.zeros()
    s.solve(rho_t, phi, tol=1e-6)
    st = s.stats()
    assert st.history[0] == 1.0 and st.residual <= 1e-6
    r1 = st.residual
    s.solve(rho_t, phi, tol=1e-10)
    st = s.stats()
    assert abs(st.history[0] - r1) <= 0.05 * r1          # the gauge shift leaves the residual alone
    assert st.residual <= 1e-10
    ref, _ = O.solve(rho, eps, h, tol=1e-14)
    assert _rel(phi.cpu().numpy(), ref) < 1e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_forces_of_every_atom_on_a_mid_size_grid(precision):
    """Both force terms on 64x64x128 in a 16 x 16 x 32 A cell (18 atoms, the
    cut-off sphere well inside the cell) against the oracle's gradient for
    every atom, on the library's own phi, with rho moving and held fixed."""
    GPSolver = _gpu()
    grid, cell = (64, 64, 128), (16.0, 16.0, 32.0)
    at = W.slab_atoms(cell, 3, 2, seed=7)
    gauss = _t(_gauss(at))
    s = GPSolver(grid, cell, precision=precision)
    pos = _t(at.pos)
    s.set_atoms(pos)
    rho = s.build_rho(pos, gauss)
    phi = s.solve(rho, tol=1e-10)
    _, _, F = s.energy_forces(phi, rho, gauss)
    Ge, Gr = O.energy_gradient(phi.cpu().numpy(), grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    assert _rel(F.cpu().numpy(), -(Ge + Gr)) < 1e-9
    _, _, Fe = s.energy_forces(phi, rho, None)
    assert _rel(Fe.cpu().numpy(), -Ge) < 1e-9
