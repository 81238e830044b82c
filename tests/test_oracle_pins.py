"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one oracle function against a closed form, an invariant, a
special case that reduces to a textbook result, or brute force on a tiny input,
chosen so that a plausible slip (a dropped term, a wrong sign, a swapped axis,
a missing periodic image, a wrong face mean) fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.special import erf, erfc

from oracle import gp_oracle as O
import workloads as W

PAR = O.DielectricParams()


def _grid_points(grid, cell):
    h = O.spacing(grid, cell)
    z, y, x = np.meshgrid(np.arange(grid[2]) * h[2], np.arange(grid[1]) * h[1],
                          np.arange(grid[0]) * h[0], indexing="ij")
    return x, y, z


def _small_slab(grid=(16, 16, 32), cell=(10.0, 10.0, 20.0), n=2, layers=2, seed=0):
    at = W.slab_atoms(cell, n, layers, seed=seed)
    eps = O.dielectric(grid, cell, at.pos)
    rho = O.charge_density(grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    return at, eps, rho


# ---------------------------------------------------------------- dielectric

def test_dielectric_single_atom_closed_form():
    """One atom: eps = 1 + (eps0-1) s(d); s(r0) = 1/2; eps = eps0 beyond rcut."""
    grid, cell = (40, 40, 40), (20.0, 20.0, 20.0)
    R = np.array([[10.0, 10.0, 10.0]])
    eps = O.dielectric(grid, cell, R)
    x, y, z = _grid_points(grid, cell)
    d = np.sqrt((x - 10) ** 2 + (y - 10) ** 2 + (z - 10) ** 2)
    expect = np.where(d < 6.0, 1 + 77.36 * 0.5 * (1 + erf((d - 2.5) / 0.5)), 78.36)
    assert np.max(np.abs(eps - expect)) < 1e-12
    # the grid point at distance exactly r0 = 2.5 A: eps = 1 + 77.36/2
    assert abs(eps[20, 20, 25] - (1 + 77.36 / 2)) < 1e-12
    # at the atom: 1 + 77.36 erfc(5)/2
    assert abs(eps[20, 20, 20] - (1 + 77.36 * 0.5 * erfc(5.0))) < 1e-12


def test_dielectric_periodic_images_and_translation():
    """Shifting every atom by one grid step rolls eps by one index (exact
    translation invariance, which needs every periodic image)."""
    grid, cell = (24, 20, 28), (9.0, 7.5, 10.5)
    rng = np.random.default_rng(3)
    R = rng.uniform(0, 1, (5, 3)) * np.array(cell)
    R[0] = [0.1, 0.2, 0.3]           # near a corner: its images matter
    h = O.spacing(grid, cell)
    e0 = O.dielectric(grid, cell, R)
    for c in range(3):
        shift = np.zeros(3)
        shift[c] = h[c]
        e1 = O.dielectric(grid, cell, np.mod(R + shift, cell))
        assert np.max(np.abs(e1 - np.roll(e0, 1, axis=O.AX[c]))) < 1e-11


def test_dielectric_grid_matches_brute_force_points():
    """Bounding-box construction equals the 27-image brute force at every point."""
    grid, cell = (12, 10, 14), (8.0, 7.0, 9.0)
    rng = np.random.default_rng(5)
    R = rng.uniform(0, 1, (4, 3)) * np.array(cell)
    e = O.dielectric(grid, cell, R)
    x, y, z = _grid_points(grid, cell)
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    assert np.max(np.abs(e.ravel() - O.dielectric_points(pts, cell, R))) < 1e-11


def test_dielectric_gradient_matches_finite_differences():
    grid, cell = (14, 12, 16), (8.0, 7.0, 9.0)
    rng = np.random.default_rng(9)
    R = rng.uniform(0, 1, (3, 3)) * np.array(cell)
    P = O.dielectric_product(grid, cell, R)
    for a in range(3):
        g = O.dielectric_gradient_atom(a, grid, cell, R, P)
        for c in range(3):
            d = 1e-5
            Rp = R.copy(); Rp[a, c] += d
            Rm = R.copy(); Rm[a, c] -= d
            fd = (O.dielectric(grid, cell, Rp) - O.dielectric(grid, cell, Rm)) / (2 * d)
            assert np.max(np.abs(fd - g[c])) < 1e-6 * max(1.0, np.max(np.abs(fd)))


# ------------------------------------------------------------ charge density

def test_gaussian_normalisation_and_neutrality():
    """h^3 sum g = 1 for a resolved Gaussian (Poisson summation: the error is
    exp(-2 pi^2 sigma^2/h^2)); the neutral rho sums to zero."""
    grid, cell = (32, 32, 32), (10.0, 10.0, 10.0)
    dv = O.cell_volume_element(grid, cell)
    pos = np.array([[3.3, 4.1, 5.7]])
    for sig in (0.5, 0.8, 1.0):
        rho = np.zeros((32, 32, 32))
        for sl, (dz, dy, dx) in O._image_boxes(pos[0], grid, cell, 8 * sig):
            d2 = dx * dx + dy * dy + dz * dz
            rho[sl] += O.gaussian(d2, sig)
        assert abs(dv * rho.sum() - 1.0) < 1e-9
    at, eps, rho = _small_slab()
    assert abs(rho.sum()) < 1e-10 * np.abs(rho).sum()


def test_charge_density_points_and_gradient():
    grid, cell = (12, 12, 14), (8.0, 8.0, 9.0)
    rng = np.random.default_rng(2)
    R = rng.uniform(0, 1, (3, 3)) * np.array(cell)
    Z = np.array([4.0, 6.0, 4.0]); sc = np.array([0.5, 0.6, 0.7]); se = np.array([0.8, 0.9, 0.75])
    raw = O.charge_density_raw(grid, cell, R, Z, sc, se)
    x, y, z = _grid_points(grid, cell)
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    assert np.max(np.abs(raw.ravel() - O.charge_density_points(pts, cell, R, Z, sc, se))) < 1e-11
    for a in range(3):
        g = O.charge_density_gradient_atom(a, grid, cell, R, Z, sc, se)
        for c in range(3):
            d = 1e-5
            Rp = R.copy(); Rp[a, c] += d
            Rm = R.copy(); Rm[a, c] -= d
            fd = (O.charge_density_raw(grid, cell, Rp, Z, sc, se)
                  - O.charge_density_raw(grid, cell, Rm, Z, sc, se)) / (2 * d)
            assert np.max(np.abs(fd - g[c])) < 1e-5 * max(1.0, np.max(np.abs(fd)))


# -------------------------------------------------------------- the operator

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_planar_closed_form(axis):
    """P2: rho and eps varying along one axis only. The discrete flux
    F_{k+1/2} = C - 4 pi h S_k (S_k = sum_{j<=k} rho_j), with C fixed by
    periodicity, C = 4 pi h sum(S_k/eps_{k+1/2}) / sum(1/eps_{k+1/2}),
    and phi_{k+1} - phi_k = h F_{k+1/2}/eps_{k+1/2}."""
    n = 48
    L = 12.0
    grid = [4, 4, 4]
    cellv = [3.0, 3.0, 3.0]
    grid[axis] = n
    cellv[axis] = L
    h = O.spacing(grid, cellv)
    hk = h[axis]
    t = np.arange(n) * hk
    r1 = np.exp(-((t - 4.0) / 0.7) ** 2) - np.exp(-((t - 7.5) / 1.1) ** 2) * 0.7 / 1.1
    r1 -= r1.mean()
    e1 = 1 + 30 * (1 + np.tanh((t - 6.0) / 0.8)) + 5 * np.sin(2 * np.pi * t / L) ** 2
    shape = (grid[2], grid[1], grid[0])
    bshape = [1, 1, 1]
    bshape[O.AX[axis]] = n
    rho = np.broadcast_to(r1.reshape(bshape), shape).copy()
    eps = np.broadcast_to(e1.reshape(bshape), shape).copy()
    phi, info = O.solve(rho, eps, h, tol=1e-14)
    ef = 0.5 * (e1 + np.roll(e1, -1))
    S = np.cumsum(r1)
    C = 4 * np.pi * hk * np.sum(S / ef) / np.sum(1 / ef)
    F = C - 4 * np.pi * hk * S
    dphi = hk * F / ef
    p1 = np.concatenate([[0.0], np.cumsum(dphi)[:-1]])
    p1 -= p1.mean()
    got = np.moveaxis(phi, O.AX[axis], 0)[:, 0, 0]
    assert np.max(np.abs(got - p1)) < 1e-10 * np.max(np.abs(p1))
    # closure: the last increment returns to the start
    assert abs(np.sum(dphi)) < 1e-12 * np.max(np.abs(p1))


def test_uniform_eps_scales_vacuum_solution():
    """P1: eps = c everywhere gives phi = phi_vac / c."""
    at, eps, rho = _small_slab()
    h = O.spacing((16, 16, 32), (10.0, 10.0, 20.0))
    vac = O.vacuum_potential(rho, h)
    for c in (1.0, 7.5, 78.36):
        phi, info = O.solve(rho, np.full_like(rho, c), h, tol=1e-14)
        assert np.max(np.abs(phi - vac / c)) < 1e-11 * np.max(np.abs(vac))


def _neutral_pair_potential(r, Z, s1, s2):
    """Free-space potential of +Z N(0,s1^2) and -Z N(0,s2^2): Z[erf(r/(s1 sqrt2)) - erf(r/(s2 sqrt2))]/r."""
    r = np.asarray(r)
    rs = np.where(r > 0, r, 1.0)
    v = Z * (erf(rs / (s1 * math.sqrt(2))) - erf(rs / (s2 * math.sqrt(2)))) / rs
    v0 = Z * math.sqrt(2 / math.pi) * (1 / s1 - 1 / s2)
    return np.where(r > 0, v, v0)


def test_gaussian_pair_in_vacuum_erf_potential():
    """P3: a neutral core/cloud pair in a large periodic box against its erf
    potential. The 7-point solution converges at O(h^2): error ratio ~4 per
    halving of h."""
    L = 16.0
    c = np.array([8.0, 8.0, 8.0])
    Z, s1, s2 = 3.0, 0.6, 0.9
    errs = []
    for n in (32, 64):
        grid, cell = (n, n, n), (L, L, L)
        h = O.spacing(grid, cell)
        rho = O.charge_density_raw(grid, cell, c[None], np.array([Z]), np.array([s1]), np.array([s2]))
        rho -= rho.mean()
        phi = O.vacuum_potential(rho, h)
        x, y, z = _grid_points(grid, cell)
        r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
        ref = _neutral_pair_potential(r, Z, s1, s2)
        ref -= ref.mean()
        errs.append(np.max(np.abs(phi - ref)) / np.max(np.abs(ref)))
    assert errs[1] < 0.02
    assert 3.3 < errs[0] / errs[1] < 4.7


def test_dense_direct_solve_8cubed():
    """P4: brute force. The dense 512x512 matrix (columns A e_j) with the
    rank-one gauge fix, solved by LAPACK, equals the PCG solution."""
    grid, cell = (8, 8, 8), (6.5, 6.5, 6.5)
    rng = np.random.default_rng(1)
    h = O.spacing(grid, cell)
    eps = 1 + 40 * rng.uniform(0, 1, (8, 8, 8))
    rho = rng.standard_normal((8, 8, 8))
    rho -= rho.mean()
    n = 512
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n); e[j] = 1
        M[:, j] = O.apply_A(e.reshape(8, 8, 8), eps, h).ravel()
    assert np.max(np.abs(M - M.T)) < 1e-12 * np.max(np.abs(M))       # symmetric
    assert np.max(np.abs(M.sum(axis=0))) < 1e-10 * np.max(np.abs(M))  # constants in the kernel
    x = np.linalg.solve(M - np.ones((n, n)) / n, -4 * np.pi * rho.ravel())
    phi, info = O.solve(rho, eps, h, tol=1e-15)
    assert np.max(np.abs(phi.ravel() - x)) < 1e-12 * np.max(np.abs(x))


def test_green_reciprocity_and_neutrality():
    """P5: rho1.phi2 = rho2.phi1 (A symmetric); P6: sum(A phi) = 0."""
    at, eps, _ = _small_slab()
    h = O.spacing((16, 16, 32), (10.0, 10.0, 20.0))
    rng = np.random.default_rng(4)
    r1 = rng.standard_normal(eps.shape); r1 -= r1.mean()
    r2 = rng.standard_normal(eps.shape); r2 -= r2.mean()
    p1, _ = O.solve(r1, eps, h)
    p2, _ = O.solve(r2, eps, h)
    a, b = float(np.sum(r1 * p2)), float(np.sum(r2 * p1))
    assert abs(a - b) < 1e-11 * max(abs(a), abs(b))
    q = O.apply_A(rng.standard_normal(eps.shape), eps, h)
    assert abs(q.sum()) < 1e-10 * np.abs(q).sum()


def test_eps_one_solve_equals_fft():
    """P7: with eps = 1 the generalized solve and the FFT solve coincide."""
    at, eps, rho = _small_slab()
    h = O.spacing((16, 16, 32), (10.0, 10.0, 20.0))
    phi, _ = O.solve(rho, np.ones_like(rho), h, tol=1e-15)
    vac = O.vacuum_potential(rho, h)
    assert np.max(np.abs(phi - vac)) < 1e-12 * np.max(np.abs(vac))


def test_energy_identity():
    """P8: 1/2 h^3 rho.phi = h^3/(8 pi) sum_f eps_f (grad_f phi)^2 at the
    solution (discrete integration by parts, Eq. 4); J equals E."""
    grid, cell = (16, 16, 32), (10.0, 10.0, 20.0)
    at, eps, rho = _small_slab()
    h = O.spacing(grid, cell)
    phi, info = O.solve(rho, eps, h, tol=1e-14)
    E = O.energy(rho, phi, grid, cell)
    E2 = O.field_energy(phi, eps, grid, cell)
    J = O.variational_energy(rho, phi, eps, grid, cell)
    assert abs(E - E2) < 1e-11 * abs(E)
    assert abs(E - J) < 1e-11 * abs(E)
    assert E > 0


def test_manufactured_solution_second_order():
    """P11 (the paper's accuracy test with a smooth profile): phi = exp(-a r^2),
    eps = 1 + beta exp(-b r^2); rho = -div(eps grad phi)/(4 pi) analytically.
    The discrete solution converges at O(h^2)."""
    a, b, beta = 0.9, 0.6, 20.0
    L = 14.0
    c = np.array([7.0, 7.0, 7.0])
    errs = []
    for n in (28, 56):
        grid, cell = (n, n, n), (L, L, L)
        h = O.spacing(grid, cell)
        x, y, z = _grid_points(grid, cell)
        X, Y, Zc = x - c[0], y - c[1], z - c[2]
        r2 = X * X + Y * Y + Zc * Zc
        ph = np.exp(-a * r2)
        eb = np.exp(-b * r2)
        eps = 1 + beta * eb
        lap = (4 * a * a * r2 - 6 * a) * ph
        gradeps_dot_gradphi = (-2 * b * beta * eb) * (-2 * a * ph) * r2
        div = gradeps_dot_gradphi + eps * lap
        rho = -div / (4 * np.pi)
        rho -= rho.mean()
        phi, info = O.solve(rho, eps, h, tol=1e-13)
        ref = ph - ph.mean()
        errs.append(np.max(np.abs(phi - ref)))
    assert errs[1] < 0.03
    assert 3.3 < errs[0] / errs[1] < 4.7


# ------------------------------------------------------------------- forces

@pytest.mark.parametrize("rho_moves", [False, True])
def test_forces_match_central_differences(rho_moves):
    """P9: dE/dR_a from Eq. 11 (discrete) against central differences of the
    variational energy J, for three atoms; rho frozen (eps term only) or moving
    with its atoms (both terms)."""
    grid, cell = (16, 16, 24), (8.0, 8.0, 12.0)
    at = W.slab_atoms(cell, 2, 2, seed=1)
    h = O.spacing(grid, cell)
    pos = at.pos

    def E_of(p):
        eps = O.dielectric(grid, cell, p)
        src = p if rho_moves else pos
        rho = O.charge_density(grid, cell, src, at.Z, at.sigma_core, at.sigma_cloud)
        phi, _ = O.solve(rho, eps, h, tol=1e-14)
        return O.variational_energy(rho, phi, eps, grid, cell)

    eps = O.dielectric(grid, cell, pos)
    rho = O.charge_density(grid, cell, pos, at.Z, at.sigma_core, at.sigma_cloud)
    phi, _ = O.solve(rho, eps, h, tol=1e-14)
    sel = [0, 3, 5]
    Ge, Gr = O.energy_gradient(phi, grid, cell, pos, at.Z, at.sigma_core, at.sigma_cloud,
                               atoms=sel, rho_moves=rho_moves)
    G = Ge + Gr
    fd = np.zeros((len(sel), 3))
    d = 1e-4
    for t, a in enumerate(sel):
        for c in range(3):
            pp = pos.copy(); pp[a, c] += d
            pm = pos.copy(); pm[a, c] -= d
            fd[t, c] = (E_of(pp) - E_of(pm)) / (2 * d)
    scale = np.max(np.abs(fd))
    assert scale > 1e-3
    assert np.max(np.abs(fd - G[sel])) < 1e-6 * scale


def test_vacuum_force_between_gaussian_atoms_closed_form():
    """P12 (the eps = 1 limit of Eq. 11, the Hartree force of Eq. 14): two
    neutral atoms, each a +Z core and a -Z cloud Gaussian, interact through
    E_int(R) = sum_ij q_i q_j erf(R/s_ij)/R with s_ij = sqrt(2(sigma_i^2 + sigma_j^2)),
    since a spherically symmetric neutral charge has no field outside itself
    (images decay like erfc). The discrete gradient G^rho of Eq. 11 converges
    to dE_int/dR_a at O(h^2)."""
    L = 16.0
    pos = np.array([[8.1, 7.9, 8.3], [9.3, 8.6, 7.5]])
    Z = np.array([4.0, 6.0])
    sc, scl = np.array([0.5, 0.55]), np.array([0.9, 1.0])
    d = pos[0] - pos[1]
    R = np.linalg.norm(d)
    dE = 0.0
    for qi, si in ((Z[0], sc[0]), (-Z[0], scl[0])):
        for qj, sj in ((Z[1], sc[1]), (-Z[1], scl[1])):
            s = math.sqrt(2.0 * (si * si + sj * sj))
            dE += qi * qj * (2.0 / math.sqrt(math.pi) * math.exp(-(R / s) ** 2) / (s * R) - erf(R / s) / R ** 2)
    G_exact = dE * d / R
    errs = []
    for n in (48, 96):
        grid, cell = (n, n, n), (L, L, L)
        h = O.spacing(grid, cell)
        rho = O.charge_density(grid, cell, pos, Z, sc, scl)
        phi = O.vacuum_potential(rho, h)
        Ge, Gr = O.energy_gradient(phi, grid, cell, pos, Z, sc, scl, p=O.DielectricParams(eps0=1.0), atoms=[0])
        assert np.max(np.abs(Ge)) == 0.0                    # no dielectric term at eps = 1
        errs.append(np.linalg.norm(Gr[0] - G_exact) / np.linalg.norm(G_exact))
    assert errs[1] < 5e-3, errs
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


# -------------------------------------------------------------- dry/wet split

def test_plan_band_brute_force():
    """The band planner on hand-made dry flags."""
    dry = np.zeros(32, dtype=bool)
    dry[10:17] = True                       # run of 7 dry planes, 10..16
    assert O.plan_band(dry, levels=3, n_dirichlet=1) == (13, 1)
    assert O.plan_band(dry, levels=3, n_dirichlet=0) == (11, 5)   # 1 + 4m <= 7 -> 5
    assert O.plan_band(dry, levels=2, n_dirichlet=0) == (10, 7)   # 1 + 2m <= 7 -> 7
    wrap = np.zeros(32, dtype=bool)
    wrap[[30, 31, 0, 1, 2]] = True          # run wraps through z = 0
    assert O.plan_band(wrap, levels=2, n_dirichlet=0) == (30, 5)
    assert O.plan_band(wrap, levels=3, n_dirichlet=1) == (0, 1)
    assert O.plan_band(np.zeros(8, dtype=bool), 2) is None
    assert O.band_planes(8, 6, 3) == [1, 2, 3, 4, 5]


def test_split_fixed_point_equals_full_box():
    """P10: the self-consistent dry/wet iteration converges to the full-box
    solution; its first pass is the paper's one-shot Scheme 1."""
    grid, cell = (16, 16, 32), (10.0, 10.0, 20.0)
    at, eps, rho = _small_slab(grid, cell, n=2, layers=3)
    h = O.spacing(grid, cell)
    dry = O.dry_planes(eps)
    band = O.plan_band(dry, levels=2, n_dirichlet=1)
    assert band is not None
    full, _ = O.solve(rho, eps, h, tol=1e-14)
    split, hist = O.split_solve(rho, eps, h, band, tol=1e-13)
    assert hist[-1] < 1e-12
    assert np.max(np.abs(split - full)) < 1e-10 * np.max(np.abs(full))
    # the one-shot scheme (one band solve on the vacuum potential's Dirichlet
    # data) is a close approximation but not the solution: the reason the
    # coupling is iterated to self-consistency
    one, _ = O.split_solve(rho, eps, h, band, tol=1e-13, maxit=1)
    err1 = np.max(np.abs(one - full)) / np.max(np.abs(full))
    err_vac = np.max(np.abs(O.vacuum_potential(rho, h) - full)) / np.max(np.abs(full))
    assert 1e-4 < err1 < 1e-2 and err1 < 0.1 * err_vac


# -------------------------------------------------------------- Eq. 9-10 dielectric

def _radii(Z):
    return W.vdw_radii(Z)


def test_gamma_dielectric_is_centred_on_the_vdw_radius():
    """Eq. 10: one atom, a point at |r - R| = Rvdw has gamma = 1 and eps = (1 + eps0)/2
    whatever beta; eps grows monotonically with the distance along a ray."""
    # a 40 A cell, so that the other images add below 1e-15 to gamma at the point
    grid, cell = (80, 80, 80), (40.0, 40.0, 40.0)          # h = 0.5
    pos = np.array([[20.0, 20.0, 20.0]])
    rv = np.array([1.5])
    for beta in (1.0, 2.4, 4.0):
        p = O.GammaParams(beta=beta)
        eps = O.dielectric_gamma(grid, cell, pos, rv, p)
        assert abs(eps[40, 40, 43] - 0.5 * (1.0 + p.eps0)) < 1e-12     # x = 21.5: d = 1.5
        ray = eps[40, 40, 40:54]
        assert np.all(np.diff(ray) > 0)
        assert ray[0] < 1.0 + 0.1 * (p.eps0 - 1.0) and ray[-1] > p.eps0 - 1e-2


def test_gamma_dielectric_printed_form_equals_simplified_form():
    """Eq. 10 as printed, 1 + (eps0-1)/2 (1 + (1 - t)/(1 + t)), equals 1 + (eps0-1)/(1 + t),
    t = gamma^(2 beta), which is the form the CUDA kernel evaluates."""
    rng = np.random.default_rng(3)
    g = np.concatenate([rng.uniform(0, 3, 200), [0.0, 1.0, 1e-8, 50.0]])
    p = O.GammaParams()
    simple = 1.0 + (p.eps0 - 1.0) / (1.0 + g ** (2 * p.beta))
    assert np.max(np.abs(O.eps_of_gamma(g, p) - simple)) < 1e-12 * p.eps0


def test_gamma_dielectric_grid_equals_the_point_evaluator():
    """Bounding-box images of the grid builder against the one-by-one evaluator."""
    grid, cell = (12, 10, 14), (8.0, 7.0, 9.0)
    at = W.slab_atoms(cell, 2, 1, seed=4)
    rv = _radii(at.Z)
    p = O.GammaParams()
    eps = O.dielectric_gamma(grid, cell, at.pos, rv, p)
    x, y, z = _grid_points(grid, cell)
    pts = np.stack([np.broadcast_to(x, eps.shape).ravel(), np.broadcast_to(y, eps.shape).ravel(),
                    np.broadcast_to(z, eps.shape).ravel()], axis=1)
    ref = O.dielectric_gamma_points(pts, cell, at.pos, rv, p).reshape(eps.shape)
    assert np.max(np.abs(eps - ref)) < 1e-12 * p.eps0


def test_gamma_dielectric_gradient_matches_fd_and_fixes_eq12_sign():
    """d eps/d R_a against central differences of the grid eps; the printed Eq. 12
    (positive prefactor) has the opposite sign of the finite differences."""
    grid, cell = (16, 16, 16), (8.0, 8.0, 8.0)
    pos = np.array([[3.1, 4.2, 3.9], [5.0, 3.3, 4.6]])
    rv = np.array([1.52, 2.0])
    p = O.GammaParams()
    G = O.dummy_density(grid, cell, pos, rv, p)
    de = O.dielectric_gamma_gradient_atom(0, grid, cell, pos, rv, G, p)
    d = 1e-5
    for c in range(3):
        pp = pos.copy(); pp[0, c] += d
        pm = pos.copy(); pm[0, c] -= d
        fd = (O.dielectric_gamma(grid, cell, pp, rv, p) - O.dielectric_gamma(grid, cell, pm, rv, p)) / (2 * d)
        scale = np.max(np.abs(fd))
        assert scale > 1.0
        assert np.max(np.abs(fd - de[c])) < 1e-6 * scale
        assert float(np.sum(fd * (-de[c]))) < 0          # the printed sign disagrees with the FD


def test_gamma_forces_match_central_differences():
    """P9 for the Eq. 9-10 dielectric: dE/dR_a (eps term, rho frozen) against central
    differences of the variational energy J (E(R) is smooth: the image sum's
    cut-off drops terms below 1e-17)."""
    grid, cell = (16, 16, 24), (8.0, 8.0, 12.0)
    at = W.slab_atoms(cell, 1, 2, seed=1)
    rv = _radii(at.Z)
    p = O.GammaParams()
    h = O.spacing(grid, cell)
    pos = at.pos
    rho = O.charge_density(grid, cell, pos, at.Z, at.sigma_core, at.sigma_cloud)

    def E_of(q):
        eps = O.dielectric_gamma(grid, cell, q, rv, p)
        phi, _ = O.solve(rho, eps, h, tol=1e-14)
        return O.variational_energy(rho, phi, eps, grid, cell)

    eps = O.dielectric_gamma(grid, cell, pos, rv, p)
    phi, _ = O.solve(rho, eps, h, tol=1e-14)
    sel = [0, 3]
    Ge, Gr = O.energy_gradient(phi, grid, cell, pos, at.Z, at.sigma_core, at.sigma_cloud, p=p, atoms=sel,
                               rho_moves=False, rvdw=rv)
    fd = np.zeros((len(sel), 3))
    d = 1e-4
    for t, a in enumerate(sel):
        for c in range(3):
            pp = pos.copy(); pp[a, c] += d
            pm = pos.copy(); pm[a, c] -= d
            fd[t, c] = (E_of(pp) - E_of(pm)) / (2 * d)
    scale = np.max(np.abs(fd))
    assert scale > 1e-3
    assert np.max(np.abs(fd - Ge[sel])) < 1e-6 * scale


# -------------------------------------------------------------- Eq. 19 solvent exclusion

def _eq19_case(seed=0, n=2):
    grid, cell = (16, 16, 32), (8.0, 8.0, 16.0)
    at = W.slab_atoms(cell, n, 3, seed=seed)
    zs = np.sort(at.pos[:, 2])
    zlim = 0.5 * (zs[len(zs) // 3 - 1] + zs[len(zs) // 3])  # between layers 1 and 2: layer 1 is lower
    return grid, cell, at, W.vdw_radii(at.Z), zlim


def test_eq19_without_lower_atoms_is_eq10():
    """With z_lim below every atom, Eq. 19 is Eq. 9 term by term."""
    grid, cell, at, rv, _ = _eq19_case()
    p = O.GammaParams()
    a = O.dielectric_eq19(grid, cell, at.pos, rv, -1.0, p)
    b = O.dielectric_gamma(grid, cell, at.pos, rv, p)
    assert np.max(np.abs(a - b)) < 1e-12 * p.eps0


def test_eq19_dries_the_region_below_the_lower_layer():
    """Below the lower atoms eps saturates to 1 (dry planes); far above the slab
    it is the solvent's eps0; with Eq. 10 alone the region below stays wet."""
    grid, cell, at, rv, zlim = _eq19_case()
    p = O.GammaParams()
    eps = O.dielectric_eq19(grid, cell, at.pos, rv, zlim, p)
    pm = (eps - 1.0).reshape(grid[2], -1).max(axis=1)
    zmin = at.pos[:, 2].min()
    h = O.spacing(grid, cell)[2]
    below = [k for k in range(grid[2]) if k * h < zmin - 3.0]
    assert below and np.all(pm[below] < 1e-6)
    assert O.dielectric_gamma(grid, cell, at.pos, rv, p).reshape(grid[2], -1).max(axis=1)[below[0]] > 1.0
    zmax = at.pos[:, 2].max()
    above = [k for k in range(grid[2]) if zmax + 5.0 < k * h < cell[2] - 1.0]
    assert above and np.all(eps.reshape(grid[2], -1)[above].min(axis=1) > p.eps0 - 0.1)


def test_eq19_sign_is_plus_on_the_atom_plane():
    """At z = z_I a lower atom's term decays (the sign factor is +1 there)."""
    grid, cell = (16, 16, 16), (8.0, 8.0, 8.0)
    pos = np.array([[4.0, 4.0, 4.0]])                      # on grid point (8, 8, 8)
    rv = np.array([1.5])
    p = O.GammaParams()
    eps19 = O.dielectric_eq19(grid, cell, pos, rv, 5.0, p)
    eps10 = O.dielectric_gamma(grid, cell, pos, rv, p)
    assert np.max(np.abs(eps19[8] - eps10[8])) < 1e-13 * p.eps0      # the plane z = z_I
    x, y, z = _grid_points(grid, cell)
    d = np.sqrt((x - 4.0) ** 2 + (y - 4.0) ** 2 + (z - 4.0) ** 2)
    out = np.broadcast_to((z < 4.0) & (d > rv[0]), eps19.shape)
    assert np.all(eps19[out] <= eps10[out])                      # below, outside the vdW sphere: drier


def test_eq19_gradient_matches_fd():
    """d eps/d R for both branches against central differences (the atom's z is
    away from grid planes, so no point changes side)."""
    grid, cell, at, rv, zlim = _eq19_case(seed=2, n=1)
    p = O.GammaParams()
    pos = at.pos.copy()
    a = int(np.argmin(pos[:, 2]))                              # a lower atom
    G, S = O.dummy_density_eq19(grid, cell, pos, rv, zlim, p)
    de = O.dielectric_eq19_gradient_atom(a, grid, cell, pos, rv, zlim, G, S, p)
    d = 1e-4
    for c in range(3):
        pp = pos.copy(); pp[a, c] += d
        pm = pos.copy(); pm[a, c] -= d
        fd = (O.dielectric_eq19(grid, cell, pp, rv, zlim, p) - O.dielectric_eq19(grid, cell, pm, rv, zlim, p)) / (2 * d)
        scale = np.max(np.abs(fd))
        assert scale > 0.1
        assert np.max(np.abs(fd - de[c])) < 1e-6 * scale


def test_eq19_forces_match_central_differences():
    """P9 for Eq. 19: dE/dR_a (eps term, rho frozen) against central differences of J."""
    grid, cell, at, rv, zlim = _eq19_case(seed=1, n=1)
    p = O.GammaParams()
    h = O.spacing(grid, cell)
    pos = at.pos
    rho = O.charge_density(grid, cell, pos, at.Z, at.sigma_core, at.sigma_cloud)

    def E_of(q):
        eps = O.dielectric_eq19(grid, cell, q, rv, zlim, p)
        phi, _ = O.solve(rho, eps, h, tol=1e-14)
        return O.variational_energy(rho, phi, eps, grid, cell)

    eps = O.dielectric_eq19(grid, cell, pos, rv, zlim, p)
    phi, _ = O.solve(rho, eps, h, tol=1e-14)
    sel = [int(np.argmin(pos[:, 2])), int(np.argmax(pos[:, 2]))]
    Ge, _ = O.energy_gradient(phi, grid, cell, pos, at.Z, at.sigma_core, at.sigma_cloud, p=p, atoms=sel,
                              rho_moves=False, rvdw=rv, zlim=zlim)
    fd = np.zeros((len(sel), 3))
    d = 1e-4
    for t, a in enumerate(sel):
        for c in range(3):
            pp = pos.copy(); pp[a, c] += d
            pm = pos.copy(); pm[a, c] -= d
            fd[t, c] = (E_of(pp) - E_of(pm)) / (2 * d)
    scale = np.max(np.abs(fd))
    assert scale > 1e-3
    assert np.max(np.abs(fd - Ge[sel])) < 1e-6 * scale
