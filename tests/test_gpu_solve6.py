"""GPU parity of the sixth-order solve, its adjoint and its forces (Sec. III,
Eq. 16-18; Eq. 11 through the adjoint, Appendix B) through the C ABI
(gp_solve6, gp_adjoint6, gp_energy_forces6) against the oracle's solve6,
adjoint6 and energy_gradient6, and against central differences of the
library's own energy.

Tolerances: phi and lam within 1e-10 of their largest value (both sides solve
to 1e-13 or below); the residual of the returned (phi, mu), measured by the
oracle's operator, at the requested tolerance; forces within 1e-8 of the
oracle's gradient evaluated on the same fields (FP64; the dielectric force
kernels evaluate their per-pair terms in df64, ~1e-12), and within 1e-8 of the
oracle's own solution's gradient; central differences (h = 1e-4 A) within
1e-6 of the largest component.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import gp_oracle as O

pytestmark = pytest.mark.gpu

DEV = "cuda"

CASES = [((8, 8, 8), (6.5, 6.5, 6.5), 1, 1),          # the smallest grid the library takes
         ((32, 32, 64), (10.0, 10.0, 20.0), 2, 3),      # the 32x32x64 workload
         ((48, 16, 24), (14.0, 7.0, 12.0), 1, 2)]       # anisotropic, 3 * 2^k extents


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
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _case(k, seed=0):
    grid, cell, n, layers = CASES[k]
    at = W.slab_atoms(cell, n, layers, seed=seed + k)
    h = O.spacing(grid, cell)
    eps = O.dielectric(grid, cell, at.pos)
    rho = O.charge_density(grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    return grid, cell, at, h, eps, rho


@pytest.fixture(scope="module")
def oracle_cases():
    out = []
    for k in range(len(CASES)):
        grid, cell, at, h, eps, rho = _case(k)
        phi, mu, info = O.solve6(rho, eps, h, tol=1e-14)
        lam, nu, info_t = O.adjoint6(rho, eps, h, tol=1e-14)
        out.append((grid, cell, at, h, eps, rho, phi, mu, lam, nu, info, info_t))
    return out


@pytest.mark.parametrize("k", range(len(CASES)))
@pytest.mark.parametrize("precision", [0, 1])
def test_solve6_matches_oracle(oracle_cases, k, precision):
    GPSolver = _gpu()
    grid, cell, at, h, eps, rho, phi_o, mu_o, _, _, info, _ = oracle_cases[k]
    assert info.residual < 1e-12
    s = GPSolver(grid, cell, precision=precision)
    s.set_atoms(_t(at.pos))
    phi, mu = s.solve6(_t(rho), tol=1e-13)
    p = phi.cpu().numpy()
    st = s.stats()
    assert st.residual <= 1e-13
    assert O.residual6_norm(p, mu, rho, eps, h) < 2e-13          # measured by the oracle's operator
    assert _rel(p, phi_o) < 1e-10
    assert abs(float(p.mean())) < 1e-14 * np.max(np.abs(p))      # sum(phi) = 0
    assert abs(mu - mu_o) <= 1e-9 * abs(mu_o) + 1e-13 * np.max(np.abs(4 * np.pi * rho))
    # warm start from the answer: one residual evaluation, no Krylov step
    s.solve6(_t(rho), phi=phi, tol=1e-12)
    assert s.stats().outer_iterations == 1 and s.stats().inner_iterations == 0


@pytest.mark.parametrize("k", range(len(CASES)))
@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint6_matches_oracle(oracle_cases, k, precision):
    GPSolver = _gpu()
    grid, cell, at, h, eps, rho, _, _, lam_o, nu_o, _, info_t = oracle_cases[k]
    assert info_t.residual < 1e-12
    s = GPSolver(grid, cell, precision=precision)
    s.set_atoms(_t(at.pos))
    lam, nu = s.adjoint6(_t(rho), tol=1e-13)
    l = lam.cpu().numpy()
    assert s.stats().residual <= 1e-13
    rt = (rho - rho.mean()) - O.apply_A6_transpose(l, eps, h) - nu
    # the library's eps agrees with the oracle's to 1e-13 of its maximum, which
    # alone moves A6^T lam by ~1e-12 of rho here (7e-13 measured on the
    # anisotropic grid): the residual the oracle measures is held to 3e-12
    assert np.linalg.norm(rt) < 3e-12 * np.linalg.norm(rho - rho.mean())
    assert abs(float(np.sum(eps * l))) < 1e-12 * float(np.sum(np.abs(eps * l)))
    assert _rel(l, lam_o) < 1e-10
    assert abs(nu - nu_o) <= 1e-9 * abs(nu_o) + 1e-13 * np.max(np.abs(rho))


@pytest.mark.parametrize("k", [1, 2])
def test_forces6_match_oracle_gradient(oracle_cases, k):
    """Both force terms: the library's forces on its own (phi, mu, lam) against
    energy_gradient6 on the same fields, and against the oracle's gradient on
    the oracle's own solution."""
    GPSolver = _gpu()
    grid, cell, at, h, eps, rho, phi_o, mu_o, lam_o, _, _, _ = oracle_cases[k]
    s = GPSolver(grid, cell, precision=0)
    s.set_atoms(_t(at.pos))
    rho_t = _t(rho)
    phi, mu = s.solve6(rho_t, tol=1e-13)
    lam, _ = s.adjoint6(rho_t, tol=1e-13)
    E, F = s.energy_forces6(phi, mu, lam, rho_t, _t(_gauss(at)))
    p, l = phi.cpu().numpy(), lam.cpu().numpy()
    Ge, Gr = O.energy_gradient6(p, mu, l, grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    F = F.cpu().numpy()
    assert _rel(F, -(Ge + Gr)) < 1e-8
    Ge_o, Gr_o = O.energy_gradient6(phi_o, mu_o, lam_o, grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    assert _rel(F, -(Ge_o + Gr_o)) < 1e-8
    Eo = O.energy(rho - rho.mean(), phi_o, grid, cell)
    assert abs(E - Eo) < 1e-10 * abs(Eo)
    # the solvent term alone (rho held fixed)
    _, Fe = s.energy_forces6(phi, mu, lam, rho_t, None)
    assert _rel(Fe.cpu().numpy(), -Ge) < 1e-8


def test_forces6_gamma_dielectric_match_oracle_gradient():
    """The same forces with the dielectric of Eq. 9-10 (the gamma branch)."""
    GPSolver = _gpu()
    grid, cell = (32, 32, 48), (10.0, 10.0, 15.0)
    at = W.slab_atoms(cell, 2, 3, seed=2)
    rv = W.vdw_radii(at.Z)
    p = O.GammaParams()
    h = O.spacing(grid, cell)
    rho = O.charge_density(grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    s = GPSolver(grid, cell, precision=0, kind=1)
    s.set_atoms(_t(at.pos), radii=_t(rv))
    rho_t = _t(rho)
    phi, mu = s.solve6(rho_t, tol=1e-13)
    lam, _ = s.adjoint6(rho_t, tol=1e-13)
    _, F = s.energy_forces6(phi, mu, lam, rho_t, _t(_gauss(at)))
    Ge, Gr = O.energy_gradient6(phi.cpu().numpy(), mu, lam.cpu().numpy(), grid, cell, at.pos, at.Z,
                                at.sigma_core, at.sigma_cloud, p=p, rvdw=rv)
    assert _rel(F.cpu().numpy(), -(Ge + Gr)) < 1e-8


@pytest.mark.parametrize("rho_moves", [False, True])
def test_forces6_match_central_differences(rho_moves):
    """-dE/dR from the adjoint against central differences (h = 1e-4 A) of the
    library's own sixth-order energy on 4 seeded atoms, every step on the GPU:
    rho frozen (the solvent term) and rho moving with its atoms (both terms)."""
    GPSolver = _gpu()
    grid, cell = (32, 32, 64), (10.0, 10.0, 20.0)
    at = W.slab_atoms(cell, 2, 3, seed=4)
    gauss = _t(_gauss(at))
    s = GPSolver(grid, cell, precision=0)
    rho0 = s.build_rho(_t(at.pos), gauss)

    def energy(q):
        qt = _t(q)
        s.set_atoms(qt)
        rho = s.build_rho(qt, gauss) if rho_moves else rho0
        phi, mu = s.solve6(rho, tol=1e-13)
        E, _ = s.energy_forces6(phi, mu, None, rho, forces=False)
        return E

    s.set_atoms(_t(at.pos))
    phi, mu = s.solve6(rho0, tol=1e-13)
    lam, _ = s.adjoint6(rho0, tol=1e-13)
    _, F = s.energy_forces6(phi, mu, lam, rho0, gauss if rho_moves else None)
    F = F.cpu().numpy()
    sel = np.random.default_rng(9).choice(len(at.pos), 4, replace=False)
    d = 1e-4
    fd = np.zeros((len(sel), 3))
    for t_, a in enumerate(sel):
        for c in range(3):
            pp = at.pos.copy(); pp[a, c] += d
            pm = at.pos.copy(); pm[a, c] -= d
            fd[t_, c] = -(energy(pp) - energy(pm)) / (2 * d)
    scale = np.max(np.abs(fd))
    assert scale > 1e-3
    assert np.max(np.abs(fd - F[sel])) < 1e-6 * scale


def test_solve6_errors():
    GPSolver = _gpu()
    from paper_0904_4887_gb300 import GPError
    s = GPSolver((16, 16, 16), (8.0, 8.0, 8.0))
    z = s.zeros()
    with pytest.raises(GPError) as e:
        s.solve6(z)                                         # no dielectric yet
    assert e.value.status == 8
    s.set_atoms(torch.zeros((0, 3), dtype=torch.float64, device=DEV))
    with pytest.raises(GPError) as e:
        s.solve6(z, tol=0.0)
    assert e.value.status == 1
    one = torch.ones_like(z)
    with pytest.raises(GPError) as e:
        s.solve6(one)                                       # not neutral
    assert e.value.status == 2
    phi, mu = s.solve6(z)                                   # b = 0: phi = 0
    assert float(phi.abs().max()) == 0.0 and mu == 0.0
