"""Pins for the oracle's low-level helpers, each against a fact that does not
come from the helper itself: closed forms, symmetries, finite differences,
eigenfunctions, and brute force through a differently written operator."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import gp_oracle as O  # noqa: E402


def test_switching_symmetry_and_closed_form():
    """s(d) = (1 + erf((d - r0)/w))/2: one half at r0, s(r0+x) + s(r0-x) = 1
    (erf is odd), and s(0) = erfc(r0/w)/2 from the standard library."""
    p = O.DielectricParams()
    assert O.switching(np.array([p.r0]), p)[0] == 0.5
    x = np.random.default_rng(0).uniform(0.0, 3.0, 50)
    s = O.switching(p.r0 + x, p) + O.switching(p.r0 - x, p)
    assert np.max(np.abs(s - 1.0)) < 1e-15
    # (1 + erf)/2 is exact to half an ulp of 1 in absolute terms, so it meets erfc/2 to ~1e-16
    assert abs(O.switching(np.array([0.0]), p)[0] - 0.5 * math.erfc(p.r0 / p.w)) < 2e-16
    assert np.all(np.diff(O.switching(np.linspace(0.0, 6.0, 200), p)) >= 0.0)


def test_switching_derivative_matches_central_differences():
    p = O.DielectricParams()
    d = np.linspace(0.5, 5.5, 41)
    e = 1e-6
    fd = (O.switching(d + e, p) - O.switching(d - e, p)) / (2 * e)
    assert np.max(np.abs(fd - O.switching_derivative(d, p))) < 1e-8


def _lattice_count(r, cell, point, center):
    """Images center + nL within distance r of `point`, counted one by one."""
    L = np.asarray(cell)
    K = [int(math.ceil((r + L[a]) / L[a])) + 1 for a in range(3)]
    n = 0
    for i in range(-K[0], K[0] + 1):
        for j in range(-K[1], K[1] + 1):
            for k in range(-K[2], K[2] + 1):
                d = point - (center + np.array([i, j, k]) * L)
                n += float(np.sqrt(d @ d)) <= r
    return n


def test_image_count_bound_holds():
    """The counting step of gamma_tail_bound: at most (4 pi/3)(r + c)^3 / V
    images of an atom lie within r of any point (c = half the cell diagonal),
    checked by counting lattice points one by one."""
    cell = (3.0, 4.0, 5.5)
    V = cell[0] * cell[1] * cell[2]
    c = 0.5 * math.sqrt(sum(x * x for x in cell))
    rng = np.random.default_rng(2)
    for r in (0.5, 2.0, 7.0, 13.0):
        for _ in range(3):
            pt, ce = rng.uniform(0, 1, 3) * cell, rng.uniform(0, 1, 3) * cell
            assert _lattice_count(r, cell, pt, ce) <= 4.0 * math.pi / 3.0 * (r + c) ** 3 / V


def test_gamma_cutoff_is_the_smallest_radius_meeting_the_tail():
    """gamma_cutoff returns a radius whose bound is at most the tail, while a
    radius 1e-5 A shorter is not; the bound falls with the radius."""
    cell = (10.0, 10.0, 20.0)
    rv = np.array([2.0, 1.52, 1.52, 2.0])
    for tail in (1e-6, 1e-10, 1e-13):
        rc = O.gamma_cutoff(cell, rv, tail)
        assert O.gamma_tail_bound(rc, cell, rv) <= tail < O.gamma_tail_bound(rc - 1e-5, cell, rv)
    r = np.linspace(1.0, 60.0, 100)
    b = [O.gamma_tail_bound(x, cell, rv) for x in r]
    assert np.all(np.diff(b) < 0)


def test_gamma_tail_is_within_its_bound_against_a_larger_brute_force_sum():
    """gamma (Eq. 9) from the oracle's tail-bounded image sum against an
    independent brute-force sum over every image within the cut-off + 12 A, at
    random points of a small cell: they differ by less than the stated bound
    (the neglected tail), and the difference is not negligible compared with
    it (the bound is not vacuous by orders of magnitude)."""
    cell = (6.0, 5.0, 7.0)
    pos = np.array([[1.0, 2.0, 3.0], [4.2, 0.7, 6.1], [3.3, 3.9, 0.4]])
    rv = np.array([2.0, 1.52, 1.7])
    for tail in (1e-6, 1e-13):
        p = O.GammaParams(tail=tail)
        rc = O.gamma_cutoff(cell, rv, tail)
        pts = np.random.default_rng(7).uniform(0.0, 1.0, (6, 3)) * np.asarray(cell)
        eps = O.dielectric_gamma_points(pts, cell, pos, rv, p)
        R = rc + 12.0
        L = np.asarray(cell)
        K = [int(math.ceil((R + L[a]) / L[a])) + 1 for a in range(3)]
        ii, jj, kk = np.meshgrid(*[np.arange(-K[a], K[a] + 1) for a in range(3)], indexing="ij")
        shifts = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1) * L
        for m, pt in enumerate(pts):
            g = 0.0
            for R0, r0 in zip(pos, rv):
                d = np.linalg.norm(pt - (R0 + shifts), axis=1)
                g += float(np.sum(np.exp(r0 - d[d < R])))
            # invert Eq. 10 for the oracle's gamma: eps = 1 + (eps0-1)/(1 + gamma^(2 beta))
            go = ((p.eps0 - 1.0) / (eps[m] - 1.0) - 1.0) ** (1.0 / (2.0 * p.beta))
            diff = g - go
            assert -1e-13 * g <= diff <= O.gamma_tail_bound(rc, cell, rv) + 1e-13 * g
        if tail == 1e-6:
            assert diff > 1e-4 * tail          # the neglected tail is real at this tolerance


def test_deps_dgamma_matches_the_complex_step_derivative():
    """d eps/d gamma against Im eps(gamma + i delta)/delta, which has no
    cancellation (eps sits near eps0 at small gamma, where a real difference
    loses most digits)."""
    p = O.GammaParams()
    g = np.array([0.05, 0.3, 0.9, 1.0, 1.7, 4.0])
    delta = 1e-30
    cs = np.imag(O.eps_of_gamma(g + 1j * delta, p)) / delta
    assert np.max(np.abs(cs - O.deps_dgamma(g, p)) / np.abs(cs)) < 1e-13
    assert O.deps_dgamma(np.array([0.0]), p)[0] == 0.0


def test_saturation_exponent_leaves_eps_minus_one_below_1e16():
    p = O.GammaParams()
    gamma = math.exp(O.sat_exponent(p))
    assert O.eps_of_gamma(np.array([gamma]), p)[0] - 1.0 < 1e-16


def test_min_image_is_congruent_and_centred():
    L = 7.3
    dv = np.random.default_rng(1).uniform(-30.0, 30.0, 200)
    m = O._min_image(dv, L)
    assert np.all(np.abs(m) <= L / 2 + 1e-12)
    k = (dv - m) / L
    assert np.max(np.abs(k - np.round(k))) < 1e-12


def test_laplacian_symbol_is_the_eigenvalue_of_plane_waves():
    """cos(2 pi k.x) is an eigenfunction of the periodic 7-point Laplacian; its
    eigenvalue from apply_L (real space) equals the symbol entry."""
    grid = (8, 6, 10)
    h = (0.3, 0.5, 0.4)
    lam = O.laplacian_symbol(grid, h)
    z, y, x = np.meshgrid(np.arange(grid[2]), np.arange(grid[1]), np.arange(grid[0]), indexing="ij")
    for kx, ky, kz in [(1, 0, 0), (0, 2, 0), (0, 0, 3), (2, 1, 4), (4, 3, 5)]:
        phi = np.cos(2 * np.pi * (kx * x / grid[0] + ky * y / grid[1] + kz * z / grid[2]))
        Lphi = O.apply_L(phi, h)
        mu = lam[kz % grid[2], ky % grid[1], kx]
        assert np.max(np.abs(Lphi - mu * phi)) < 1e-11 * max(1.0, abs(mu))


def test_fft_poisson_inverts_the_real_space_laplacian():
    grid = (12, 10, 14)
    h = (0.2, 0.3, 0.25)
    src = np.random.default_rng(2).standard_normal((grid[2], grid[1], grid[0]))
    src -= src.mean()
    phi = O.fft_poisson(src, h)
    assert abs(phi.mean()) < 1e-14
    assert np.max(np.abs(O.apply_L(phi, h) - src)) < 1e-11 * np.max(np.abs(src))


def test_assembled_matrix_equals_apply_A_column_by_column():
    rng = np.random.default_rng(3)
    shape = (5, 3, 4)
    eps = 1.0 + 5.0 * rng.random(shape)
    h = (0.4, 0.6, 0.5)
    A = O.assemble_A(eps, h).toarray()
    for j in range(eps.size):
        e = np.zeros(eps.size)
        e[j] = 1.0
        col = O.apply_A(e.reshape(shape), eps, h).ravel()
        assert np.max(np.abs(A[:, j] - col)) < 1e-12 * np.max(np.abs(A))
    assert np.max(np.abs(A - A.T)) < 1e-12 * np.max(np.abs(A))          # symmetric (Appendix B)


def test_residual_norm_by_brute_force_and_at_a_direct_solution():
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    rng = np.random.default_rng(4)
    shape = (6, 5, 4)
    eps = 1.0 + 3.0 * rng.random(shape)
    h = (0.4, 0.5, 0.3)
    rho = rng.standard_normal(shape)
    rho -= rho.mean()
    phi = rng.standard_normal(shape)
    A = O.assemble_A(eps, h)
    b = -4.0 * math.pi * rho.ravel()
    brute = np.linalg.norm(b - A @ phi.ravel()) / np.linalg.norm(b)
    assert abs(O.residual_norm(phi, rho, eps, h) - brute) < 1e-13 * brute
    # the singular periodic operator with the mean fixed: bordered system
    n = eps.size
    K = sp.bmat([[A, sp.csr_matrix(np.ones((n, 1)))], [sp.csr_matrix(np.ones((1, n))), None]]).tocsc()
    x = spla.spsolve(K, np.concatenate([b, [0.0]]))[:n]
    assert O.residual_norm(x.reshape(shape), rho, eps, h) < 1e-12


def test_polarisation_term_is_the_dielectric_excess_of_the_operator():
    """A(eps) = L + div((eps - 1) grad): the face means are linear in eps."""
    rng = np.random.default_rng(5)
    shape = (7, 6, 5)
    eps = 1.0 + 4.0 * rng.random(shape)
    phi = rng.standard_normal(shape)
    h = (0.35, 0.3, 0.45)
    lhs = O.apply_A(phi, eps, h)
    rhs = O.apply_L(phi, h) + O.polarisation_term(phi, eps, h)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(lhs))
    assert np.max(np.abs(O.polarisation_term(phi, np.ones(shape), h))) == 0.0


def test_eq10_beta_default_is_the_printed_value():
    """beta of Eq. 10: the oracle's default and the library's default both equal
    the value the paper prints (tests/golden/paper_parameters.txt)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_parameters.txt")
    vals = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    assert O.GammaParams().beta == vals["beta"]
    from paper_0904_4887_gb300 import gp as G
    assert G.default_params().beta == vals["beta"]
