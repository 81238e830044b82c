"""Plain FP64 CPU oracle for the generalized-Poisson hot path.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may call it. It shares no code with the CUDA library.

Every function restates, in plain and slow NumPy, a definition from
Sanchez, Sued & Scherlis, "First-principles molecular dynamics simulations at
solid-liquid interfaces with a continuum solvent" (arXiv:0904.4887):

  * Eq. 3   generalized Poisson equation  div(eps grad phi) = -4 pi rho
  * Eq. 4   Hartree energy  E = 1/2 int rho phi = 1/(8 pi) int eps |grad phi|^2
  * Eq. 11  dE/dR_I = -1/(8 pi) int (d eps/d R_I)|grad phi|^2 + int phi d rho/d R_I
            (Appendix B, Eq. 26-31)
  * Eq. 15  FFT Poisson solve in vacuum
  * Sec. II.C, Scheme 1   dry/wet split: FFT on the whole box, multigrid on the
            wet sub-domain with Dirichlet values from the FFT solution,
            combined self-consistently (abstract; Sec. I)
  * Sec. III, Eq. 16-18   the sixth-order non-conservative stencil, its solve
            and the adjoint solve its forces need (the last section)

Readings of points where the paper is silent (the dielectric form, the
stencil, the charge model, the split's self-consistent loop) are listed in the
repository's design notes; each function states the one it uses.

Array layout: fields are float64 arrays of shape (nz, ny, nx) in C order, so
the flat index is i + nx*(j + ny*k): x fastest, z-planes contiguous.
Units: Angstrom and elementary charge, Gaussian electrostatics (k = 1).

Parity status: every function below is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py``, ``tests/test_oracle_helper_pins.py`` or
``tests/test_oracle_stencil6_pins.py`` (closed forms, invariants, brute force,
the paper's printed values under ``tests/golden/``).
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np
from scipy.special import erf

FOUR_PI = 4.0 * math.pi
# numpy axis of each Cartesian direction for (nz, ny, nx) arrays
AX = {0: 2, 1: 1, 2: 0}


@dataclasses.dataclass(frozen=True)
class DielectricParams:
    """eps(r) = 1 + (eps0 - 1) * prod_a s(|r - R_a|),  s(d) = (1 + erf((d - r0)/w))/2.

    Position-dependent dielectric built from the atomic coordinates, the idea of
    Sec. II.B (Eq. 9-10) with the erf switching function of the workloads; the
    product runs over atoms and their periodic images with d < rcut (s = 1
    beyond: 1 - s(6 A) is about 1e-23).
    """
    eps0: float = 78.36
    r0: float = 2.5
    w: float = 0.5
    rcut: float = 6.0


GAUSS_CUT_SIGMAS = 8.0   # Gaussian window half-width in sigmas: exp(-32) ~ 1e-14 of the peak


def spacing(grid, cell):
    """Grid spacing h = L/N per axis of the real-space mesh (Sec. III)."""
    return tuple(float(cell[a]) / int(grid[a]) for a in range(3))


def cell_volume_element(grid, cell):
    """h_x h_y h_z: the volume element of the grid sums that stand for the
    integrals of Eq. 4 and Eq. 11."""
    hx, hy, hz = spacing(grid, cell)
    return hx * hy * hz


# ----------------------------------------------------------------------------
# periodic images: sub-boxes of grid points within `radius` of each image
# ----------------------------------------------------------------------------

def _image_boxes(center, grid, cell, radius):
    """Yield (slices, (dz, dy, dx)) for every periodic image of `center` that
    has grid points within `radius`; d* are broadcastable displacement arrays
    r - (center + n L) over the sub-box. Images beyond +-1 cell cannot reach
    the grid when radius <= L (each point and the centre lie in [0, L))."""
    h = spacing(grid, cell)
    for a in range(3):
        assert radius <= cell[a], "cut-off radius must not exceed the cell"
    for n in itertools.product((-1, 0, 1), repeat=3):
        c = [center[a] + n[a] * cell[a] for a in range(3)]
        lo = [max(int(math.ceil((c[a] - radius) / h[a])), 0) for a in range(3)]
        hi = [min(int(math.floor((c[a] + radius) / h[a])), grid[a] - 1) for a in range(3)]
        if any(lo[a] > hi[a] for a in range(3)):
            continue
        dx = np.arange(lo[0], hi[0] + 1) * h[0] - c[0]
        dy = np.arange(lo[1], hi[1] + 1) * h[1] - c[1]
        dz = np.arange(lo[2], hi[2] + 1) * h[2] - c[2]
        sl = (slice(lo[2], hi[2] + 1), slice(lo[1], hi[1] + 1), slice(lo[0], hi[0] + 1))
        yield sl, (dz[:, None, None], dy[None, :, None], dx[None, None, :])


# ----------------------------------------------------------------------------
# dielectric eps(R) and its atomic derivative
# ----------------------------------------------------------------------------

def switching(d, p: DielectricParams):
    """s(d) = (1 + erf((d - r0)/w))/2: one atom's factor in the erf-product
    dielectric, the reading used for the position-dependent eps of Sec. II.B."""
    return 0.5 * (1.0 + erf((d - p.r0) / p.w))


def switching_derivative(d, p: DielectricParams):
    """ds/dd = exp(-((d - r0)/w)^2) / (w sqrt(pi)), the factor d eps/d R of
    Eq. 11 needs for the erf-product dielectric."""
    return np.exp(-((d - p.r0) / p.w) ** 2) / (p.w * math.sqrt(math.pi))


def dielectric_product(grid, cell, pos, p: DielectricParams = DielectricParams()):
    """P = prod over atoms and images within rcut of s(d); eps = 1 + (eps0-1) P
    (Sec. II.B, erf-product reading)."""
    P = np.ones((grid[2], grid[1], grid[0]))
    for R in pos:
        for sl, (dz, dy, dx) in _image_boxes(R, grid, cell, p.rcut):
            d = np.sqrt(dx * dx + dy * dy + dz * dz)
            f = np.where(d < p.rcut, switching(d, p), 1.0)
            P[sl] *= f
    return P


def dielectric(grid, cell, pos, p: DielectricParams = DielectricParams()):
    """eps on the grid (position-dependent dielectric, Sec. II.B)."""
    return 1.0 + (p.eps0 - 1.0) * dielectric_product(grid, cell, pos, p)


def dielectric_points(points, cell, pos, p: DielectricParams = DielectricParams()):
    """eps at arbitrary points (M, 3), one by one over atoms and all 27 images
    (Sec. II.B, erf-product reading)."""
    points = np.asarray(points, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    P = np.ones(len(points))
    for R in pos:
        for n in itertools.product((-1, 0, 1), repeat=3):
            d = np.linalg.norm(points - (R + np.asarray(n) * cell), axis=1)
            P *= np.where(d < p.rcut, switching(d, p), 1.0)
    return 1.0 + (p.eps0 - 1.0) * P


def dielectric_gradient_atom(a, grid, cell, pos, P, p: DielectricParams = DielectricParams()):
    """d eps_i / d R_a on the grid, as three arrays (x, y, z components): the
    derivative inside the solvent term of Eq. 11 (Appendix B).

    Product rule over the factors that belong to atom a (one per image within
    rcut): d eps/dR_a = (eps0-1) sum_images [P / s(d)] s'(d) dd/dR_a, with
    dd/dR_a = -(r - R_a)/d. P / s(d) is the product of all other factors;
    every factor is at least erfc(r0/w)/2 > 0, so the division is exact up to
    rounding.
    """
    out = [np.zeros_like(P) for _ in range(3)]
    for sl, (dz, dy, dx) in _image_boxes(pos[a], grid, cell, p.rcut):
        d = np.sqrt(dx * dx + dy * dy + dz * dz)
        inside = d < p.rcut
        dsafe = np.where(d > 0, d, 1.0)
        coef = np.where(inside, (p.eps0 - 1.0) * P[sl] / switching(d, p)
                        * switching_derivative(d, p) / dsafe, 0.0)
        coef = np.where(d > 0, coef, 0.0)
        out[0][sl] += -coef * dx
        out[1][sl] += -coef * dy
        out[2][sl] += -coef * dz
    return out


# ----------------------------------------------------------------------------
# the dummy-density dielectric of Eq. 9-10 and its atomic derivative (Eq. 12)
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class GammaParams:
    """Eq. 9: gamma(r) = sum_I exp(-(|r - R_I| - Rvdw_I)) over every atom and
    every periodic image; Eq. 10: eps = 1 + (eps0 - 1)/2 (1 + (1 - gamma^(2 beta))
    /(1 + gamma^(2 beta))).

    The paper sums over all atoms. The image sum converges (its terms decay like
    exp(-d) while their number grows like d^2), so it is taken over the images
    within the radius gamma_cutoff(cell, rvdw, tail), beyond which
    gamma_tail_bound proves the neglected part of gamma to be below `tail`
    everywhere. No taper: a term at the cut-off is below ~1e-17, so the step it
    puts into E(R) where a cut-off sphere crosses a grid point is below
    rounding.
    """
    eps0: float = 78.36
    beta: float = 2.4
    tail: float = 1e-13


def gamma_tail_bound(radius, cell, rvdw):
    """Upper bound on sum_I exp(-(d_I - Rvdw_I)) over all atoms and images with
    d_I > radius, at any point of the cell.

    The images of one atom form the lattice {R + nL}. Around each image put the
    cell-shaped box it is the centre of; these boxes do not overlap, and every
    box of an image within distance r lies inside the ball of radius r + c, c
    half the cell diagonal. So at most N(r) = (4 pi/3)(r + c)^3 / V images lie
    within r. With that count, sum_{d > R} exp(-d) = int_R^inf exp(-r) dN(r)
    <= int_R^inf exp(-r) N(r) dr (integration by parts, the boundary term being
    negative), and int_R^inf exp(-r)(r + c)^3 dr = exp(-R)(u^3 + 3u^2 + 6u + 6)
    with u = R + c. Each atom's sum carries the factor exp(Rvdw_I).
    """
    L = np.asarray(cell, dtype=np.float64)
    V = float(L[0] * L[1] * L[2])
    u = float(radius) + 0.5 * float(np.sqrt(np.sum(L * L)))
    poly = u ** 3 + 3.0 * u ** 2 + 6.0 * u + 6.0
    return (4.0 * math.pi / (3.0 * V)) * math.exp(-float(radius)) * poly * float(np.sum(np.exp(rvdw)))


def gamma_cutoff(cell, rvdw, tail):
    """The smallest radius (to 1e-6 A, by bisection) at which gamma_tail_bound
    is at most `tail`; the bound falls monotonically with the radius (its
    derivative is -exp(-R) u^3)."""
    lo, hi = 0.0, 1.0
    while gamma_tail_bound(hi, cell, rvdw) > tail:
        hi *= 2.0
    while hi - lo > 1e-6:
        mid = 0.5 * (lo + hi)
        if gamma_tail_bound(mid, cell, rvdw) > tail:
            lo = mid
        else:
            hi = mid
    return hi


def _image_boxes_any(center, grid, cell, radius):
    """Like _image_boxes for any radius (also beyond one cell): every image
    centre + n L within `radius` of the grid's box [0, L) per axis, with the
    sub-box of grid points within `radius` of it."""
    h = spacing(grid, cell)
    rng = []
    for a in range(3):
        n0 = int(math.floor((-radius - center[a]) / cell[a]))
        n1 = int(math.ceil((cell[a] + radius - center[a]) / cell[a]))
        rng.append(range(n0, n1 + 1))
    for n in itertools.product(*rng):
        c = [center[a] + n[a] * cell[a] for a in range(3)]
        lo = [max(int(math.ceil((c[a] - radius) / h[a])), 0) for a in range(3)]
        hi = [min(int(math.floor((c[a] + radius) / h[a])), grid[a] - 1) for a in range(3)]
        if any(lo[a] > hi[a] for a in range(3)):
            continue
        dx = np.arange(lo[0], hi[0] + 1) * h[0] - c[0]
        dy = np.arange(lo[1], hi[1] + 1) * h[1] - c[1]
        dz = np.arange(lo[2], hi[2] + 1) * h[2] - c[2]
        sl = (slice(lo[2], hi[2] + 1), slice(lo[1], hi[1] + 1), slice(lo[0], hi[0] + 1))
        yield sl, (dz[:, None, None], dy[None, :, None], dx[None, None, :])


def _point_images(points, center, cell, radius):
    """Displacements (M, 3) from every image of `center` that lies within
    `radius` of the cell box to the points, one image at a time."""
    rng = []
    for a in range(3):
        n0 = int(math.floor((-radius - center[a]) / cell[a]))
        n1 = int(math.ceil((cell[a] + radius - center[a]) / cell[a]))
        rng.append(range(n0, n1 + 1))
    for n in itertools.product(*rng):
        yield points - (center + np.asarray(n) * cell)


def dummy_density(grid, cell, pos, rvdw, p: GammaParams = GammaParams()):
    """gamma on the grid (Eq. 9), over every image within gamma_cutoff."""
    rc = gamma_cutoff(cell, rvdw, p.tail)
    g = np.zeros((grid[2], grid[1], grid[0]))
    for R, rv in zip(pos, rvdw):
        for sl, (dz, dy, dx) in _image_boxes_any(R, grid, cell, rc):
            d = np.sqrt(dx * dx + dy * dy + dz * dz)
            g[sl] += np.where(d < rc, np.exp(-(d - rv)), 0.0)
    return g


def eps_of_gamma(gamma, p: GammaParams = GammaParams()):
    """Eq. 10, written as the paper prints it."""
    t = gamma ** (2.0 * p.beta)
    return 1.0 + 0.5 * (p.eps0 - 1.0) * (1.0 + (1.0 - t) / (1.0 + t))


def deps_dgamma(gamma, p: GammaParams = GammaParams()):
    """d eps/d gamma of Eq. 10: -(eps0 - 1) 2 beta gamma^(2 beta - 1)/(1 + gamma^(2 beta))^2."""
    t = gamma ** (2.0 * p.beta)
    gm = np.where(gamma > 0, gamma, 1.0)
    return np.where(gamma > 0, -(p.eps0 - 1.0) * 2.0 * p.beta * t / gm / (1.0 + t) ** 2, 0.0)


def dielectric_gamma(grid, cell, pos, rvdw, p: GammaParams = GammaParams()):
    """eps on the grid from Eq. 9-10."""
    return eps_of_gamma(dummy_density(grid, cell, pos, rvdw, p), p)


def dielectric_gamma_points(points, cell, pos, rvdw, p: GammaParams = GammaParams()):
    """Eq. 9-10 at arbitrary points (M, 3), one atom image at a time over every
    image within gamma_cutoff."""
    points = np.asarray(points, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    rc = gamma_cutoff(cell, rvdw, p.tail)
    g = np.zeros(len(points))
    for R, rv in zip(pos, rvdw):
        for dv in _point_images(points, np.asarray(R, dtype=np.float64), cell, rc):
            d = np.linalg.norm(dv, axis=1)
            g += np.where(d < rc, np.exp(-(d - rv)), 0.0)
    return eps_of_gamma(g, p)


def dielectric_gamma_gradient_atom(a, grid, cell, pos, rvdw, gamma, p: GammaParams = GammaParams()):
    """d eps_i / d R_a (x, y, z arrays) for Eq. 9-10: by the chain rule,
    (d eps/d gamma) sum_images exp(-(d - Rvdw_a)) (r - R_a)/d, because
    d|r - R_a|/dR_a = -(r - R_a)/d. This is Eq. 12 with the opposite sign to
    the printed one: moving an atom towards r raises gamma there and lowers eps.
    """
    rc = gamma_cutoff(cell, rvdw, p.tail)
    fe = deps_dgamma(gamma, p)
    out = [np.zeros_like(gamma) for _ in range(3)]
    for sl, (dz, dy, dx) in _image_boxes_any(pos[a], grid, cell, rc):
        d = np.sqrt(dx * dx + dy * dy + dz * dz)
        dsafe = np.where(d > 0, d, 1.0)
        coef = np.where((d > 0) & (d < rc), fe[sl] * np.exp(-(d - rvdw[a])) / dsafe, 0.0)
        out[0][sl] += coef * dx
        out[1][sl] += coef * dy
        out[2][sl] += coef * dz
    return out


# ----------------------------------------------------------------------------
# Eq. 19: the dummy density with the solvent excluded below z_lim
# ----------------------------------------------------------------------------
# Reading of Eq. 19 (the paper states it for a cell whose z runs from 0 at the
# bottom to Lz at the top): for an atom with z_I <= z_lim the exponent's sign is
# that of z - z_I, both taken inside the cell [0, Lz) (+1 at z = z_I), so below
# such an atom its term grows as exp(+(|r - R_I| - Rvdw)) and eps saturates to 1.
# A growing term uses the nearest periodic image of the atom (an image sum of
# growing exponentials has no limit) and no cut-off. Once one growing exponent
# reaches sat_exponent(p) = (ln(eps0 - 1) + 37)/(2 beta), eps - 1 is below
# exp(-37) < 1e-16 and d eps/d gamma is as small: such a point is "saturated",
# with eps = 1 and d eps/d gamma = 0. Atoms with z_I > z_lim, and lower atoms at
# points with z >= z_I, contribute as in Eq. 9 (every image within
# gamma_cutoff).
def sat_exponent(p):
    """Growing exponent of Eq. 19 beyond which eps - 1 = (eps0-1)/(1+gamma^(2 beta))
    is below 1e-16 (exp(-37) of eps0 - 1), so that eps is taken as exactly 1."""
    return (math.log(p.eps0 - 1.0) + 37.0) / (2.0 * p.beta)


def _min_image(dv, L):
    """The periodic image of a displacement closest to zero (used by Eq. 19)."""
    return dv - L * np.round(dv / L)


def dummy_density_eq19(grid, cell, pos, rvdw, zlim, p: GammaParams = GammaParams()):
    """(gamma, saturated) on the grid for Eq. 19 (see the reading above)."""
    x, y, z = _grid_coords(grid, cell)
    g = np.zeros((grid[2], grid[1], grid[0]))
    sat = np.zeros(g.shape, dtype=bool)
    posw = np.mod(pos, np.asarray(cell))
    lower = posw[:, 2] <= zlim
    rc = gamma_cutoff(cell, rvdw, p.tail)
    for a, (R, rv) in enumerate(zip(posw, rvdw)):
        below = (z < R[2]) if lower[a] else np.zeros_like(z, dtype=bool)
        for sl, (dz, dy, dx) in _image_boxes_any(R, grid, cell, rc):
            d = np.sqrt(dx * dx + dy * dy + dz * dz)
            keep = ~np.broadcast_to(below, g.shape)[sl]
            g[sl] += np.where(keep & (d < rc), np.exp(-(d - rv)), 0.0)
        if lower[a]:
            ddx = _min_image(x - R[0], cell[0])
            ddy = _min_image(y - R[1], cell[1])
            ddz = _min_image(z - R[2], cell[2])
            d = np.sqrt(ddx * ddx + ddy * ddy + ddz * ddz)
            e = d - rv
            es = sat_exponent(p)
            grow = np.broadcast_to(below, g.shape)
            sat |= grow & (e >= es)
            g += np.where(grow & (e < es), np.exp(np.minimum(e, es)), 0.0)
    return g, sat


def dielectric_eq19(grid, cell, pos, rvdw, zlim, p: GammaParams = GammaParams()):
    """eps on the grid for Eq. 19 with Eq. 10 (simplified form, which stays finite)."""
    g, sat = dummy_density_eq19(grid, cell, pos, rvdw, zlim, p)
    t = np.where(sat, np.inf, g ** (2.0 * p.beta))
    return np.where(sat, 1.0, 1.0 + (p.eps0 - 1.0) / (1.0 + t))


def dielectric_eq19_gradient_atom(a, grid, cell, pos, rvdw, zlim, gamma, sat, p: GammaParams = GammaParams()):
    """d eps_i/d R_a for Eq. 19: decaying terms as Eq. 9, a growing term
    exp(+(d - Rvdw)) gives -(d eps/d gamma) exp(d - Rvdw) (r - R_a)/d; zero at
    saturated points."""
    x, y, z = _grid_coords(grid, cell)
    fe = np.where(sat, 0.0, deps_dgamma(np.where(sat, 1.0, gamma), p))
    out = [np.zeros_like(gamma) for _ in range(3)]
    posw = np.mod(pos, np.asarray(cell))
    R, rv = posw[a], rvdw[a]
    lower = R[2] <= zlim
    below = np.broadcast_to((z < R[2]) if lower else np.zeros_like(z, dtype=bool), gamma.shape)
    rc = gamma_cutoff(cell, rvdw, p.tail)
    for sl, (dz, dy, dx) in _image_boxes_any(R, grid, cell, rc):
        d = np.sqrt(dx * dx + dy * dy + dz * dz)
        dsafe = np.where(d > 0, d, 1.0)
        coef = np.where((d > 0) & (d < rc) & ~below[sl], fe[sl] * np.exp(-(d - rv)) / dsafe, 0.0)
        out[0][sl] += coef * dx
        out[1][sl] += coef * dy
        out[2][sl] += coef * dz
    if lower:
        ddx = np.broadcast_to(_min_image(x - R[0], cell[0]), gamma.shape)
        ddy = np.broadcast_to(_min_image(y - R[1], cell[1]), gamma.shape)
        ddz = np.broadcast_to(_min_image(z - R[2], cell[2]), gamma.shape)
        d = np.sqrt(ddx * ddx + ddy * ddy + ddz * ddz)
        dsafe = np.where(d > 0, d, 1.0)
        es = sat_exponent(p)
        coef = np.where(below & (d - rv < es) & (d > 0), -fe * np.exp(np.minimum(d - rv, es)) / dsafe, 0.0)
        out[0] += coef * ddx
        out[1] += coef * ddy
        out[2] += coef * ddz
    return out


def _grid_coords(grid, cell):
    """Coordinates r_ijk = (i h_x, j h_y, k h_z) as broadcastable arrays."""
    h = spacing(grid, cell)
    x = (np.arange(grid[0]) * h[0])[None, None, :]
    y = (np.arange(grid[1]) * h[1])[None, :, None]
    z = (np.arange(grid[2]) * h[2])[:, None, None]
    return x, y, z


# ----------------------------------------------------------------------------
# charge density: +Z core and -Z cloud Gaussians per atom (Sec. II.A)
# ----------------------------------------------------------------------------

def gaussian(d2, sigma):
    """Normalised 3D Gaussian of standard deviation sigma at squared distance d2
    (the Gaussian ionic charges of Sec. II.A)."""
    return np.exp(-d2 / (2.0 * sigma * sigma)) / (2.0 * math.pi * sigma * sigma) ** 1.5


def _in_window(dx, dy, dz, rad):
    """Truncation window of a Gaussian: |dx|, |dy|, |dz| all below cut*sigma
    (a cube; the paper gives no truncation, and beyond 8 sigma the Gaussian
    is below 1.3e-14 of its peak)."""
    return (np.abs(dx) < rad) & (np.abs(dy) < rad) & (np.abs(dz) < rad)


def charge_density_raw(grid, cell, pos, Z, sigma_core, sigma_cloud, cut=GAUSS_CUT_SIGMAS):
    """rho~_i = sum_a Z_a [g(d; sigma_core,a) - g(d; sigma_cloud,a)] over periodic
    images, each Gaussian truncated to its window (_in_window); Sec. II.A."""
    rho = np.zeros((grid[2], grid[1], grid[0]))
    for a, R in enumerate(pos):
        for sign, sig in ((1.0, sigma_core[a]), (-1.0, sigma_cloud[a])):
            rad = cut * sig
            for sl, (dz, dy, dx) in _image_boxes(R, grid, cell, rad):
                d2 = dx * dx + dy * dy + dz * dz
                rho[sl] += np.where(_in_window(dx, dy, dz, rad), sign * Z[a] * gaussian(d2, sig), 0.0)
    return rho


def charge_density(grid, cell, pos, Z, sigma_core, sigma_cloud, cut=GAUSS_CUT_SIGMAS):
    """Neutral rho: the raw Gaussian sum minus its grid mean (discrete neutrality
    of the periodic Eq. 3)."""
    raw = charge_density_raw(grid, cell, pos, Z, sigma_core, sigma_cloud, cut)
    return raw - raw.mean()


def charge_density_points(points, cell, pos, Z, sigma_core, sigma_cloud, cut=GAUSS_CUT_SIGMAS):
    """rho~ (before mean removal) at arbitrary points, one by one (Sec. II.A)."""
    points = np.asarray(points, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    out = np.zeros(len(points))
    for a, R in enumerate(pos):
        for n in itertools.product((-1, 0, 1), repeat=3):
            dd = points - (R + np.asarray(n) * cell)
            d2 = np.sum(dd ** 2, axis=1)
            for sign, sig in ((1.0, sigma_core[a]), (-1.0, sigma_cloud[a])):
                rad = cut * sig
                inside = _in_window(dd[:, 0], dd[:, 1], dd[:, 2], rad)
                out += np.where(inside, sign * Z[a] * gaussian(d2, sig), 0.0)
    return out


def charge_density_gradient_atom(a, grid, cell, pos, Z, sigma_core, sigma_cloud,
                                 cut=GAUSS_CUT_SIGMAS):
    """d rho~_i / d R_a (x, y, z arrays): d g/dR = g (r - R)/sigma^2; the charge
    term of Eq. 11."""
    out = [np.zeros((grid[2], grid[1], grid[0])) for _ in range(3)]
    for sign, sig in ((1.0, sigma_core[a]), (-1.0, sigma_cloud[a])):
        rad = cut * sig
        for sl, (dz, dy, dx) in _image_boxes(pos[a], grid, cell, rad):
            d2 = dx * dx + dy * dy + dz * dz
            c = np.where(_in_window(dx, dy, dz, rad), sign * Z[a] * gaussian(d2, sig) / (sig * sig), 0.0)
            out[0][sl] += c * dx
            out[1][sl] += c * dy
            out[2][sl] += c * dz
    return out


# ----------------------------------------------------------------------------
# the operator of Eq. 3 and the FFT solve of Eq. 15
# ----------------------------------------------------------------------------

def face_mean(eps, axis):
    """eps on the face between i and i+1 along `axis`: the arithmetic mean (the
    face coefficient of the conservative discretisation of Eq. 3)."""
    return 0.5 * (eps + np.roll(eps, -1, axis=axis))


def apply_A(phi, eps, h):
    """(A phi)_i = sum_axes [eps_{i+1/2}(phi_{i+1}-phi_i) - eps_{i-1/2}(phi_i-phi_{i-1})]/h^2.

    The conservative 7-point discretisation of div(eps grad phi) (Eq. 3),
    periodic in all three directions.
    """
    out = np.zeros_like(phi)
    for c in range(3):
        ax = AX[c]
        flux = face_mean(eps, ax) * (np.roll(phi, -1, axis=ax) - phi) / (h[c] * h[c])
        out += flux - np.roll(flux, 1, axis=ax)
    return out


def apply_L(phi, h):
    """The same 7-point operator with eps = 1 (the vacuum Laplacian of Eq. 2)."""
    return apply_A(phi, np.ones_like(phi), h)


def polarisation_term(phi, eps, h):
    """div((eps-1) grad phi) on the grid: the charge 4 pi rho_pol that the
    dielectric adds to the vacuum problem, so that A phi = L phi + this
    (the coupling of Sec. II.C, Scheme 1)."""
    return apply_A(phi, eps - 1.0, h)


def laplacian_symbol(grid, h):
    """Eigenvalues of the 7-point Laplacian on the periodic grid (the divisor of
    the FFT solve of Eq. 15 in its discrete form),
    lambda(k) = sum_axes (2 cos(2 pi k_a / N_a) - 2)/h_a^2, as an (nz, ny, nx//2+1)
    array matching numpy's rfftn layout."""
    nx, ny, nz = grid
    lx = (2.0 * np.cos(2.0 * np.pi * np.arange(nx // 2 + 1) / nx) - 2.0) / h[0] ** 2
    ly = (2.0 * np.cos(2.0 * np.pi * np.fft.fftfreq(ny) ) - 2.0) / h[1] ** 2
    lz = (2.0 * np.cos(2.0 * np.pi * np.fft.fftfreq(nz)) - 2.0) / h[2] ** 2
    return lz[:, None, None] + ly[None, :, None] + lx[None, None, :]


def fft_poisson(src, h):
    """Solve L phi = src on the periodic grid (Eq. 15 with the symbol of the
    discrete operator, so that the result satisfies the 7-point equation to
    rounding). The k = 0 mode is set to zero: phi has mean zero."""
    grid = (src.shape[2], src.shape[1], src.shape[0])
    lam = laplacian_symbol(grid, h)
    s = np.fft.rfftn(src)
    lam[0, 0, 0] = 1.0
    s = s / lam
    s[0, 0, 0] = 0.0
    return np.fft.irfftn(s, s=src.shape, axes=(0, 1, 2))


def vacuum_potential(rho, h):
    """phi solving the vacuum equation L phi = -4 pi rho (Eq. 2, 15)."""
    return fft_poisson(-FOUR_PI * rho, h)


# ----------------------------------------------------------------------------
# the generalized Poisson solve, to near machine precision
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class SolveInfo:
    """Iterations and final relative residual of a solve of Eq. 3 (or Eq. 16)."""
    iterations: int
    residual: float      # ||b - A phi|| / ||b|| of the returned phi


def residual_norm(phi, rho, eps, h):
    """||b - A phi||_2 / ||b||_2 with b = -4 pi rho, all in FP64 (Eq. 3)."""
    b = -FOUR_PI * rho
    r = b - apply_A(phi, eps, h)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(r) / nb) if nb > 0 else float(np.linalg.norm(r))


def solve(rho, eps, h, tol=1e-14, maxiter=3000, phi0=None):
    """phi with A phi = -4 pi rho and mean(phi) = 0 (Eq. 3).

    Conjugate gradients on -A (symmetric, positive definite on mean-zero
    vectors), preconditioned by the inverse vacuum Laplacian (the FFT solve).
    Any convergent method reaches the same discrete solution; this one is
    textbook PCG. Stops when the recursively updated relative residual is
    below `tol` or stagnates.
    """
    b = -FOUR_PI * (rho - rho.mean())
    nb = np.linalg.norm(b)
    phi = np.zeros_like(rho) if phi0 is None else phi0 - phi0.mean()
    if nb == 0:
        return np.zeros_like(rho), SolveInfo(0, 0.0)
    # M = -A, preconditioner P^-1 r = -(L^-1) r
    r = -(b - apply_A(phi, eps, h))          # residual of M phi = -b
    r -= r.mean()
    z = -fft_poisson(r, h)
    p = z.copy()
    rz = float(np.vdot(r, z))
    best = np.inf
    stall = 0
    it = 0
    for it in range(1, maxiter + 1):
        q = -apply_A(p, eps, h)
        alpha = rz / float(np.vdot(p, q))
        phi += alpha * p
        r -= alpha * q
        rn = np.linalg.norm(r) / nb
        if rn < tol:
            break
        if rn < 0.5 * best:
            best = rn
            stall = 0
        else:
            stall += 1
            if stall > 50:
                break
        z = -fft_poisson(r, h)
        rz_new = float(np.vdot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    phi -= phi.mean()
    return phi, SolveInfo(it, residual_norm(phi, rho - rho.mean(), eps, h))


# ----------------------------------------------------------------------------
# energy (Eq. 4) and forces (Eq. 11, Appendix B)
# ----------------------------------------------------------------------------

def energy(rho, phi, grid, cell):
    """E = 1/2 h^3 sum rho phi (Eq. 4, first form)."""
    return 0.5 * cell_volume_element(grid, cell) * float(np.sum(rho * phi))


def field_energy(phi, eps, grid, cell):
    """E' = h^3/(8 pi) sum_faces eps_f (Delta_f phi / h)^2 (Eq. 4, second form)."""
    h = spacing(grid, cell)
    tot = 0.0
    for c in range(3):
        ax = AX[c]
        g = (np.roll(phi, -1, axis=ax) - phi) / h[c]
        tot += float(np.sum(face_mean(eps, ax) * g * g))
    return cell_volume_element(grid, cell) * tot / (8.0 * math.pi)


def variational_energy(rho, phi, eps, grid, cell):
    """J(phi) = h^3 rho.phi + h^3/(8 pi) phi.A phi; equals E of Eq. 4 at the
    solution, with an error quadratic in the error of phi."""
    h = spacing(grid, cell)
    dv = cell_volume_element(grid, cell)
    return dv * float(np.sum(rho * phi)) + dv / (8.0 * math.pi) * float(np.sum(phi * apply_A(phi, eps, h)))


def energy_gradient(phi, grid, cell, pos, Z, sigma_core, sigma_cloud,
                    p=DielectricParams(), atoms=None, rho_moves=True, rvdw=None, zlim=None):
    """G_a = dE/dR_a = G^eps_a + G^rho_a, the discrete Eq. 11.

    G^eps_a = -h^3/(8 pi) sum_faces (d eps_f/dR_a)(Delta_f phi/h)^2, with
              d eps_f = (d eps_i + d eps_{i+1})/2 (the face mean of Eq. 3)
    G^rho_a = h^3 sum_i phi_i d rho_i/dR_a, with rho = rho~ - mean(rho~)

    Returns (G_eps, G_rho), each (n_atoms, 3); rows of atoms not in `atoms` are
    zero. `phi` must be the solution for this geometry: because A is symmetric
    it is its own adjoint (Appendix B), so no further solve is needed.
    `p` is DielectricParams (erf product) or GammaParams (Eq. 9-10, with the
    radii `rvdw`; Eq. 19 when `zlim` is given).
    """
    h = spacing(grid, cell)
    dv = cell_volume_element(grid, cell)
    n = len(pos)
    atoms = range(n) if atoms is None else atoms
    gamma_form = isinstance(p, GammaParams)
    if gamma_form and zlim is not None:
        G, SAT = dummy_density_eq19(grid, cell, pos, rvdw, zlim, p)
    elif gamma_form:
        G = dummy_density(grid, cell, pos, rvdw, p)
    else:
        P = dielectric_product(grid, cell, pos, p)
    grads2 = []
    for c in range(3):
        ax = AX[c]
        g = (np.roll(phi, -1, axis=ax) - phi) / h[c]
        grads2.append((ax, g * g))
    Ge = np.zeros((n, 3))
    Gr = np.zeros((n, 3))
    for a in atoms:
        if gamma_form and zlim is not None:
            de = dielectric_eq19_gradient_atom(a, grid, cell, pos, rvdw, zlim, G, SAT, p)
        elif gamma_form:
            de = dielectric_gamma_gradient_atom(a, grid, cell, pos, rvdw, G, p)
        else:
            de = dielectric_gradient_atom(a, grid, cell, pos, P, p)
        for comp in range(3):
            s = 0.0
            for ax, g2 in grads2:
                s += float(np.sum(face_mean(de[comp], ax) * g2))
            Ge[a, comp] = -dv / (8.0 * math.pi) * s
        if rho_moves:
            dr = charge_density_gradient_atom(a, grid, cell, pos, Z, sigma_core, sigma_cloud)
            for comp in range(3):
                Gr[a, comp] = dv * float(np.sum(phi * (dr[comp] - dr[comp].mean())))
    return Ge, Gr


# ----------------------------------------------------------------------------
# dry/wet split (Sec. II.C, Scheme 1) made self-consistent
# ----------------------------------------------------------------------------

def dry_planes(eps, thresh=1e-3):
    """z-planes on which eps - 1 < thresh everywhere ("dry": eps is 1 there;
    Sec. II.C)."""
    return (eps - 1.0).max(axis=(1, 2)) < thresh


def plan_band(dry, levels, n_dirichlet=1):
    """Choose the wet band Omega_1 (a periodic run of z-planes) and its
    Dirichlet planes, from the per-plane dry flags (Sec. II.C).

    Reading: the Dirichlet planes sit in the middle of the longest periodic run
    of dry planes; there are n_dirichlet of them (0 = as many as the run holds),
    reduced to the form 1 + m 2^(levels-1) so that the band (all other planes,
    nz - n_dirichlet interior planes between Dirichlet walls) coarsens
    `levels - 1` times. Returns (first_dirichlet_plane, n_dirichlet) or None
    when no plane is dry.
    """
    nz = len(dry)
    if not np.any(dry):
        return None
    if np.all(dry):
        run_start, run_len = 0, nz
    else:
        # start scanning just after a wet plane so that runs do not wrap mid-way
        k0 = int(np.argmin(dry))
        run_start, run_len, cur_start, cur_len = 0, 0, None, 0
        for t in range(1, nz + 1):
            k = (k0 + t) % nz
            if dry[k]:
                if cur_len == 0:
                    cur_start = k
                cur_len += 1
                if cur_len > run_len:
                    run_start, run_len = cur_start, cur_len
            else:
                cur_len = 0
    step = 2 ** (levels - 1)
    want = run_len if n_dirichlet <= 0 else min(n_dirichlet, run_len)
    nd = 1 + ((want - 1) // step) * step
    if nd >= nz:
        nd = 1
    first = (run_start + (run_len - nd) // 2) % nz
    return first, nd


def band_planes(nz, first, nd):
    """Interior planes of the band, in order: the nz - nd planes after the
    Dirichlet block (periodic; Sec. II.C)."""
    return [(first + nd + t) % nz for t in range(nz - nd)]


def assemble_A(eps, h):
    """A as a scipy sparse matrix (same definition as apply_A, Eq. 3), flat x-fastest."""
    import scipy.sparse as sp
    nz, ny, nx = eps.shape
    n = eps.size
    idx = np.arange(n).reshape(eps.shape)
    rows, cols, vals = [], [], []
    diag = np.zeros(eps.shape)
    for c in range(3):
        ax = AX[c]
        ef = face_mean(eps, ax) / (h[c] * h[c])
        nb = np.roll(idx, -1, axis=ax)
        rows += [idx.ravel(), nb.ravel()]
        cols += [nb.ravel(), idx.ravel()]
        vals += [ef.ravel(), ef.ravel()]
        diag -= ef + np.roll(ef, 1, axis=ax)
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def split_solve(rho, eps, h, band, tol=1e-13, maxit=200):
    """Scheme 1 iterated to self-consistency (reading of Sec. II.C):

      phi^0 = vacuum FFT solution on the whole box Omega;
      repeat:  solve A phi = b on the wet band Omega_1 with Dirichlet values
               phi^k on the planes outside it (keep phi^k there);
               4 pi rho_pol = div((eps - 1) grad phi) on Omega;
               phi^{k+1} = FFT solution of L phi = b - 4 pi rho_pol.

    The fixed point satisfies L phi + div((eps-1) grad phi) = A phi = b, the
    full-box equation. `band` = (first_dirichlet_plane, n_dirichlet).
    Band solves are exact (sparse LU), so use small grids.
    Returns (phi, history of the relative change per iteration).
    """
    import scipy.sparse.linalg as spl
    nz, ny, nx = rho.shape
    first, nd = band
    planes = band_planes(nz, first, nd)
    wet = np.zeros(nz, dtype=bool)
    wet[planes] = True
    wmask = np.broadcast_to(wet[:, None, None], rho.shape).ravel()
    widx = np.nonzero(wmask)[0]
    bidx = np.nonzero(~wmask)[0]
    A = assemble_A(eps, h)
    Aww = A[widx][:, widx].tocsc()
    Awb = A[widx][:, bidx]
    lu = spl.splu(Aww)
    b = (-FOUR_PI * rho).ravel()
    phi = fft_poisson(b.reshape(rho.shape), h)
    hist = []
    combined = phi
    for _ in range(maxit):
        p = phi.ravel().copy()
        p[widx] = lu.solve(b[widx] - Awb @ p[bidx])
        combined = p.reshape(rho.shape)
        pol = polarisation_term(combined, eps, h)
        new = fft_poisson(b.reshape(rho.shape) - pol, h)
        change = np.linalg.norm(new - phi) / max(np.linalg.norm(new), 1e-300)
        hist.append(change)
        phi = new
        if change < tol:
            break
    return combined - combined.mean(), hist


# ----------------------------------------------------------------------------
# the sixth-order non-conservative stencil (Sec. III, Eq. 16-18)
# ----------------------------------------------------------------------------
#
# Eq. 16 expands Eq. 3 by the product rule, grad(eps).grad(phi) + eps lap(phi)
# = -4 pi rho (the printed eps lap(eps) is read as eps lap(phi)), and Eq. 17-18
# discretise each first and second derivative with seven points along its axis.
# The resulting 19-point operator A6 annihilates constants but is neither
# symmetric nor conservative: its left null vector is not the constant vector,
# so a neutral rho is not exactly in its range on the periodic grid. The
# reading used here adds the smallest correction that restores solvability in
# the divided form lap(phi) + grad(ln eps).grad(phi) = -4 pi rho/eps, a uniform
# shift there, i.e. mu * eps here:
#
#     A6 phi + mu eps = -4 pi rho,   sum(phi) = 0,
#
# whose mu vanishes with the truncation error (O(h^6) for smooth fields).

# Eq. 17-18 as printed: alpha_{-n} = -alpha_n, beta_{-n} = beta_n, n = 0..3
FD6_ALPHA = (0.0, 3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0)
FD6_BETA = (-49.0 / 18.0, 27.0 / 18.0, -27.0 / 180.0, 2.0 / 180.0)


def fd6_first(u, c, h):
    """du/dx_c at every grid point, (1/h) sum_{n=-3..3} alpha_n u_{i+n} (Eq. 17),
    periodic."""
    ax = AX[c]
    out = np.zeros_like(u)
    for n in (1, 2, 3):
        out += FD6_ALPHA[n] * (np.roll(u, -n, axis=ax) - np.roll(u, n, axis=ax))
    return out / h[c]


def fd6_second(u, c, h):
    """d2u/dx_c^2 at every grid point, (1/h^2) sum_{n=-3..3} beta_n u_{i+n}
    (Eq. 18), periodic."""
    ax = AX[c]
    out = FD6_BETA[0] * u
    for n in (1, 2, 3):
        out = out + FD6_BETA[n] * (np.roll(u, -n, axis=ax) + np.roll(u, n, axis=ax))
    return out / (h[c] * h[c])


def apply_A6(phi, eps, h):
    """(A6 phi)_i = sum_axes [(D1 eps)_i (D1 phi)_i + eps_i (D2 phi)_i]: Eq. 16
    with the derivatives of Eq. 17-18."""
    out = np.zeros_like(phi)
    for c in range(3):
        out += fd6_first(eps, c, h) * fd6_first(phi, c, h) + eps * fd6_second(phi, c, h)
    return out


def apply_A6_transpose(lam, eps, h):
    """A6^T lam (Eq. 16-18). D1 is antisymmetric and D2 symmetric on the periodic grid, so
    A6^T lam = sum_axes [-D1((D1 eps) lam) + D2(eps lam)]."""
    out = np.zeros_like(lam)
    for c in range(3):
        out += -fd6_first(fd6_first(eps, c, h) * lam, c, h) + fd6_second(eps * lam, c, h)
    return out


def assemble_A6(eps, h):
    """A6 as a scipy sparse matrix (same definition as apply_A6, Eq. 16-18), flat x-fastest.
    Row i, column i+n along axis c holds (D1 eps)_i alpha_n/h_c + eps_i beta_n/h_c^2."""
    import scipy.sparse as sp
    n = eps.size
    idx = np.arange(n).reshape(eps.shape)
    rows, cols, vals = [], [], []
    diag = np.zeros(eps.shape)
    for c in range(3):
        ax = AX[c]
        de = fd6_first(eps, c, h)
        diag += eps * FD6_BETA[0] / (h[c] * h[c])
        for m in (1, 2, 3):
            for sgn in (1, -1):
                coef = sgn * FD6_ALPHA[m] * de / h[c] + FD6_BETA[m] * eps / (h[c] * h[c])
                rows.append(idx.ravel())
                cols.append(np.roll(idx, -sgn * m, axis=ax).ravel())
                vals.append(coef.ravel())
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def fd6_symbol(grid, h):
    """Eigenvalues of sum_axes D2 (Eq. 18; the eps = 1 case of A6) on the periodic grid,
    sum_axes (beta_0 + 2 sum_n beta_n cos(n theta_a))/h_a^2, in numpy's rfftn
    layout (nz, ny, nx//2+1)."""
    nx, ny, nz = grid

    def axis(N, hh, k):
        t = 2.0 * np.pi * k / N
        return (FD6_BETA[0] + 2.0 * sum(FD6_BETA[n] * np.cos(n * t) for n in (1, 2, 3))) / (hh * hh)

    lx = axis(nx, h[0], np.arange(nx // 2 + 1))
    ly = axis(ny, h[1], np.fft.fftfreq(ny) * ny)
    lz = axis(nz, h[2], np.fft.fftfreq(nz) * nz)
    return lz[:, None, None] + ly[None, :, None] + lx[None, None, :]


def _fd6_lap_inverse(src, lam):
    """Mean-zero solution of (sum_axes D2) u = src - mean(src) by FFT."""
    s = np.fft.rfftn(src)
    l = lam.copy()
    l[0, 0, 0] = 1.0
    s = s / l
    s[0, 0, 0] = 0.0
    return np.fft.irfftn(s, s=src.shape, axes=(0, 1, 2))


def _bordered6(eps, h, rhs, transpose, tol, method):
    """Solve the bordered system K [x; m] = [rhs; 0] with
    K = [[A6, eps], [1^T, 0]] (or its transpose K^T = [[A6^T, 1], [eps^T, 0]]).

    method "direct": sparse LU of K (small grids). method "gmres": restarted
    GMRES on K, preconditioned by the exact inverse of the bordered system
    with A6 replaced by diag(eps) D2 (D2 diag(eps) for the transpose), which
    the FFT inverts. Returns (x, m, iterations, relative residual)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    shape = rhs.shape
    n = rhs.size
    if method is None:
        method = "direct" if n <= 4096 else "gmres"
    col_e = eps.ravel()[:, None]
    nb = np.linalg.norm(rhs)

    def K(v):
        x = v[:n].reshape(shape)
        m = v[n]
        if transpose:
            return np.concatenate([(apply_A6_transpose(x, eps, h) + m).ravel(), [float(np.sum(eps * x))]])
        return np.concatenate([(apply_A6(x, eps, h) + m * eps).ravel(), [float(np.sum(x))]])

    if method == "direct":
        A = assemble_A6(eps, h)
        ones = np.ones((n, 1))
        if transpose:
            Kmat = sp.bmat([[A.T, sp.csr_matrix(ones)], [sp.csr_matrix(col_e.T), None]])
        else:
            Kmat = sp.bmat([[A, sp.csr_matrix(col_e)], [sp.csr_matrix(ones.T), None]])
        v = spl.spsolve(Kmat.tocsc(), np.concatenate([rhs.ravel(), [0.0]]))
        iters = 1
    else:
        lam = fd6_symbol((shape[2], shape[1], shape[0]), h)
        inv_e = 1.0 / eps

        def P(v):
            r = v[:n].reshape(shape)
            s = v[n]
            if transpose:
                # A6^T ~ D2 diag(eps): m = mean(r), eps x = D2^-1 (r - m) + c, sum(eps x) = s
                m = float(np.mean(r))
                x = (_fd6_lap_inverse(r - m, lam) + s / n) * inv_e
            else:
                # A6 ~ diag(eps) D2: r/eps - m has mean zero, x = D2^-1 (r/eps - m) + s/n
                q = r * inv_e
                m = float(np.mean(q))
                x = _fd6_lap_inverse(q - m, lam) + s / n
            return np.concatenate([x.ravel(), [m]])

        count = [0]
        Kop = spl.LinearOperator((n + 1, n + 1), matvec=K)
        Pop = spl.LinearOperator((n + 1, n + 1), matvec=P)
        v, _ = spl.gmres(Kop, np.concatenate([rhs.ravel(), [0.0]]), rtol=tol, atol=0.0, restart=60,
                         maxiter=50, M=Pop, callback=lambda _r: count.__setitem__(0, count[0] + 1),
                         callback_type="pr_norm")
        iters = count[0]
    r = K(v)
    r[:n] -= rhs.ravel()
    res = float(np.linalg.norm(r) / nb) if nb > 0 else float(np.linalg.norm(r))
    return v[:n].reshape(shape), float(v[n]), iters, res


def solve6(rho, eps, h, tol=1e-13, method=None):
    """phi, mu with A6 phi + mu eps = -4 pi rho and sum(phi) = 0 (Eq. 16-18 with
    the compatibility shift described above). rho has its grid mean removed
    first, as for the conservative operator. Returns (phi, mu, SolveInfo); the
    info's residual is ||b - A6 phi - mu eps|| / ||b||."""
    b = -FOUR_PI * (rho - rho.mean())
    phi, mu, it, res = _bordered6(eps, h, b, False, tol, method)
    return phi, mu, SolveInfo(it, res)


def adjoint6(rho, eps, h, tol=1e-13, method=None):
    """lam, nu with A6^T lam + nu = rho - mean(rho) and sum(eps lam) = 0: the
    transposed bordered system, whose solution gives rho . dphi for any change
    of the right side or of eps (Appendix B without the symmetry that makes
    phi its own adjoint for the conservative operator)."""
    lam, nu, it, res = _bordered6(eps, h, rho - rho.mean(), True, tol, method)
    return lam, nu, SolveInfo(it, res)


def residual6_norm(phi, mu, rho, eps, h):
    """||b - A6 phi - mu eps||_2 / ||b||_2 with b = -4 pi (rho - mean(rho)) (Eq. 16-18)."""
    b = -FOUR_PI * (rho - rho.mean())
    r = b - apply_A6(phi, eps, h) - mu * eps
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def energy_gradient6(phi, mu, lam, grid, cell, pos, Z, sigma_core, sigma_cloud,
                     p=DielectricParams(), atoms=None, rho_moves=True, rvdw=None):
    """G_a = dE/dR_a for E = 1/2 h^3 rho.phi (Eq. 4) with phi from the sixth-order
    system (solve6), given its adjoint lam (adjoint6).

    Differentiating [A6 phi + mu eps = b, sum(phi) = 0] and using lam:
      rho . dphi = lam . (db - (dA6) phi - mu d eps),  db = -4 pi d rho,
    and A6 is linear in eps, so lam . (dA6) phi = sum_j d eps_j g_j with
      g = sum_axes [-D1(lam D1 phi) + lam D2 phi].
    Hence
      G^eps_a = -h^3/2 sum_j (d eps_j/dR_a) (g_j + mu lam_j)
      G^rho_a =  h^3/2 sum_j (phi_j - 4 pi lam_j) d rho_j/dR_a,
    with rho = rho~ - mean(rho~). Returns (G_eps, G_rho), each (n_atoms, 3);
    rows of atoms not in `atoms` are zero. `p` is DielectricParams (erf
    product) or GammaParams (Eq. 9-10, with the radii `rvdw`).
    """
    h = spacing(grid, cell)
    dv = cell_volume_element(grid, cell)
    n = len(pos)
    atoms = range(n) if atoms is None else atoms
    gamma_form = isinstance(p, GammaParams)
    if gamma_form:
        G = dummy_density(grid, cell, pos, rvdw, p)
    else:
        P = dielectric_product(grid, cell, pos, p)
    g = np.zeros_like(phi)
    for c in range(3):
        g += -fd6_first(lam * fd6_first(phi, c, h), c, h) + lam * fd6_second(phi, c, h)
    weps = g + mu * lam
    wrho = phi - FOUR_PI * lam
    Ge = np.zeros((n, 3))
    Gr = np.zeros((n, 3))
    for a in atoms:
        if gamma_form:
            de = dielectric_gamma_gradient_atom(a, grid, cell, pos, rvdw, G, p)
        else:
            de = dielectric_gradient_atom(a, grid, cell, pos, P, p)
        for comp in range(3):
            Ge[a, comp] = -0.5 * dv * float(np.sum(de[comp] * weps))
        if rho_moves:
            dr = charge_density_gradient_atom(a, grid, cell, pos, Z, sigma_core, sigma_cloud)
            for comp in range(3):
                Gr[a, comp] = 0.5 * dv * float(np.sum(wrho * (dr[comp] - dr[comp].mean())))
    return Ge, Gr
