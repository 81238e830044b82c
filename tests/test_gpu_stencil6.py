"""GPU parity of the sixth-order residual (Sec. III, Eq. 16-18) through the C
ABI (gp_residual6) against the oracle's apply_A6, element by element, with the
compatibility shift mu eps of the periodic non-conservative system."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import gp_oracle as O

pytestmark = pytest.mark.gpu

DEV = "cuda"

# extents from 8 up (the smallest the library takes) past a 256-thread row, with
# row counts below and above the 608 reduction blocks
CASES = [((8, 8, 8), (6.5, 6.5, 6.5), 1, 1),
         ((32, 32, 64), (10.0, 10.0, 20.0), 2, 3),
         ((24, 24, 48), (10.0, 10.0, 20.0), 2, 3),
         ((48, 16, 24), (14.0, 7.0, 12.0), 1, 2),
         ((384, 16, 32), (52.0, 8.0, 14.0), 1, 2)]


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0904_4887_gb300 import GPSolver
    return GPSolver


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("k", range(len(CASES)))
@pytest.mark.parametrize("mu", [0.0, 0.37])
def test_residual6_matches_oracle(k, mu):
    GPSolver = _gpu()
    grid, cell, n, layers = CASES[k]
    at = W.slab_atoms(cell, n, layers, seed=k)
    h = O.spacing(grid, cell)
    eps = O.dielectric(grid, cell, at.pos)
    rho = O.charge_density(grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    phi = W.random_field(eps.shape, seed=20 + k)
    s = GPSolver(grid, cell)
    s.set_atoms(_t(at.pos))
    r, rel = s.residual6(_t(rho), _t(phi), mu)
    ref = -4 * math.pi * rho - O.apply_A6(phi, eps, h) - mu * eps
    got = r.cpu().numpy()
    scale = max(np.max(np.abs(O.apply_A6(phi, eps, h))), np.max(np.abs(ref)))
    # eps itself agrees with the oracle to 1e-13 of its maximum, which alone can
    # move A6 phi by ~1e-13 of its scale; FP64 rounding adds far less
    assert np.max(np.abs(got - ref)) < 1e-12 * scale
    assert abs(rel - np.linalg.norm(ref) / np.linalg.norm(4 * math.pi * rho)) < 1e-12 * rel


def test_residual6_of_the_oracle_solution_is_at_its_tolerance():
    """phi, mu from the oracle's bordered solve: the GPU residual of that pair is
    at the oracle's solve tolerance (a property of the solution, at any size)."""
    GPSolver = _gpu()
    grid, cell = (32, 32, 64), (10.0, 10.0, 20.0)
    at = W.slab_atoms(cell, 2, 3, seed=5)
    h = O.spacing(grid, cell)
    eps = O.dielectric(grid, cell, at.pos)
    rho = O.charge_density(grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    rho = rho - rho.mean()
    phi, mu, info = O.solve6(rho, eps, h, tol=1e-13)
    assert info.residual < 1e-12
    s = GPSolver(grid, cell)
    s.set_atoms(_t(at.pos))
    _, rel = s.residual6(_t(rho), _t(phi), mu)
    assert rel < 1e-12
    _, rel0 = s.residual6(_t(rho), _t(phi), 0.0)
    assert rel0 > 10 * rel            # the shift matters on this grid


def test_residual6_errors():
    GPSolver = _gpu()
    s = GPSolver((16, 16, 16), (8.0, 8.0, 8.0))
    z = s.zeros()
    from paper_0904_4887_gb300 import gp as G
    with pytest.raises(RuntimeError):
        s.residual6(z, z, 0.0)        # no dielectric yet
    s.set_atoms(torch.zeros((0, 3), dtype=torch.float64, device=DEV))
    with pytest.raises(RuntimeError):
        s.residual6(z, z, float("nan"))
    r, rel = s.residual6(z, z, 0.0)
    assert float(r.abs().max()) == 0.0
