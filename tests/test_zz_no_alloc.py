"""The allocation-free residual entry point (gp_residual_noalloc).

It serves callers that cannot allocate device memory: it takes eps, rho, phi
and the output arrays from the caller and keeps its reduction scratch in a
static device array. This test calls it through the C ABI and checks it
against the context-based gp_residual, twice in a row with different inputs
(the shared scratch keeps the previous call's contents). The file name makes
pytest collect it last.
"""
import os
import re

import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import gp_oracle as O

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _max_planes():
    """GP_NOALLOC_MAX_PLANES as the header defines it (so that the limit test
    follows any change of the limit)."""
    text = open(os.path.join(ROOT, "include", "gp.h")).read()
    m = re.search(r"#define\s+GP_NOALLOC_MAX_PLANES\s+(\d+)", text)
    assert m, "GP_NOALLOC_MAX_PLANES is not defined in include/gp.h"
    return int(m.group(1))


G_MAX = _max_planes()


def test_noalloc_residual_matches_gp_residual_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0904_4887_gb300 import GPSolver
    from paper_0904_4887_gb300 import gp as G
    grid, cell = (32, 24, 48), (10.0, 9.0, 15.0)
    at = W.slab_atoms(cell, 2, 2, seed=5)
    dev = "cuda"
    s = GPSolver(grid, cell)
    s.set_atoms(torch.tensor(at.pos, dtype=torch.float64, device=dev))
    eps = s.eps()
    rho = torch.tensor(O.charge_density(grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud),
                       dtype=torch.float64, device=dev)
    for call in range(2):
        phi = torch.tensor(W.random_field(eps.shape, seed=20 + call), dtype=torch.float64, device=dev)
        r_ref, rel_ref = s.residual(rho, phi)
        r = torch.full_like(phi, float("nan"))
        rel = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        st = G.gp_residual_noalloc(grid, cell, eps, rho, phi, r, rel)
        assert st == 0
        torch.cuda.synchronize()
        scale = float(r_ref.abs().max())
        assert float((r - r_ref).abs().max()) <= 1e-13 * scale
        assert abs(float(rel) - rel_ref) <= 1e-12 * rel_ref


def test_noalloc_rejects_too_many_planes():
    """One plane more than the scratch holds is refused before any launch; the
    arrays are grid-sized, so even a call that went ahead would stay in bounds."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0904_4887_gb300 import gp as G
    grid = (8, 8, G_MAX + 1)
    n = grid[0] * grid[1] * grid[2]
    eps = torch.ones(n, dtype=torch.float64, device="cuda")
    rho = torch.zeros(n, dtype=torch.float64, device="cuda")
    phi = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    rel = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    st = G.gp_residual_noalloc(grid, (8.0, 8.0, 8.0 * grid[2] / 8), eps, rho, phi, r, rel)
    torch.cuda.synchronize()
    assert st == 1                                   # GP_ERR_INVALID_ARG
    assert bool((r == 7.0).all()) and float(rel) == 7.0   # nothing was written
