"""The allocation-free residual entry point (gp_residual_noalloc).

It serves callers that cannot allocate device memory: it takes eps, rho, phi
and the output arrays from the caller and keeps its reduction scratch in a
static device array. This test calls it through the C ABI and checks it
against the context-based gp_residual, twice in a row with different inputs
(the shared scratch keeps the previous call's contents). The file name makes
pytest collect it last.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import gp_oracle as O

pytestmark = pytest.mark.gpu


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
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0904_4887_gb300 import gp as G
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = G.gp_residual_noalloc((8, 8, G_MAX + 1), (8.0, 8.0, 8.0), x, x, x, x, x)
    assert st == 1


G_MAX = 4096
