"""Every compile-time instance of the hand-written FFT Poisson solve (Eq. 15
with the symbol of the 7-point operator) against the oracle, in both
precisions.

The library compiles one kernel per (precision, extent, pass): the x, y and z
passes each have an instance for every legal extent 8 ... 512. Each extent
below appears in the x, the y and the z position (three cyclic rotations of a
triple of extents), so every instance the library can launch runs here once in
FP64 (gp_fft_poisson) and once in FP32 (gp_fft_poisson_f32, the instance the
mixed-precision split applies). The 192x192x384 workload grid runs at full
size in both precisions as well.

Tolerances, relative to max |phi|: FP64 1e-12 (a few hundred roundings of
1e-16 through three transforms and the division by the symbol); FP32 1e-5 (the
same in 6e-8 arithmetic, the division by the smallest symbol value amplifying
the low modes' rounding). A wrong twiddle, radix step or symbol is an O(1)
error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import gp_oracle as O

pytestmark = pytest.mark.gpu

TRIPLES = [(8, 512, 12), (16, 384, 24), (32, 256, 48), (64, 192, 96), (128, 12, 8)]
GRIDS = [tuple(t[(i + r) % 3] for i in range(3)) for t in TRIPLES for r in range(3)]
EXTENTS = (8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512)


def test_the_grids_cover_every_extent_in_every_position():
    for n in EXTENTS:
        for axis in range(3):
            assert any(g[axis] == n for g in GRIDS), (n, axis)


def _check(grid, seed, fp32_tol=1e-5):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0904_4887_gb300 import GPSolver
    cell = tuple(0.25 * n for n in grid)          # h = 0.25 A on every axis
    h = O.spacing(grid, cell)
    s = GPSolver(grid, cell)
    src = W.random_field(s.shape, seed=seed)
    ref = O.fft_poisson(src, h)
    scale = float(np.max(np.abs(ref)))
    ours = s.fft_poisson(torch.tensor(src, dtype=torch.float64, device="cuda")).cpu().numpy()
    err64 = float(np.max(np.abs(ours - ref))) / scale
    assert err64 < 1e-12, (grid, err64)
    src32 = src.astype(np.float32)
    ref32 = O.fft_poisson(src32.astype(np.float64), h)      # the same input, rounded to FP32
    ours32 = s.fft_poisson_f32(torch.tensor(src32, device="cuda")).cpu().numpy().astype(np.float64)
    err32 = float(np.max(np.abs(ours32 - ref32))) / float(np.max(np.abs(ref32)))
    assert err32 < fp32_tol, (grid, err32)
    assert err32 > 1e-9                                     # it did run in FP32
    return err64, err32


@pytest.mark.parametrize("grid", GRIDS, ids=["x".join(map(str, g)) for g in GRIDS])
def test_every_fft_instance_matches_the_oracle(grid):
    _check(grid, seed=60 + sum(grid))


def test_fft_full_size_workload_grid_both_precisions():
    _check((192, 192, 384), seed=77)
