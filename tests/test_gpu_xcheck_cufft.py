"""Cross-check of the hand-written FFT Poisson solve (Eq. 15) against cuFFT
through torch.fft, on the device: the same 7-point symbol, the same dropped
k = 0 mode, on grids up to the 96x96x192 split workload. cuFFT serves only
here, as a check; the solver never calls it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import gp_oracle as O

pytestmark = pytest.mark.gpu

GRIDS = [((24, 24, 48), (10.0, 10.0, 20.0)),
         ((32, 32, 64), (10.0, 10.0, 20.0)),
         ((96, 96, 192), (13.0, 13.0, 40.0))]


def _cufft_poisson(src, lam):
    s = torch.fft.rfftn(src, dim=(0, 1, 2))
    lam = lam.clone()
    lam[0, 0, 0] = 1.0
    s = s / lam
    s[0, 0, 0] = 0.0
    return torch.fft.irfftn(s, s=tuple(src.shape), dim=(0, 1, 2))


@pytest.mark.parametrize("k", range(len(GRIDS)))
def test_fft_poisson_matches_cufft(k):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0904_4887_gb300 import GPSolver
    grid, cell = GRIDS[k]
    h = O.spacing(grid, cell)
    s = GPSolver(grid, cell)
    src = torch.tensor(W.random_field(s.shape, seed=40 + k), dtype=torch.float64, device="cuda")
    lam = torch.tensor(O.laplacian_symbol(grid, h), dtype=torch.float64, device="cuda")
    ours = s.fft_poisson(src)
    ref = _cufft_poisson(src, lam)
    err = float((ours - ref).abs().max() / ref.abs().max())
    assert err < 1e-12, err
    assert abs(float(ours.mean())) < 1e-12 * float(ref.abs().max())
