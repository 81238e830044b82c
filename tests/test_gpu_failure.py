"""Failure detection on the GPU without a fault: the whole-row smoothers'
bounded mbarrier waits are made to expire (the test hook sets their poll
budget to zero, so the first wait gives up at once), the kernel drains its own
copies with the normal bound and records the expiry, gp_solve reports
GP_ERR_TIMEOUT after the first outer correction (no V-cycle runs on the
undefined fields that follow), and a new context on the same GPU works
normally."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import gp_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("shape", [4, 7])     # CTA-barrier row tiles; producer-warp row tiles
def test_expired_smoother_wait_reports_timeout_and_gpu_stays_usable(shape):
    from paper_0904_4887_gb300 import GPSolver, GPError
    grid, cell = (64, 48, 48), (10.0, 7.5, 12.0)
    at = W.slab_atoms(cell, 2, 2, seed=0)
    rho = O.charge_density(grid, cell, at.pos, at.Z, at.sigma_core, at.sigma_cloud)
    os.environ["GP_TEST_SWEEP_WAIT_POLLS"] = "0"
    try:
        s = GPSolver(grid, cell, precision=1, sweep_shape=shape)  # whole-row tiles: nx = 64
        s.set_atoms(_t(at.pos))
        with pytest.raises(GPError) as e:
            s.solve(_t(rho), tol=1e-8)
        assert e.value.status == 5                                # GP_ERR_TIMEOUT
        assert "wait expired" in str(e.value)
        # the solve stops at the first residual readback after the expiry: only
        # the initial residual is recorded, and no second correction ran
        st = s.stats()
        assert st.outer_iterations == 1 and st.history_len == 1
        del s
    finally:
        del os.environ["GP_TEST_SWEEP_WAIT_POLLS"]
    s2 = GPSolver(grid, cell, precision=1, sweep_shape=shape)
    s2.set_atoms(_t(at.pos))
    phi = s2.solve(_t(rho), tol=1e-12).cpu().numpy()
    eps = O.dielectric(grid, cell, at.pos)
    ref, _ = O.solve(rho, eps, O.spacing(grid, cell), tol=1e-14)
    assert float(np.max(np.abs(phi - ref)) / np.max(np.abs(ref))) < 1e-8
