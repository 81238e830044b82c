"""The C ABI library loads on a machine without a GPU, exports every function
that include/gp.h declares, and its host-only planners agree with the oracle."""
import os
import re

import numpy as np
import pytest

from paper_0904_4887_gb300 import gp as G
from oracle import gp_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gp_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = G.load()
    names = declared_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(G._SIGNATURES)


def test_default_params_host_only():
    p = G.default_params()
    assert p.eps0 == 78.36 and p.r0 == 2.5 and p.w == 0.5 and p.rcut == 6.0
    assert p.dry_thresh == 1e-3 and p.nu1 == 2 and p.nu2 == 2 and p.precision == 1


@pytest.mark.parametrize("seed", range(40))
def test_band_planner_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    nz = int(rng.choice([16, 24, 32, 48, 64]))
    dry = np.zeros(nz, dtype=bool)
    for _ in range(int(rng.integers(0, 4))):
        a = int(rng.integers(0, nz)); L = int(rng.integers(1, nz // 2))
        dry[[(a + t) % nz for t in range(L)]] = True
    for levels in (2, 3, 4):
        for nd in (0, 1, 3, 5):
            assert G.gp_plan_band(dry, levels, nd) == O.plan_band(dry, levels, nd)


def test_level_planner():
    assert G.gp_plan_levels(32, 32, 64) == 5          # 2 x 2 x 4 = 16 points
    assert G.gp_plan_levels(192, 192, 384) == 7       # 3 x 3 x 6 = 54
    assert G.gp_plan_levels(96, 96, 192, 1, 5) == 5   # requested: 6 x 6 x 12 = 432
    assert G.gp_plan_levels(8, 8, 8) == 2
    assert G.gp_plan_levels(192, 192, 383, 0) == 7    # Dirichlet band: (383+1)/64 - 1 = 5 planes
    assert G.gp_plan_levels(96, 96, 192, 1, 9) == -1


def _levels_rule(nx, ny, nz, zper, requested):
    """The documented level rule, restated: coarse extents at depth l, then the
    requested count or the automatic choice (<= 64 points, else <= 512)."""
    def coarse(l):
        m = 2 ** l
        if nx % m or ny % m:
            return None
        cx, cy = nx // m, ny // m
        if zper:
            if nz % m:
                return None
            cz = nz // m
            if cz < 2:
                return None
        else:
            if (nz + 1) % m:
                return None
            cz = (nz + 1) // m - 1
            if cz < 1:
                return None
        if cx < 2 or cy < 2:
            return None
        return cx * cy * cz
    if requested > 0:
        pts = coarse(requested - 1) if requested <= 16 else None
        return requested if pts is not None and pts <= 512 else -1
    depths = []
    for l in range(1, 16):
        pts = coarse(l)
        if pts is None:
            break
        depths.append((l, pts))
    for l, pts in depths:
        if pts <= 64:
            return l + 1
    ok = [l for l, pts in depths if pts <= 512]
    return max(ok) + 1 if ok else -1


def test_level_planner_matches_the_documented_rule():
    ext = [8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512]
    dir_nz = [7, 11, 15, 23, 31, 47, 63, 95, 127, 191, 255, 383, 9, 13]
    cases = 0
    for nx in ext:
        for ny in ext[::2]:
            for zper, zs in ((1, ext), (0, dir_nz)):
                for nz in zs:
                    for req in (0, 1, 2, 3, 5, 7, 9, 17):
                        got = G.gp_plan_levels(nx, ny, nz, zper, req)
                        assert got == _levels_rule(nx, ny, nz, zper, req), (nx, ny, nz, zper, req, got)
                        cases += 1
    assert cases > 2000


def test_binding_checks_array_sizes_before_any_device_call():
    """The C ABI takes bare pointers, so the binding checks every array's size
    against the grid (or the atom count) first: a wrong size raises ValueError
    before the CUDA check; a right size gets as far as the CUDA check (no GPU
    here)."""
    import torch
    class NoLib:                                  # every C function fails if it is ever reached
        def __getattr__(self, name):
            def reached(*args):
                raise AssertionError("%s reached the library" % name)
            return reached

    ctx = G.Context.__new__(G.Context)          # no gp_create: nothing reaches the library
    ctx.grid, ctx._npts, ctx._n_atoms, ctx._h = (8, 8, 16), 8 * 8 * 16, 5, None
    ctx._lib = NoLib()
    good = torch.zeros((16, 8, 8), dtype=torch.float64)
    short = torch.zeros((16, 8, 7), dtype=torch.float64)
    # on the CPU every right-sized tensor stops at the CUDA check, so each call
    # varies the first array it checks
    calls = [lambda a: ctx.gp_solve(a, good, 1e-8), lambda a: ctx.gp_residual(a, good, good),
             lambda a: ctx.gp_residual6(a, good, 0.0, good), lambda a: ctx.gp_fft_poisson(a, good),
             lambda a: ctx.gp_get_eps(a), lambda a: ctx.gp_energy_forces(a, good)]
    for call in calls:
        with pytest.raises(ValueError):
            call(short)
        with pytest.raises(TypeError):          # size fine: stops at "not a CUDA tensor"
            call(good)
    atoms5 = torch.zeros((5, 3), dtype=torch.float64)
    with pytest.raises(TypeError):
        ctx.gp_build_rho(atoms5, atoms5, good)
    for bad in (torch.zeros(15, dtype=torch.float64), torch.zeros((5, 2), dtype=torch.float64)):
        with pytest.raises(ValueError):
            ctx.gp_set_dielectric(bad, G.gp_params())           # not (n, 3)
        with pytest.raises(ValueError):
            ctx.gp_build_rho(bad, atoms5, good)
    with pytest.raises(ValueError):
        ctx.gp_set_vdw_radii(torch.zeros((5, 1), dtype=torch.float64))
    with pytest.raises(ValueError):
        G._ptr(torch.zeros(7, dtype=torch.float64), 8, "x")


def test_host_argument_checks_return_before_any_device_work():
    """Calls whose arguments are rejected on the host return their status
    without touching CUDA, so they behave the same on a machine without a GPU:
    bad extents or cell for gp_create, and every context call given a NULL
    context."""
    import ctypes
    lib = G.load()
    INVALID = 1                                             # GP_ERR_INVALID_ARG
    h = ctypes.c_void_p(123)
    for grid, cell in (((10, 16, 16), (8.0, 8.0, 8.0)),     # 10 is not 2^a 3^b
                       ((4, 16, 16), (8.0, 8.0, 8.0)),      # below 8
                       ((24, 16, 18), (8.0, 8.0, 8.0)),     # 18 = 2 * 9
                       ((16, 16, 16), (8.0, 0.0, 8.0))):    # non-positive side
        assert lib.gp_create(G.gp_grid(*grid), G.gp_cell(*cell), None, ctypes.byref(h)) == INVALID
        assert h.value is None                              # *out is cleared
    assert lib.gp_create(G.gp_grid(16, 16, 16), G.gp_cell(8.0, 8.0, 8.0), None, None) == INVALID
    p = G.gp_params()
    lib.gp_default_params(ctypes.byref(p))
    assert lib.gp_set_dielectric(None, None, 0, ctypes.byref(p)) == INVALID
    assert lib.gp_set_vdw_radii(None, None, 0) == INVALID
    assert lib.gp_build_rho(None, None, None, 0, None) == INVALID
    assert lib.gp_solve(None, None, None, ctypes.c_double(1e-8)) == INVALID
    assert lib.gp_energy_forces(None, None, None, None, None, None) == INVALID
    assert lib.gp_residual(None, None, None, None, None) == INVALID
    assert lib.gp_residual6(None, None, None, ctypes.c_double(0.0), None, None) == INVALID
    assert lib.gp_fft_poisson(None, None, None) == INVALID
    assert lib.gp_get_eps(None, None) == INVALID
    assert lib.gp_get_plane_max(None, None) == INVALID
    assert lib.gp_get_stats(None, None) == INVALID
    assert lib.gp_profile(None, 1) == INVALID
    assert lib.gp_last_error(None) == b"null context"
    lib.gp_destroy(None)                                    # a no-op
