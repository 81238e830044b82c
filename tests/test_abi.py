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
