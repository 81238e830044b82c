"""User-facing solver object and the autograd wrapper.

``GPSolver`` holds one library context (grid, cell, stream) and exposes the
hot path: dielectric from atoms, Gaussian charge density, the generalized
Poisson solve, energy and forces. ``PoissonEnergy`` puts the solve behind
``torch.autograd.Function``: forward returns E = h^3/2 sum rho phi; backward
returns dE/drho = h^3 phi and dE/dR from the library's force kernel. Only phi
is saved for backward; no multigrid state is kept (the operator is symmetric,
so phi is its own adjoint: Appendix B of the paper).
"""
from __future__ import annotations

import math

import torch

from . import gp as _gp


class GPSolver:
    def __init__(self, grid, cell, stream=None, **params):
        self.ctx = _gp.Context(grid, cell, stream)
        self.params = _gp.default_params(**params)
        self.grid = self.ctx.grid
        self.cell = self.ctx.cell
        self.dv = (self.cell[0] / self.grid[0]) * (self.cell[1] / self.grid[1]) * (self.cell[2] / self.grid[2])
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._atoms_version = 0
        self._atoms_key = None

    @property
    def shape(self):
        return self.ctx.shape

    def zeros(self):
        return torch.zeros(self.shape, dtype=torch.float64, device=self.device)

    def set_atoms(self, pos: torch.Tensor, radii: torch.Tensor = None, **params):
        """Build eps(R) and the multigrid hierarchy for these atom positions.
        `radii`: van der Waals radii (Angstrom, one per atom) for the kind-1
        dielectric of Eq. 9-10; kept by the context for later calls."""
        for k, v in params.items():
            setattr(self.params, k, v)
        if radii is not None:
            self.ctx.gp_set_vdw_radii(radii.detach().to(self.device, torch.float64).contiguous())
        pos = pos.detach().to(self.device, torch.float64).contiguous()
        self.ctx.gp_set_dielectric(pos, self.params)
        self._atoms_version += 1
        self._atoms_key = (pos.data_ptr(), pos._version, self._atoms_version)
        self._pos = pos
        return self._atoms_version

    def build_rho(self, pos: torch.Tensor, gauss: torch.Tensor, out=None):
        out = self.zeros() if out is None else out
        self.ctx.gp_build_rho(pos.detach().contiguous(), gauss.detach().contiguous(), out)
        return out

    def solve(self, rho: torch.Tensor, phi=None, tol=1e-10, check=True):
        """phi with div(eps grad phi) = -4 pi rho; `phi` (if given) is the warm start and is overwritten."""
        phi = self.zeros() if phi is None else phi
        st = self.ctx.gp_solve(rho, phi, tol, check=check)
        return phi if check else (phi, st)

    def energy_forces(self, phi, rho, gauss=None, forces=True):
        F = torch.zeros((self._pos.shape[0], 3), dtype=torch.float64, device=self.device) if forces else None
        E, E2 = self.ctx.gp_energy_forces(phi, rho, gauss, F)
        return E, E2, F

    def residual(self, rho, phi):
        r = self.zeros()
        rel = self.ctx.gp_residual(rho, phi, r)
        return r, rel

    def residual6(self, rho, phi, mu=0.0):
        """b - A6 phi - mu eps with the sixth-order operator of Eq. 16-18, and its
        norm relative to b = -4 pi rho."""
        r = self.zeros()
        rel = self.ctx.gp_residual6(rho, phi, mu, r)
        return r, rel

    def solve6(self, rho, phi=None, tol=1e-10):
        """(phi, mu) of the sixth-order bordered system A6 phi + mu eps =
        -4 pi (rho - mean rho), sum(phi) = 0 (Sec. III); `phi` is the warm start."""
        phi = self.zeros() if phi is None else phi
        mu, _ = self.ctx.gp_solve6(rho, phi, tol)
        return phi, mu

    def adjoint6(self, rho, lam=None, tol=1e-10):
        """(lam, nu) of the transposed system A6^T lam + nu = rho - mean rho,
        sum(eps lam) = 0, which the sixth-order forces need."""
        lam = self.zeros() if lam is None else lam
        nu, _ = self.ctx.gp_adjoint6(rho, lam, tol)
        return lam, nu

    def energy_forces6(self, phi, mu, lam, rho, gauss=None, forces=True):
        """E and -dE/dR for the sixth-order solution (phi, mu) with its adjoint lam."""
        F = torch.zeros((self._pos.shape[0], 3), dtype=torch.float64, device=self.device) if forces else None
        E = self.ctx.gp_energy_forces6(phi, mu, lam, rho, gauss, F)
        return E, F

    def fft_poisson(self, src):
        out = self.zeros()
        self.ctx.gp_fft_poisson(src.contiguous(), out)
        return out

    def fft_poisson_f32(self, src):
        """The FP32 instance of the vacuum solve (the one the mixed split uses)."""
        out = torch.zeros(self.shape, dtype=torch.float32, device=self.device)
        self.ctx.gp_fft_poisson_f32(src.contiguous(), out)
        return out

    def eps(self):
        out = self.zeros()
        self.ctx.gp_get_eps(out)
        return out

    def plane_max(self):
        return self.ctx.gp_get_plane_max()

    def stats(self):
        return self.ctx.gp_get_stats()


class PoissonEnergy(torch.autograd.Function):
    """E(pos, rho) = h^3/2 sum rho phi with div(eps(pos) grad phi) = -4 pi rho.

    forward(pos, rho, solver, tol, gauss) -> (E, phi); phi is returned
    detached. If `gauss` is given, rho is taken to be the Gaussian density of
    those atoms, so dE/dpos includes the charge-motion term of Eq. 11;
    otherwise rho is an independent input and dE/dpos is the dielectric
    ("solvent") term only.
    """

    @staticmethod
    def forward(ctx, pos, rho, solver: GPSolver, tol=1e-10, gauss=None):
        solver.set_atoms(pos)
        rho = rho.detach().contiguous()
        phi = solver.solve(rho, tol=tol)
        E, _, _ = solver.energy_forces(phi, rho, None, forces=False)
        ctx.solver = solver
        ctx.gauss = gauss
        ctx.key = solver._atoms_key
        ctx.save_for_backward(pos.detach(), rho, phi)
        ctx.mark_non_differentiable(phi)
        return torch.tensor(E, dtype=torch.float64, device=rho.device), phi

    @staticmethod
    def backward(ctx, gE, gphi):
        pos, rho, phi = ctx.saved_tensors
        solver = ctx.solver
        if solver._atoms_key != ctx.key:
            solver.set_atoms(pos)          # recompute eps: nothing else was stored
        _, _, F = solver.energy_forces(phi, rho, ctx.gauss, forces=True)
        g = gE.to(torch.float64)
        grad_pos = (-F) * g if ctx.needs_input_grad[0] else None
        grad_rho = (solver.dv * phi) * g if ctx.needs_input_grad[1] else None
        return grad_pos, grad_rho, None, None, None


def poisson_energy(pos, rho, solver, tol=1e-10, gauss=None):
    E, phi = PoissonEnergy.apply(pos, rho, solver, tol, gauss)
    return E, phi
