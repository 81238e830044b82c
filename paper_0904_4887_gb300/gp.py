"""Thin ctypes binding of the C ABI in ``include/gp.h``.

Every function here only marshals arguments (device pointers of torch
tensors, the stream, plain structs) and calls the library of the same name;
all arithmetic runs in the CUDA kernels of ``libgp_gb300.so``. There is no
fallback: if the library cannot be loaded, or no CUDA device is present when a
compute call is made, the call raises.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

GP_OK = 0
STATUS_NAMES = {0: "GP_OK", 1: "GP_ERR_INVALID_ARG", 2: "GP_ERR_NOT_NEUTRAL", 3: "GP_ERR_NOT_CONVERGED",
                4: "GP_ERR_DIVERGED", 5: "GP_ERR_TIMEOUT", 6: "GP_ERR_CUDA", 7: "GP_ERR_OOM", 8: "GP_ERR_STATE"}
GP_HISTORY = 64


class gp_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class gp_cell(ctypes.Structure):
    _fields_ = [("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double)]


class gp_params(ctypes.Structure):
    _fields_ = [("eps0", ctypes.c_double), ("r0", ctypes.c_double), ("w", ctypes.c_double),
                ("rcut", ctypes.c_double), ("dry_thresh", ctypes.c_double), ("split", ctypes.c_int),
                ("n_dirichlet", ctypes.c_int), ("precision", ctypes.c_int), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("levels", ctypes.c_int), ("inner", ctypes.c_int),
                ("max_outer", ctypes.c_int), ("accel", ctypes.c_int), ("restart", ctypes.c_int),
                ("band_vcycles", ctypes.c_int), ("graph_outer", ctypes.c_int),
                ("sweep_shape", ctypes.c_int), ("kind", ctypes.c_int), ("beta", ctypes.c_double),
                ("zlim", ctypes.c_double), ("nu_coarse", ctypes.c_int), ("inner_adapt", ctypes.c_int),
                ("gamma_tail", ctypes.c_double)]


class gp_stats(ctypes.Structure):
    _fields_ = [("outer_iterations", ctypes.c_int), ("inner_iterations", ctypes.c_int),
                ("vcycles", ctypes.c_int), ("levels", ctypes.c_int), ("split_active", ctypes.c_int),
                ("band_first", ctypes.c_int), ("band_dirichlet", ctypes.c_int), ("dry_planes", ctypes.c_int),
                ("wet_fraction", ctypes.c_double), ("b_norm", ctypes.c_double), ("residual", ctypes.c_double),
                ("history_len", ctypes.c_int), ("history", ctypes.c_double * GP_HISTORY),
                ("sweep_shape", ctypes.c_int), ("gamma_cutoff", ctypes.c_double)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "gp_default_params": (None, [ctypes.POINTER(gp_params)]),
    "gp_create": (ctypes.c_int, [gp_grid, gp_cell, _P, ctypes.POINTER(_P)]),
    "gp_set_dielectric": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.POINTER(gp_params)]),
    "gp_set_vdw_radii": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "gp_build_rho": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "gp_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_double]),
    "gp_energy_forces": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "gp_residual": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "gp_residual6": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, _P, ctypes.POINTER(ctypes.c_double)]),
    "gp_solve6": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double), ctypes.c_double]),
    "gp_adjoint6": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double), ctypes.c_double]),
    "gp_energy_forces6": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, _P, _P, ctypes.POINTER(ctypes.c_double),
                                         _P]),
    "gp_fft_poisson": (ctypes.c_int, [_P, _P, _P]),
    "gp_fft_poisson_f32": (ctypes.c_int, [_P, _P, _P]),
    "gp_get_eps": (ctypes.c_int, [_P, _P]),
    "gp_get_plane_max": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "gp_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(gp_stats)]),
    "gp_last_error": (ctypes.c_char_p, [_P]),
    "gp_destroy": (None, [_P]),
    "gp_plan_band": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "gp_plan_levels": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "gp_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "gp_get_profile": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long),
                                      ctypes.POINTER(ctypes.c_long), ctypes.c_int]),
    "gp_launch_count": (ctypes.c_long, []),
    "gp_residual_noalloc": (ctypes.c_int, [gp_grid, gp_cell, _P, _P, _P, _P, _P, _P]),
}

PROF_KINDS = ["eps", "rho", "forces_eps", "forces_rho", "res64", "smooth0", "mg_fine", "mg_coarse", "krylov",
              "fft", "setup", "misc", "update64", "energy", "smooth0_zero"]


def gp_launch_count():
    return int(load().gp_launch_count())

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libgp_gb300.so (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libgp_gb300.so is missing; run paper_0904_4887_gb300._build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def gp_plan_band(dry, levels, n_dirichlet=1):
    """Host-only band planner; returns (first, nd) or None when no plane is dry."""
    arr = (ctypes.c_int * len(dry))(*[1 if v else 0 for v in dry])
    first, nd = ctypes.c_int(), ctypes.c_int()
    r = load().gp_plan_band(arr, len(dry), int(levels), int(n_dirichlet), ctypes.byref(first), ctypes.byref(nd))
    if r < 0:
        raise ValueError("bad arguments to gp_plan_band")
    return (first.value, nd.value) if r == 1 else None


def gp_plan_levels(nx, ny, nz, zper=1, requested=0):
    return load().gp_plan_levels(int(nx), int(ny), int(nz), int(zper), int(requested))


def gp_residual_noalloc(grid, cell, eps, rho, phi, r, rel, stream=None):
    """Allocation-free FP64 residual (no context); rel is a 1-element device tensor."""
    import torch
    st = torch.cuda.current_stream() if stream is None else stream
    # no size checks here: this wrapper passes its arguments through unchanged so
    # that the C function's own argument checks stay reachable
    return load().gp_residual_noalloc(gp_grid(*grid), gp_cell(*cell), _ptr(eps), _ptr(rho), _ptr(phi), _ptr(r),
                                      _ptr(rel), ctypes.c_void_p(st.cuda_stream))


class GPError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


def default_params(**overrides) -> gp_params:
    p = gp_params()
    load().gp_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(t, numel=None, what="array"):
    """Device pointer of a contiguous float64 CUDA tensor (None passes through).
    The C ABI takes bare pointers and cannot see sizes, so `numel`, when given,
    is checked first: a short array would let the kernels write past its end."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError("%s: expected %d float64 values, got %d" % (what, numel, t.numel()))
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _ptr32(t, numel, what="array"):
    """Device pointer of a contiguous float32 CUDA tensor of `numel` values."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if t.numel() != numel:
        raise ValueError("%s: expected %d float32 values, got %d" % (what, numel, t.numel()))
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _atoms_count(t, what):
    """n for an (n, 3) array of atoms."""
    if t.dim() != 2 or t.shape[1] != 3:
        raise ValueError("%s: expected shape (n, 3), got %s" % (what, tuple(t.shape)))
    return int(t.shape[0])


class Context:
    """Owns one gp_ctx. Methods mirror the C functions one to one."""

    def __init__(self, grid, cell, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the solver has no CPU path")
        lib = load()
        self._lib = lib
        self.grid = tuple(int(v) for v in grid)
        self.cell = tuple(float(v) for v in cell)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = _P()
        st = lib.gp_create(gp_grid(*self.grid), gp_cell(*self.cell), ctypes.c_void_p(stream.cuda_stream),
                           ctypes.byref(h))
        if st != GP_OK:
            raise GPError(st, "gp_create failed (grid extents must be 2^a 3^b, >= 8, nx even)")
        self._h = h
        self.params = None
        self._npts = self.grid[0] * self.grid[1] * self.grid[2]
        self._n_atoms = None          # atoms of the last gp_set_dielectric

    # -- plumbing
    def _check(self, st):
        if st != GP_OK:
            raise GPError(st, self._lib.gp_last_error(self._h).decode())
        return st

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        nx, ny, nz = self.grid
        return (nz, ny, nx)

    # -- the C calls
    def _field(self, t, what):
        return _ptr(t, self._npts, what)

    def gp_set_dielectric(self, atoms, params: gp_params):
        n = _atoms_count(atoms, "atoms")
        p = _ptr(atoms, 3 * n, "atoms")
        self.params = params
        st = self._check(self._lib.gp_set_dielectric(self._h, p, n, ctypes.byref(params)))
        self._n_atoms = n
        return st

    def gp_set_vdw_radii(self, radii):
        if radii.dim() != 1:
            raise ValueError("radii: expected shape (n,), got %s" % (tuple(radii.shape),))
        n = int(radii.shape[0])
        return self._check(self._lib.gp_set_vdw_radii(self._h, _ptr(radii, n, "radii"), n))

    def gp_build_rho(self, atoms, gauss, rho):
        n = _atoms_count(atoms, "atoms")
        return self._check(self._lib.gp_build_rho(self._h, _ptr(atoms, 3 * n, "atoms"), _ptr(gauss, 3 * n, "gauss"),
                                                  n, self._field(rho, "rho")))

    def gp_solve(self, rho, phi, tol, check=True):
        st = self._lib.gp_solve(self._h, self._field(rho, "rho"), self._field(phi, "phi"), ctypes.c_double(tol))
        return self._check(st) if check else st

    def gp_energy_forces(self, phi, rho, gauss=None, forces=None):
        # gauss and forces belong to the atoms of the last gp_set_dielectric
        na = None if self._n_atoms is None else 3 * self._n_atoms
        e = (ctypes.c_double * 2)()
        self._check(self._lib.gp_energy_forces(self._h, self._field(phi, "phi"), self._field(rho, "rho"),
                                               _ptr(gauss, na, "gauss"), e, _ptr(forces, na, "forces")))
        return e[0], e[1]

    def gp_residual(self, rho, phi, r):
        rel = ctypes.c_double()
        self._check(self._lib.gp_residual(self._h, self._field(rho, "rho"), self._field(phi, "phi"),
                                          self._field(r, "r"), ctypes.byref(rel)))
        return rel.value

    def gp_residual6(self, rho, phi, mu, r):
        rel = ctypes.c_double()
        self._check(self._lib.gp_residual6(self._h, self._field(rho, "rho"), self._field(phi, "phi"),
                                           ctypes.c_double(mu), self._field(r, "r"), ctypes.byref(rel)))
        return rel.value

    def gp_solve6(self, rho, phi, tol, check=True):
        mu = ctypes.c_double()
        st = self._lib.gp_solve6(self._h, self._field(rho, "rho"), self._field(phi, "phi"), ctypes.byref(mu),
                                 ctypes.c_double(tol))
        if check:
            self._check(st)
        return mu.value, st

    def gp_adjoint6(self, rho, lam, tol, check=True):
        nu = ctypes.c_double()
        st = self._lib.gp_adjoint6(self._h, self._field(rho, "rho"), self._field(lam, "lam"), ctypes.byref(nu),
                                   ctypes.c_double(tol))
        if check:
            self._check(st)
        return nu.value, st

    def gp_energy_forces6(self, phi, mu, lam, rho, gauss=None, forces=None):
        na = None if self._n_atoms is None else 3 * self._n_atoms
        e = (ctypes.c_double * 1)()
        self._check(self._lib.gp_energy_forces6(self._h, self._field(phi, "phi"), ctypes.c_double(mu),
                                                None if lam is None else self._field(lam, "lam"),
                                                self._field(rho, "rho"), _ptr(gauss, na, "gauss"), e,
                                                _ptr(forces, na, "forces")))
        return e[0]

    def gp_fft_poisson(self, src, out):
        return self._check(self._lib.gp_fft_poisson(self._h, self._field(src, "src"), self._field(out, "out")))

    def gp_fft_poisson_f32(self, src, out):
        return self._check(self._lib.gp_fft_poisson_f32(self._h, _ptr32(src, self._npts, "src"),
                                                        _ptr32(out, self._npts, "out")))

    def gp_get_eps(self, out):
        return self._check(self._lib.gp_get_eps(self._h, self._field(out, "out")))

    def gp_get_plane_max(self):
        import numpy as np
        out = np.zeros(self.grid[2], dtype=np.float64)
        self._check(self._lib.gp_get_plane_max(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def gp_profile(self, enable=True):
        return self._check(self._lib.gp_profile(self._h, 1 if enable else 0))

    def gp_get_profile(self):
        n = len(PROF_KINDS)
        ms = (ctypes.c_double * n)()
        la = (ctypes.c_long * n)()
        gr = (ctypes.c_long * n)()
        self._check(self._lib.gp_get_profile(self._h, ms, la, gr, n))
        return {k: {"ms": ms[i], "launches": la[i], "groups": gr[i]} for i, k in enumerate(PROF_KINDS)}

    def gp_get_stats(self) -> gp_stats:
        s = gp_stats()
        self._check(self._lib.gp_get_stats(self._h, ctypes.byref(s)))
        return s
