"""Poisson step and Schroedinger-Poisson loop (Sec. II B) through the C ABI.

`Poisson` wraps khp_poisson_create / khp_poisson_solve / khp_sp_update
(include/khp.h).  `sp_solve` runs the self-consistent loop: the library's
eigensolver (warm-started from the previous iteration), occupations from a
fixed hole number at temperature T (the library's Fermi level over the n
eigenvalues, khp_fermi_level), the library's density, the library's Poisson
solve and potential update.  All grid-sized work runs in the library.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import List

import numpy as np
import torch

from . import _lib
from .solver import _dev, _ptr

KB_EV = 8.617333262e-5   # eV / K
EPS_SI = 11.7


class Poisson:
    """FD Poisson operator on a grid with gate (Dirichlet) points."""

    PRECONDITIONERS = {"jacobi": 0, "multigrid": 1}

    def __init__(self, nx, ny, nz, h, gate_mask, gate_phi, eps_r=EPS_SI, device="cuda", stream=None,
                 preconditioner="multigrid"):
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.nx, self.ny, self.nz, self.h = int(nx), int(ny), int(nz), float(h)
        self.np_ = self.nx * self.ny * self.nz
        self._gate = _dev(np.asarray(gate_mask, dtype=np.uint8).reshape(-1), torch.uint8, self.device)
        self._gphi = _dev(np.asarray(gate_phi, dtype=np.float64).reshape(-1), torch.float64, self.device)
        if self._gate.numel() != self.np_ or self._gphi.numel() != self.np_:
            raise ValueError("gate mask and gate potential need nx*ny*nz entries")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h_ = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self.lib.khp_poisson_create(ctypes.byref(h_), self.nx, self.ny, self.nz, self.h,
                                                   float(eps_r), _ptr(self._gate), _ptr(self._gphi),
                                                   ctypes.c_void_p(self.stream.cuda_stream)))
        self.handle = h_
        self.set_preconditioner(preconditioner)

    def set_preconditioner(self, kind):
        """'multigrid' (geometric V-cycle, the default) or 'jacobi' for the
        later solves; sets and returns `mg_levels`, the multigrid levels in
        use (0: the Jacobi preconditioner, also where the hierarchy could
        not be built)."""
        if kind not in self.PRECONDITIONERS:
            raise ValueError(f"preconditioner must be one of {sorted(self.PRECONDITIONERS)}")
        lv = ctypes.c_int(0)
        _lib.check(self.lib.khp_poisson_set_preconditioner(self.handle, self.PRECONDITIONERS[kind], ctypes.byref(lv)))
        self.preconditioner, self.mg_levels = kind, lv.value
        return lv.value

    def solve(self, rho, phi=None, tol=1e-12, max_iter=20000):
        """phi [Np] (V) for the hole density rho [Np] (nm^-3); `phi` (if
        given) is the starting guess and is overwritten."""
        rho = _dev(rho, torch.float64, self.device).reshape(-1)
        if phi is None:
            phi = torch.zeros(self.np_, dtype=torch.float64, device=self.device)
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        _lib.check(self.lib.khp_poisson_solve(self.handle, _ptr(rho), _ptr(phi), float(tol), int(max_iter),
                                              ctypes.byref(it), ctypes.byref(rel)))
        self.last_iterations, self.last_residual = it.value, rel.value
        return phi

    def solve_many(self, rho, phi=None, grounded=False, tol=1e-12, max_iter=20000):
        """phi [nrhs, Np] (V) of the densities rho [nrhs, Np] (nm^-3),
        solved side by side (khp_poisson_solve_many); grounded=True sets the
        gate potentials to zero.  `phi` (if given) holds the starting
        guesses and is overwritten."""
        rho = _dev(rho, torch.float64, self.device).reshape(-1, self.np_).contiguous()
        nrhs = rho.shape[0]
        if phi is None:
            phi = torch.zeros(nrhs, self.np_, dtype=torch.float64, device=self.device)
        if phi.shape != (nrhs, self.np_) or not phi.is_contiguous():
            raise ValueError("phi must be a contiguous [nrhs, Np] tensor")
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        _lib.check(self.lib.khp_poisson_solve_many(self.handle, _ptr(rho), _ptr(phi), int(nrhs), int(bool(grounded)),
                                                   float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(rel)))
        self.last_iterations, self.last_residual = it.value, rel.value
        return phi

    def update(self, V, phi, mix, V_ext=None):
        """V <- (1 - mix) V + mix (V_ext + phi) in place; returns max |dV|."""
        ch = ctypes.c_double(0.0)
        _lib.check(self.lib.khp_sp_update(self.handle, _ptr(V_ext), _ptr(phi), float(mix), _ptr(V),
                                          ctypes.byref(ch)))
        return ch.value

    def anderson(self, V, phi, beta, depth, V_ext=None):
        """Anderson-mixed update of V in place (khp_sp_anderson: residual
        V_ext + phi - V, history of the last `depth` calls on the handle);
        returns max |dV|."""
        ch = ctypes.c_double(0.0)
        _lib.check(self.lib.khp_sp_anderson(self.handle, _ptr(V_ext), _ptr(phi), float(beta), int(depth), _ptr(V),
                                            ctypes.byref(ch)))
        return ch.value

    def relax(self, dens, E, n_holes, kT, V, V_ext=None, phi=None, tol=1e-12):
        """phi (V) of one update with relaxed occupations
        (khp_sp_relax_occupations); returns (phi, occupations, mu)."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        n = E.size
        if phi is None:
            phi = torch.empty(self.np_, dtype=torch.float64, device=self.device)
        occ = np.zeros(n)
        mu = ctypes.c_double(0.0)
        _lib.check(self.lib.khp_sp_relax_occupations(self.handle, _ptr(dens), _lib.dptr(E), n, float(n_holes),
                                                     float(kT), _ptr(V), _ptr(V_ext), _ptr(phi), float(tol),
                                                     _lib.dptr(occ), ctypes.byref(mu)))
        return phi, occ, mu.value

    def reset_mixing(self):
        _lib.check(self.lib.khp_sp_anderson_reset(self.handle))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.khp_poisson_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fermi_level(E, n_holes, kT):
    """(mu, occupations): the Fermi level holding `n_holes` holes in the
    levels E at thermal energy kT, and the Fermi-Dirac occupations there
    (khp_fermi_level, host side of the library)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    occ = np.empty_like(E)
    mu = ctypes.c_double(0.0)
    lib = _lib.load()
    _lib.check(lib.khp_fermi_level(_lib.dptr(E), int(E.size), float(n_holes), float(kT), ctypes.byref(mu),
                                   _lib.dptr(occ)))
    return mu.value, occ


@dataclass
class SPResult:
    V: torch.Tensor
    evals: np.ndarray
    evecs: torch.Tensor
    mu: float
    occupations: np.ndarray = None
    history: List[float] = field(default_factory=list)
    poisson_iterations: List[int] = field(default_factory=list)


def sp_solve(grid, poisson, V_ext, n_states, n_holes, T=1.5, mix=0.3, iters=20, tol_v=1e-8, strain=None,
             B=None, gauge=0, solve_kw=None, anderson_depth=0, relax=False, warm=True):
    """Self-consistent loop from V = V_ext: `iters` iterations at most, or
    until max |dV| <= tol_v.  Linear mixing with weight `mix`, or Anderson
    mixing (damping `mix`) over `anderson_depth` > 0 previous iterates.
    relax=True relaxes the occupations within each update
    (khp_sp_relax_occupations) instead of fixing them at the Fermi-Dirac
    values of the current levels.  warm=True starts every eigensolve from
    the previous iteration's eigenvectors; warm='block' from the previous
    iteration's whole Ritz block (eigenvectors and guard columns; the first
    solve takes the start of solve_kw); warm=False takes the start of
    solve_kw (e.g. start='coarse').  Returns SPResult (V on the device)."""
    kw = dict(block_m=max(n_states + 8, 16), degree=40, tol=1e-11, seed=1)
    kw.update(solve_kw or {})
    V_ext = _dev(V_ext, torch.float64, grid.device).reshape(-1)
    V = V_ext.clone()
    phi = torch.zeros_like(V)
    kT = KB_EV * T
    hist, piters = [], []
    prev = None
    block = None
    if warm == "block":
        bm = kw["block_m"] + kw["block_m"] % 2
        kw["block_m"] = bm
        block = [torch.empty((grid.N, bm), dtype=torch.complex128, device=grid.device) for _ in range(2)]
    if anderson_depth > 0:
        poisson.reset_mixing()
    for it in range(iters):
        grid.set_fields(V, strain, None, None, B, gauge)
        if block is not None:
            # the previous block starts this solve while the other receives its block
            r = grid.eigensolve(n_states, warm_start=prev, block_out=block[it % 2], **kw)
            prev = block[it % 2]
        else:
            r = grid.eigensolve(n_states, warm_start=prev, **kw)
            prev = r.evecs if warm else None
        if relax:
            dens = grid.state_densities(r.evecs)
            _, f, mu = poisson.relax(dens, r.evals, n_holes, kT, V, V_ext, phi)
            piters.append(0)
        else:
            mu, f = fermi_level(r.evals, n_holes, kT)
            rho = grid.density(r.evecs, f / grid.h ** 3)
            poisson.solve(rho, phi)
            piters.append(poisson.last_iterations)
        if anderson_depth > 0:
            dv = poisson.anderson(V, phi, mix, anderson_depth, V_ext)
        else:
            dv = poisson.update(V, phi, mix, V_ext)
        hist.append(dv)
        if dv <= tol_v:
            break
    return SPResult(V, r.evals, r.evecs, mu, f, hist, piters)
