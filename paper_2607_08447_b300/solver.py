"""Python front end of the CUDA k.p hole eigensolver (marshalling only).

`KPGrid` wraps one C-ABI handle.  Device arrays are torch CUDA tensors
(float64, complex128 or complex64) and are passed by pointer; all
arithmetic runs in libkhp's kernels.  `KPEigs` is a torch.autograd.Function
whose backward is the library's Hellmann-Feynman adjoint.
"""
from __future__ import annotations

import ctypes
import json
import os
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib

_MAT_KEYS = ("gamma1", "gamma2", "gamma3", "delta_so", "kappa", "a_v", "b", "d")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype, device):
    if t is None:
        return None
    if not torch.is_tensor(t):
        t = torch.as_tensor(np.ascontiguousarray(t))
    return t.to(device=device, dtype=dtype).contiguous()


def _log_solve(grid, opts, stats, evals, status):
    """With KHP_LOG_JSONL=<path> in the environment, append one JSON object
    per eigensolve: grid, options, status, eigenvalues, the per-phase device
    times and the residual history of the outer iterations."""
    path = os.environ.get("KHP_LOG_JSONL")
    if not path:
        return
    rec = {"time": time.time(), "grid": [grid.nx, grid.ny, grid.nz], "bands": grid.bands,
           "n_states": opts.n_states, "block_m": opts.block_m, "degree": opts.degree,
           "precision": opts.precision, "tol_ev": opts.tol_ev, "status": int(status),
           "evals": [float(e) for e in evals], "stats": stats}
    with open(path, "a") as fh:
        fh.write(json.dumps(rec) + "\n")


@dataclass
class SolveResult:
    evals: np.ndarray          # float64 [n], ascending
    evecs: torch.Tensor        # complex128 [N, n] on the device
    residuals: np.ndarray      # float64 [n]
    stats: dict
    status: int


class KPGrid:
    """One grid + Hamiltonian on one CUDA device (see include/khp.h)."""

    def __init__(self, nx, ny, nz, h, material, rot=None, mask=None, device="cuda", stream=None, bands=6):
        """bands = 6: the k.p hole Hamiltonian with spin-orbit coupling;
        bands = 3: the spin-independent H0 block (no spin-orbit, B = 0)."""
        if bands not in (6, 3):
            raise ValueError("bands must be 6 or 3")
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.nx, self.ny, self.nz, self.h = int(nx), int(ny), int(nz), float(h)
        self.np_ = self.nx * self.ny * self.nz
        self.bands = bands
        self.N = bands * self.np_
        mat = _lib.Material(*[float(material[k]) for k in _MAT_KEYS])
        R = None if rot is None else np.ascontiguousarray(np.asarray(rot, dtype=np.float64).reshape(9))
        self._mask = None if mask is None else _dev(np.asarray(mask, dtype=np.uint8).reshape(-1), torch.uint8, self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h_ = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            create = self.lib.khp_create_grid if bands == 6 else self.lib.khp_create_grid_h0
            _lib.check(create(ctypes.byref(h_), self.nx, self.ny, self.nz, self.h,
                              ctypes.byref(mat), _lib.dptr(R), _ptr(self._mask),
                              ctypes.c_void_p(self.stream.cuda_stream)))
        self.handle = h_
        self.material = dict(material)
        self.rot = R

    @classmethod
    def from_problem(cls, p, device="cuda", with_levers=True, bands=6):
        """Grid + fields from any object with the attributes nx, ny, nz, h,
        material, rot, mask, V, strain, B, gauge and (optionally) levers.
        bands = 3 builds the spin-independent H0 (the field B is dropped)."""
        g = cls(p.nx, p.ny, p.nz, p.h, p.material, p.rot, getattr(p, "mask", None), device=device, bands=bands)
        lev = getattr(p, "levers", None) if with_levers else None
        B = p.B if bands == 6 else (0.0, 0.0, 0.0)
        g.set_fields(p.V, p.strain, lev, None if lev is None else np.zeros(lev.shape[0]), B, p.gauge)
        return g

    # ------------------------------------------------------------------
    def set_fields(self, V, strain=None, levers=None, alpha=None, B=None, gauge=0):
        V = _dev(V, torch.float64, self.device).reshape(-1)
        if V.numel() != self.np_:
            raise ValueError("V must have nx*ny*nz entries")
        strain = _dev(strain, torch.float64, self.device)
        if strain is not None and strain.numel() != 6 * self.np_:
            raise ValueError("strain must have 6*nx*ny*nz entries")
        levers = _dev(levers, torch.float64, self.device)
        ng = 0 if levers is None else levers.numel() // self.np_
        a = None
        if ng:
            a = np.ascontiguousarray(np.zeros(ng) if alpha is None else np.asarray(alpha, dtype=np.float64))
        Bh = None if B is None else np.ascontiguousarray(np.asarray(B, dtype=np.float64))
        _lib.check(self.lib.khp_set_potential_strain_field(self.handle, _ptr(V), _ptr(strain), _ptr(levers),
                                                           _lib.dptr(a), ng, _lib.dptr(Bh), int(gauge)))
        self._keep = (V, strain, levers)   # alive until the stream has consumed them
        self._fields = (V, strain, levers, a, ng, int(gauge))
        self.B = np.zeros(3) if Bh is None else Bh.copy()
        return self

    def set_B(self, B):
        """Change only the magnetic field (the other fields as last set)."""
        V, strain, levers, a, ng, gauge = self._fields
        Bh = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(3))
        _lib.check(self.lib.khp_set_potential_strain_field(self.handle, _ptr(V), _ptr(strain), _ptr(levers),
                                                           _lib.dptr(a), ng, _lib.dptr(Bh), gauge))
        self.B = Bh.copy()
        return self

    def apply(self, X, precision=0):
        """Y = H X for X complex128 (precision 0) or complex64 (1), shape [N, m]."""
        dt = torch.complex128 if precision == 0 else torch.complex64
        X = _dev(X, dt, self.device)
        if X.dim() == 1:
            X = X.reshape(-1, 1)
        m = X.shape[1]
        Y = torch.empty_like(X)
        _lib.check(self.lib.khp_apply(self.handle, _ptr(X), _ptr(Y), m, int(precision)))
        return Y

    def filter_step(self, x, y, alpha, beta, gamma=0.0, prev=None, src=None, src_coef=None, col0=0, ncol=None,
                    precision=1):
        """One fused Chebyshev step into y (khp_filter_step) on the columns
        [col0, col0 + ncol):  y = alpha H x + beta x + gamma prev + src_coef[col] src.
        x, prev, src, y: [N, ld] complex64 (precision 1) or complex128 (0)."""
        dt = torch.complex128 if precision == 0 else torch.complex64
        x = _dev(x, dt, self.device)
        prev = _dev(prev, dt, self.device)
        src = _dev(src, dt, self.device)
        ld = x.shape[1]
        ncol = ld - col0 if ncol is None else ncol
        sc = None if src_coef is None else np.ascontiguousarray(np.asarray(src_coef, dtype=np.float64).reshape(ld))
        _lib.check(self.lib.khp_filter_step(self.handle, _ptr(x), _ptr(prev), _ptr(src), _lib.dptr(sc), _ptr(y),
                                            ld, int(col0), int(ncol), float(alpha), float(beta), float(gamma),
                                            int(precision)))
        return y

    def project_rows(self, Y, W=None, method=0):
        """Y^H Y and Y^H W for any complex128 [rows][m] blocks (see project)."""
        Y = _dev(Y, torch.complex128, self.device)
        W = _dev(W, torch.complex128, self.device)
        rows, m = Y.shape
        G = np.zeros((m, m), dtype=np.complex128)
        S = np.zeros((m, m), dtype=np.complex128) if W is not None else None
        _lib.check(self.lib.khp_project_rows(self.handle, _ptr(Y), _ptr(W), int(rows), m, int(method),
                                             G.ctypes.data_as(ctypes.c_void_p),
                                             None if S is None else S.ctypes.data_as(ctypes.c_void_p)))
        return G, S

    def project(self, Y, W=None, method=0):
        """G = Y^H Y and S = Y^H W (Hermitian, from their upper triangles):
        method 0 on the tcgen05 tensor cores (split-digit products, FP64
        accurate, m <= 32), 1 on the FP64 ALUs, 2 the same products through
        mma.sync.  Returns numpy (G, S or None)."""
        Y = _dev(Y, torch.complex128, self.device)
        W = _dev(W, torch.complex128, self.device)
        m = Y.shape[1]
        G = np.zeros((m, m), dtype=np.complex128)
        S = np.zeros((m, m), dtype=np.complex128) if W is not None else None
        _lib.check(self.lib.khp_project(self.handle, _ptr(Y), _ptr(W), m, int(method),
                                        G.ctypes.data_as(ctypes.c_void_p),
                                        None if S is None else S.ctypes.data_as(ctypes.c_void_p)))
        return G, S

    def rotate(self, Y, Q, W=None, method=0, out=None, out_w=None):
        """X = Y Q and HX = W Q (method as in project); out/out_w may be Y/W."""
        Y = _dev(Y, torch.complex128, self.device)
        W = _dev(W, torch.complex128, self.device)
        m = Y.shape[1]
        Qh = np.ascontiguousarray(np.asarray(Q, dtype=np.complex128))
        X = out if out is not None else torch.empty_like(Y)
        HX = (out_w if out_w is not None else torch.empty_like(W)) if W is not None else None
        _lib.check(self.lib.khp_rotate(self.handle, _ptr(Y), _ptr(W), Qh.ctypes.data_as(ctypes.c_void_p), m,
                                       int(method), _ptr(X), _ptr(HX)))
        return X, HX

    def eigensolve(self, n_states, block_m=None, degree=20, max_iter=0, precision=0, refine_sweeps=2,
                   tol=1e-9, seed=1, warm_start=None, out=None, allow_not_converged=False, projections="tensor",
                   start="random", block_out=None):
        """Lowest n_states eigenpairs (khp_eigensolve).  start: 'random'
        (counter-based start block) or 'coarse' (the block of the 2x coarser
        grid, prolongated); a warm_start block takes precedence.
        block_out: a contiguous complex128 [N, block_m] device tensor that
        receives the final Ritz block (all block_m columns)."""
        block_m = block_m or max(n_states + 8, 16)
        block_m += block_m % 2
        opts = _lib.SolverOpts()
        opts.n_states, opts.block_m, opts.degree, opts.max_iter = n_states, block_m, degree, max_iter
        opts.precision, opts.refine_sweeps, opts.tol_ev, opts.seed = precision, refine_sweeps, tol, seed
        opts.projections = _projections(projections)
        if start not in ("random", "coarse", 0, 1):
            raise ValueError("start must be 'random' or 'coarse'")
        opts.start = 1 if start in ("coarse", 1) else 0
        ws = None
        if warm_start is not None:
            ws = _dev(warm_start, torch.complex128, self.device)
            opts.warm_start_dev = ctypes.c_void_p(ws.data_ptr())
            opts.warm_cols = ws.shape[1]
        if block_out is not None:
            if (block_out.dtype != torch.complex128 or tuple(block_out.shape) != (self.N, block_m)
                    or not block_out.is_contiguous() or not block_out.is_cuda):
                raise ValueError("block_out must be a contiguous complex128 [N, block_m] CUDA tensor")
            opts.block_out_dev = ctypes.c_void_p(block_out.data_ptr())
        evals = np.zeros(n_states)
        res = np.zeros(n_states)
        evecs = out if out is not None else torch.empty((self.N, n_states), dtype=torch.complex128, device=self.device)
        st = _lib.Stats()
        status = self.lib.khp_eigensolve(self.handle, ctypes.byref(opts), _lib.dptr(evals), _ptr(evecs),
                                         _lib.dptr(res), ctypes.byref(st))
        stats = st.as_dict()
        _log_solve(self, opts, stats, evals, status)
        _lib.check(status, allow=(4,) if allow_not_converged else ())
        return SolveResult(evals, evecs, res, stats, status)

    def density(self, evecs, w):
        evecs = _dev(evecs, torch.complex128, self.device)
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        rho = torch.empty(self.np_, dtype=torch.float64, device=self.device)
        _lib.check(self.lib.khp_density(self.handle, _ptr(evecs), evecs.shape[1], _lib.dptr(w), _ptr(rho)))
        return rho

    def position_moments(self, X):
        """[3][m][m] numpy: sum_p r_a(p) X(p)^H X(p), r_a the coordinate (nm)
        about the box centre (khp_position_moments)."""
        X = _dev(X, torch.complex128, self.device)
        m = X.shape[1]
        D = np.zeros((3, m, m), dtype=np.complex128)
        _lib.check(self.lib.khp_position_moments(self.handle, _ptr(X), m, D.ctypes.data_as(ctypes.c_void_p)))
        return D

    def state_densities(self, evecs):
        """float64 [n][Np]: sum_b |psi_i(p, b)|^2 per state (khp_state_densities)."""
        evecs = _dev(evecs, torch.complex128, self.device)
        n = evecs.shape[1]
        out = torch.empty((n, self.np_), dtype=torch.float64, device=self.device)
        _lib.check(self.lib.khp_state_densities(self.handle, _ptr(evecs), n, _ptr(out)))
        return out

    def pair_densities(self, evecs):
        """rho_jl(p) = sum_b conj(psi_j) psi_l for all ordered (j, l):
        complex128 [Np][n * n], pair index j n + l."""
        evecs = _dev(evecs, torch.complex128, self.device)
        n = evecs.shape[1]
        out = torch.empty((self.np_, n * n), dtype=torch.complex128, device=self.device)
        _lib.check(self.lib.khp_pair_densities(self.handle, _ptr(evecs), n, _ptr(out)))
        return out

    def backward(self, evecs, evals, dLdE, levers=None, want_strain=True):
        evecs = _dev(evecs, torch.complex128, self.device)
        n = evecs.shape[1]
        ev = np.ascontiguousarray(np.asarray(evals, dtype=np.float64))
        g = np.ascontiguousarray(np.asarray(dLdE, dtype=np.float64))
        dV = torch.empty(self.np_, dtype=torch.float64, device=self.device)
        dE = torch.empty(6 * self.np_, dtype=torch.float64, device=self.device) if want_strain else None
        levers = _dev(levers, torch.float64, self.device)
        ng = 0 if levers is None else levers.numel() // self.np_
        da = np.zeros(max(ng, 1))
        _lib.check(self.lib.khp_eigs_backward(self.handle, _ptr(evecs), _lib.dptr(ev), n, _lib.dptr(g), _ptr(dV),
                                              _ptr(dE), _ptr(levers), ng, _lib.dptr(da)))
        return dV, dE, (da[:ng] if ng else None)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.khp_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _projections(p):
    """'tensor' (split-digit products on the tcgen05 tensor cores, the
    default), 'fp64' (FP64 ALU) or 'mma' (the same products through the
    warp-level mma.sync tensor-core path)."""
    if p in ("tensor", "tcgen05", 0):
        return 0
    if p in ("fp64", 1):
        return 1
    if p in ("mma", 2):
        return 2
    raise ValueError("projections must be 'tensor', 'fp64' or 'mma'")


def solve_batched(grids, n_states, block_m=None, degree=80, max_iter=0, precision=0, refine_sweeps=-1,
                  tol=1e-9, seed=1, graph=True, autotune=False, allow_not_converged=False, projections="tensor",
                  grouped=False, start="random"):
    """Solve every grid's lowest states in one khp_eigensolve_batched call
    (lock-step rounds, optionally one CUDA graph per round, an autotuned
    block width, and grouped filter launches across the problems).  start
    'coarse' solves the problems' coarse grids together first and starts
    each from its prolongated block.  Returns a list of SolveResult."""
    lib = _lib.load()
    count = len(grids)
    opts = _lib.SolverOpts()
    bm = block_m or max(n_states + 8, 16)
    opts.n_states, opts.block_m, opts.degree, opts.max_iter = n_states, bm + bm % 2, degree, max_iter
    opts.precision, opts.refine_sweeps, opts.tol_ev, opts.seed = precision, refine_sweeps, tol, seed
    opts.projections = _projections(projections)
    if start not in ("random", "coarse", 0, 1):
        raise ValueError("start must be 'random' or 'coarse'")
    opts.start = 1 if start in ("coarse", 1) else 0
    hs = (ctypes.c_void_p * count)(*[g.handle.value for g in grids])
    outs = [torch.empty((g.N, n_states), dtype=torch.complex128, device=g.device) for g in grids]
    ptrs = (ctypes.c_void_p * count)(*[o.data_ptr() for o in outs])
    evals = np.zeros((count, n_states))
    res = np.zeros((count, n_states))
    st = (_lib.Stats * count)()
    flags = ((_lib.KHP_BATCH_GRAPH if graph else 0) | (_lib.KHP_BATCH_AUTOTUNE if autotune else 0)
             | (_lib.KHP_BATCH_GROUPED if grouped else 0))
    status = lib.khp_eigensolve_batched(hs, count, ctypes.byref(opts), _lib.dptr(evals), ptrs,
                                        _lib.dptr(res), st, flags)
    _lib.check(status, allow=(4,) if allow_not_converged else ())
    return [SolveResult(evals[i].copy(), outs[i], res[i].copy(), st[i].as_dict(), status) for i in range(count)]


class KPEigs(torch.autograd.Function):
    """Lowest eigenvalues E(V, strain, alpha) with a Hellmann-Feynman backward.

    forward(V [Np], strain [6, Np], alpha [n_gates], grid, levers, solve_kw)
      -> evals [n] (float64, on V's device)
    backward: dL/dV = sum_i g_i |psi_i|^2, dL/dstrain, dL/dalpha = <dL/dV, Phi_g>.
    """

    @staticmethod
    def forward(ctx, V, strain, alpha, grid, levers, B, solve_kw):
        grid.set_fields(V.detach(), None if strain is None else strain.detach(), levers,
                        None if alpha is None else alpha.detach().cpu().numpy(), B=B)
        r = grid.eigensolve(**solve_kw)
        ctx.grid, ctx.levers = grid, levers
        ctx.evals = r.evals
        ctx.save_for_backward(r.evecs)
        ctx.has_strain = strain is not None
        ctx.has_alpha = alpha is not None
        return torch.as_tensor(r.evals, dtype=torch.float64, device=V.device)

    @staticmethod
    def backward(ctx, grad):
        (evecs,) = ctx.saved_tensors
        g = grad.detach().cpu().numpy()
        dV, dE, da = ctx.grid.backward(evecs, ctx.evals, g, ctx.levers if ctx.has_alpha else None,
                                       want_strain=ctx.has_strain)
        dS = dE.reshape(6, -1) if ctx.has_strain else None
        dA = torch.as_tensor(da, dtype=torch.float64) if ctx.has_alpha else None
        return dV, dS, dA, None, None, None, None
