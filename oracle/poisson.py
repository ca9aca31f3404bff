"""FP64 oracle of the Poisson step and the Schroedinger-Poisson loop
(Sec. II B).  Test infrastructure only: the tests, the bench's CPU leg and
the entry module's smoke check use it; the library never does.

Poisson problem on the Schroedinger grid (N_p points, spacing h in nm):
    gate points (mask != 0):  phi_p = phi_gate(p)                 [V]
    other points:             sum_{n in nb(p)} (phi_p - phi_n) / h^2 = (e / eps) rho_p
where nb(p) are the face neighbours inside the box (a neighbour outside the
box is dropped: zero normal flux, the paper's von Neumann condition away
from the gates), rho is the hole density in nm^-3 and
e / eps = e / (eps0 eps_Si) in V nm.  The matrix is assembled in CSR and
solved by a sparse direct factorisation.

Schroedinger-Poisson loop (the paper's Sec. II B procedure; readings: a fixed
number of holes sets the Fermi level mu through Fermi-Dirac occupations at
temperature T, the hole potential energy is V = V_ext + phi (a positive
charge in the potential phi, in eV for phi in V), and the potential is
updated by linear mixing):
    E_i, psi_i = lowest n eigenpairs of H(V_k)
    mu: sum_i f((E_i - mu) / kT) = n_holes
    rho_p = sum_i f_i sum_b |psi_i(p, b)|^2 / h^3
    phi = Poisson(rho)
    V_{k+1} = (1 - a) V_k + a (V_ext + phi)
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import eig, kp, observables

E_CHARGE = 1.602176634e-19      # C
EPS0_PER_NM = 8.8541878128e-21  # F / nm
EPS_SI = 11.7
KB_EV = 8.617333262e-5           # eV / K


def e_over_eps(eps_r: float = EPS_SI) -> float:
    """e / (eps0 eps_r) in V nm."""
    return E_CHARGE / (EPS0_PER_NM * eps_r)


def assemble(nx, ny, nz, h, gate_mask):
    """CSR matrix of the Poisson operator (N_p x N_p) and the per-point
    gate flag; gate rows are the identity."""
    Np = nx * ny * nz
    gate = np.asarray(gate_mask, dtype=bool).reshape(Np)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    p = ix + nx * (iy + ny * iz)
    rows, cols, vals = [], [], []
    diag = np.zeros(Np)
    for d, (dx, dy, dz) in enumerate(((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))):
        jx, jy, jz = ix + dx, iy + dy, iz + dz
        ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz) & ~gate
        q = jx + nx * (jy + ny * jz)
        rows.append(p[ok])
        cols.append(q[ok])
        vals.append(np.full(ok.sum(), -1.0 / h ** 2))
        diag[p[ok]] += 1.0 / h ** 2
    rows.append(np.arange(Np))
    cols.append(np.arange(Np))
    vals.append(np.where(gate, 1.0, diag))
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(Np, Np))
    return A, gate


def solve(nx, ny, nz, h, gate_mask, gate_phi, rho, eps_r: float = EPS_SI):
    """phi [N_p] (V) for the hole density rho [N_p] (nm^-3)."""
    A, gate = assemble(nx, ny, nz, h, gate_mask)
    b = e_over_eps(eps_r) * np.asarray(rho, dtype=np.float64).reshape(-1)
    b = np.where(gate, np.asarray(gate_phi, dtype=np.float64).reshape(-1), b)
    return spla.spsolve(A.tocsc(), b)


def fermi_level(E, n_holes, kT):
    """mu with sum_i f((E_i - mu)/kT) = n_holes (bisection; f = Fermi-Dirac)."""
    E = np.asarray(E, dtype=np.float64)

    def count(mu):
        return np.sum(0.5 * (1.0 - np.tanh(0.5 * (E - mu) / kT)))

    lo, hi = E.min() - 50 * kT - 1.0, E.max() + 50 * kT + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if count(mid) < n_holes:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def occupations(E, mu, kT):
    return 0.5 * (1.0 - np.tanh(0.5 * (np.asarray(E) - mu) / kT))


class Anderson:
    """Anderson mixing (Anderson 1965; the "type II" form of Walker and Ni,
    SIAM J. Numer. Anal. 49, 2011) for a fixed point V = G(V).  With the
    residual F_k = G(V_k) - V_k and the differences of the last m iterates
    and residuals, dV_i = V_{i+1} - V_i and dF_i = F_{i+1} - F_i:
        gamma   = argmin || F_k - dF gamma ||_2
        V_{k+1} = V_k + beta F_k - (dV + beta dF) gamma.
    With no history (the first step) this is linear mixing with weight beta.
    The paper says only that the loop is repeated until convergence; this
    scheme is an addition (a reading), not the paper's."""

    def __init__(self, beta, depth):
        self.beta, self.depth = float(beta), int(depth)
        self.V, self.F = [], []

    def step(self, V, GV):
        F = GV - V
        self.V.append(V.copy())
        self.F.append(F.copy())
        m = min(self.depth, len(self.V) - 1)
        out = V + self.beta * F
        if m > 0:
            dV = np.stack([self.V[-m + i] - self.V[-m - 1 + i] for i in range(m)], axis=1)
            dF = np.stack([self.F[-m + i] - self.F[-m - 1 + i] for i in range(m)], axis=1)
            gamma = np.linalg.lstsq(dF, F, rcond=None)[0]
            out = out - (dV + self.beta * dF) @ gamma
        return out


def sp_loop(prob, V_ext, gate_mask, gate_phi, n_states, n_holes, T, mix, iters, bands=6, eps_r=EPS_SI,
            anderson_depth=0):
    """Fixed number of Schroedinger-Poisson iterations from V = V_ext (dense
    eigensolver; small grids).  Linear mixing with weight `mix`, or Anderson
    mixing (damping `mix`) over `anderson_depth` > 0 previous iterates.
    Returns (V, E, mu, history of max |dV|)."""
    nx, ny, nz, h = prob.nx, prob.ny, prob.nz, prob.h
    kT = KB_EV * T
    V = np.asarray(V_ext, dtype=np.float64).reshape(-1).copy()
    hist = []
    acc = Anderson(mix, anderson_depth) if anderson_depth > 0 else None
    for _ in range(iters):
        q = prob.with_(V=V.reshape(nz, ny, nx))
        H = kp.assemble(q) if bands == 6 else kp.assemble_h0(q)
        E, psi = eig.lowest_dense(H, n_states, mask=prob.mask)
        mu = fermi_level(E, n_holes, kT)
        f = occupations(E, mu, kT)
        rho = observables.density(psi, f, bands) / h ** 3
        phi = solve(nx, ny, nz, h, gate_mask, gate_phi, rho, eps_r)
        GV = np.asarray(V_ext).reshape(-1) + phi
        Vn = acc.step(V, GV) if acc is not None else (1.0 - mix) * V + mix * GV
        hist.append(float(np.abs(Vn - V).max()))
        V = Vn
    return V, E, mu, hist


# --------------------------------------------------------------------------
# Predictor-corrector Schroedinger-Poisson loop (Trellakis et al., J. Appl.
# Phys. 81, 7880 (1997)).  The paper says only that the loop is repeated
# until convergence (Sec. II B); at its temperature (1.5 K, Sec. III A)
# mixing V alone oscillates between near-degenerate wells.  The scheme
# replaces the Poisson step by a nonlinear one in which every state keeps
# its wave function while its energy follows the local change of the
# potential:
#     rho[phi](p) = sum_i P_i(p) f((E_i + phi(p) - phi_k(p) - mu) / kT),
#     P_i(p) = sum_b |psi_i(p, b)|^2 / h^3,
#     h^3 sum_p rho[phi](p) = n_holes          (fixes mu for every phi),
#     A phi = (e / eps) rho[phi]               (free points; gates fixed),
# solved by Newton's method.  At a fixed point (phi = phi_k) rho is the
# Fermi-Dirac density of the states of H(V_ext + phi), so the loop ends at
# a solution of the plain Schroedinger-Poisson equations.

def state_densities(evecs, h, bands=6):
    """P[i][p] = sum_b |psi_i(p, b)|^2 / h^3 (nm^-3)."""
    N, n = evecs.shape
    P = (np.abs(evecs) ** 2).reshape(N // bands, bands, n).sum(axis=1)
    return np.ascontiguousarray(P.T) / h ** 3


def local_density(P, E, mu, kT, dphi):
    """rho_p, D_p = -d rho_p / d phi_p at fixed mu, with the local energies
    E_i + dphi_p."""
    x = (np.asarray(E)[:, None] + dphi[None, :] - mu) / kT
    f = 0.5 * (1.0 - np.tanh(0.5 * x))
    rho = np.sum(P * f, axis=0)
    D = np.sum(P * f * (1.0 - f), axis=0) / kT
    return rho, D


def local_fermi_level(P, E, n_holes, kT, dphi, h):
    """mu with h^3 sum_p rho_p(mu) = n_holes (bisection; the count rises
    monotonically with mu)."""
    lo = np.min(E) + dphi.min() - 50 * kT - 1.0
    hi = np.max(E) + dphi.max() + 50 * kT + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        rho, _ = local_density(P, E, mid, kT, dphi)
        if h ** 3 * rho.sum() < n_holes:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def nonlinear_residual(A, gate, gate_phi, coef, phi, P, E, n_holes, kT, phi_k, h):
    """(F, mu, D): F = A phi - coef rho[phi] on free points, phi - phi_gate
    at gates; mu from the hole count; D = -d rho / d phi (local)."""
    dphi = phi - phi_k
    mu = local_fermi_level(P, E, n_holes, kT, dphi, h)
    rho, D = local_density(P, E, mu, kT, dphi)
    F = A @ phi - np.where(gate, gate_phi, coef * rho)
    return F, mu, D


def nonlinear_jacobian_solve(A, gate, coef, D, h, F):
    """delta with J delta = -F, J the derivative of F including the response
    of mu:  J = A + coef diag(D) - coef h^3 D D^T / (h^3 sum D) on the free
    points (identity rows at gates), by Sherman-Morrison over a sparse LU
    of the first two terms."""
    free = ~gate
    Dm = h ** 3 * D.sum()
    Df = np.where(free, D, 0.0)
    M = (A + sp.diags(np.where(free, coef * D, 0.0))).tocsc()
    lu = spla.splu(M)
    y1 = lu.solve(-F)
    if Dm <= 0.0:
        return y1
    u = coef * Df
    v = h ** 3 * Df / Dm
    y2 = lu.solve(u)
    return y1 + y2 * (v @ y1) / (1.0 - v @ y2)


def nonlinear_poisson(nx, ny, nz, h, gate_mask, gate_phi, P, E, n_holes, kT, phi_k, eps_r=EPS_SI,
                      tol=1e-12, max_newton=60):
    """phi solving the predictor's nonlinear Poisson problem from phi = phi_k:
    Newton steps with backtracking (the step is halved until |F| falls).
    Returns (phi, mu, Newton steps)."""
    A, gate = assemble(nx, ny, nz, h, gate_mask)
    coef = e_over_eps(eps_r)
    gphi = np.asarray(gate_phi, dtype=np.float64).reshape(-1)
    phi = np.where(gate, gphi, np.asarray(phi_k, dtype=np.float64).reshape(-1))
    phi_k = np.asarray(phi_k, dtype=np.float64).reshape(-1)
    F, mu, D = nonlinear_residual(A, gate, gphi, coef, phi, P, E, n_holes, kT, phi_k, h)
    for it in range(max_newton):
        delta = nonlinear_jacobian_solve(A, gate, coef, D, h, F)
        if np.abs(delta).max() <= tol:
            return phi + delta, mu, it + 1
        step, nF = 1.0, np.linalg.norm(F)
        for _ in range(30):
            trial = phi + step * delta
            F2, mu2, D2 = nonlinear_residual(A, gate, gphi, coef, trial, P, E, n_holes, kT, phi_k, h)
            if np.linalg.norm(F2) < nF:
                break
            step *= 0.5
        phi, F, mu, D = trial, F2, mu2, D2
    return phi, mu, max_newton


def sp_loop_pc(prob, V_ext, gate_mask, gate_phi, n_states, n_holes, T, iters, bands=6, eps_r=EPS_SI,
               newton_tol=1e-12):
    """Predictor-corrector Schroedinger-Poisson iterations from V = V_ext
    (phi_0 = 0 at free points, the gate values at gates; dense eigensolver,
    sparse direct solves).  Returns (V, E, mu, history of max |dV|)."""
    nx, ny, nz, h = prob.nx, prob.ny, prob.nz, prob.h
    kT = KB_EV * T
    V_ext = np.asarray(V_ext, dtype=np.float64).reshape(-1)
    gate = np.asarray(gate_mask, dtype=bool).reshape(-1)
    phi = np.where(gate, np.asarray(gate_phi, dtype=np.float64).reshape(-1), 0.0)
    V = V_ext + phi
    hist = []
    for _ in range(iters):
        q = prob.with_(V=V.reshape(nz, ny, nx))
        H = kp.assemble(q) if bands == 6 else kp.assemble_h0(q)
        E, psi = eig.lowest_dense(H, n_states, mask=prob.mask)
        P = state_densities(psi, h, bands)
        phi, mu, _ = nonlinear_poisson(nx, ny, nz, h, gate_mask, gate_phi, P, E, n_holes, kT, phi, eps_r,
                                       tol=newton_tol)
        Vn = V_ext + phi
        hist.append(float(np.abs(Vn - V).max()))
        V = Vn
    return V, E, mu, hist
