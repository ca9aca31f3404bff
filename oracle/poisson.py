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
Anderson mixing of the same map is offered as well, and a loop with
relaxed occupations (sp_loop_relaxed; see the section near its definition)
for the paper's 1.5 K.
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
# Schroedinger-Poisson loop with relaxed occupations.  The paper says only
# that the loop is repeated until convergence (Sec. II B); at its
# temperature (1.5 K, Sec. III A) mixing V alone lets the holes jump between
# near-degenerate wells from one iteration to the next.  The reading used
# here lets the occupations respond to the new potential inside each
# iteration, with the states of H(V_k) held fixed:
#   * Q_j: the potential of a unit occupation of state j (Poisson with the
#     gates grounded); phi_g: the potential of the gates alone;
#   * a trial potential phi = phi_g + sum_j f_j Q_j moves level i, to first
#     order, to eps_i = E_i + <psi_i| phi - phi_k |psi_i>
#                     = e0_i + sum_j K_ij f_j,
#     e0_i = E_i + <psi_i| phi_g - phi_k |psi_i>,  K_ij = <psi_i| Q_j |psi_i>;
#   * the occupations solve f_i = F((eps_i - mu) / kT), sum_i f_i = n_holes
#     (F Fermi-Dirac): the minimum of the convex free energy
#     sum_i e0_i f_i + f.K.f / 2 + kT sum_i [f_i ln f_i + (1 - f_i) ln(1 - f_i)]
#     at fixed hole number;
#   * G(V_k) = V_ext + phi_g + sum_j f_j Q_j, mixed into V (linear or
#     Anderson, as in sp_loop).
# At a fixed point phi = phi_k, so eps = E and f are the Fermi-Dirac
# occupations of H(V): the fixed point is one of the plain loop's.

def state_densities(evecs, bands=6):
    """dens[i][p] = sum_b |psi_i(p, b)|^2 (discrete norm: sum_p dens_i = 1)."""
    N, n = evecs.shape
    P = (np.abs(evecs) ** 2).reshape(N // bands, bands, n).sum(axis=1)
    return np.ascontiguousarray(P.T)


def relaxed_occupations(e0, K, n_holes, kT):
    """(f, mu, eps) of the occupation problem above, by Newton's method on
    the effective levels eps = e0 + K f(eps), f(eps) the Fermi-Dirac
    occupations at the Fermi level of eps (bisection); the step is halved
    until the residual falls."""
    e0 = np.asarray(e0, dtype=np.float64)
    n = len(e0)

    def occ(eps):
        mu = fermi_level(eps, n_holes, kT)
        return occupations(eps, mu, kT), mu

    eps = e0 + K @ occ(e0)[0]
    for _ in range(200):
        f, mu = occ(eps)
        R = eps - e0 - K @ f
        nr = np.linalg.norm(R)
        if nr <= 1e-15 * max(1e-3, np.abs(eps).max()):
            break
        s = f * (1.0 - f)
        B = np.diag(s) - (np.outer(s, s) / s.sum() if s.sum() > 0 else 0.0)
        step = np.linalg.solve(np.eye(n) + K @ B / kT, -R)
        a = 1.0
        while True:
            trial = eps + a * step
            f2, _ = occ(trial)
            if np.linalg.norm(trial - e0 - K @ f2) < nr * (1.0 - 1e-4 * a) or a < 1e-12:
                break
            a *= 0.5
        eps = trial
    f, mu = occ(eps)
    return f, mu, eps


def relaxed_step(nx, ny, nz, h, gate_mask, gate_phi, dens, E, n_holes, kT, phi_k, eps_r=EPS_SI):
    """(phi, f, mu): the potential and the relaxed occupations of one
    iteration (see above); dens from state_densities."""
    Np = nx * ny * nz
    phi_g = solve(nx, ny, nz, h, gate_mask, gate_phi, np.zeros(Np), eps_r)
    zero = np.zeros(Np)
    Q = np.stack([solve(nx, ny, nz, h, gate_mask, zero, dens[j] / h ** 3, eps_r) for j in range(len(E))])
    K = dens @ Q.T
    K = 0.5 * (K + K.T)
    e0 = np.asarray(E) + dens @ (phi_g - np.asarray(phi_k).reshape(-1))
    f, mu, _ = relaxed_occupations(e0, K, n_holes, kT)
    return phi_g + f @ Q, f, mu


def sp_loop_relaxed(prob, V_ext, gate_mask, gate_phi, n_states, n_holes, T, mix, iters, bands=6, eps_r=EPS_SI,
                    anderson_depth=0):
    """Schroedinger-Poisson iterations with relaxed occupations from
    V = V_ext (dense eigensolver, sparse direct solves); linear mixing with
    weight `mix`, or Anderson mixing (damping `mix`) over `anderson_depth`
    > 0 previous iterates.  Returns (V, E, mu, f, history of max |dV|)."""
    nx, ny, nz, h = prob.nx, prob.ny, prob.nz, prob.h
    kT = KB_EV * T
    V_ext = np.asarray(V_ext, dtype=np.float64).reshape(-1)
    V = V_ext.copy()
    acc = Anderson(mix, anderson_depth) if anderson_depth > 0 else None
    hist = []
    for _ in range(iters):
        q = prob.with_(V=V.reshape(nz, ny, nx))
        H = kp.assemble(q) if bands == 6 else kp.assemble_h0(q)
        E, psi = eig.lowest_dense(H, n_states, mask=prob.mask)
        phi, f, mu = relaxed_step(nx, ny, nz, h, gate_mask, gate_phi, state_densities(psi, bands), E, n_holes,
                                  kT, V - V_ext, eps_r)
        GV = V_ext + phi
        Vn = acc.step(V, GV) if acc is not None else (1.0 - mix) * V + mix * GV
        hist.append(float(np.abs(Vn - V).max()))
        V = Vn
    return V, E, mu, f, hist
