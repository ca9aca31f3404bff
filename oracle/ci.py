"""FP64 oracle of the configuration-interaction (CI) step (Sec. II C,
Eqs. 7-15).  Test infrastructure only.

Single-particle basis: the lowest n spatial orbitals phi_i of the
spin-independent H0 (Eq. 6a; three orbital components X, Y, Z per point)
times spin, spin-orbital a = (i, s) with index 2 i + s (s = 0 up, 1 down).
Two-hole Slater determinants |ab>, a < b: K = C(2n, 2) of them (Eq. 10).

One-body part h = H0 + H_SOI (Eqs. 6, 11-12):
    h[(i,s),(j,t)] = E_i d_ij d_st + sum_{o,q} SO[3s+o, 3t+q] O[i,o,j,q],
    O[i,o,j,q] = sum_p conj(phi_i(p,o)) phi_j(p,q),
SO = (Delta/3)(1 - L.sigma) in the index 3 s + o (the spin-orbit term H_SOI
of the 6x6 operator).
Two-body part (Eqs. 13-15): Coulomb integrals of the spatial orbitals
    J[i,j,k,l] = sum_p rho_ik(p) V_jl(p),
    rho_ik(p) = sum_o conj(phi_i(p,o)) phi_k(p,o),
    V_jl = potential of the density rho_jl / h^3 (Poisson step, grounded gates),
and <ab|cd> = d(s_a,s_c) d(s_b,s_d) J[i_a,i_b,i_c,i_d] (the Coulomb operator
does not act on spin, Eq. 14).
CI matrix (Slater-Condon rules for two particles, Eq. 13):
    H[(ab),(cd)] = h_ac d_bd + h_bd d_ac - h_ad d_bc - h_bc d_ad + <ab|cd> - <ab|dc>.
Exchange (Eq. 1): J_ex = E_triplet - E_singlet, the lowest CI states whose
total-spin expectation <S^2> is near 2 and near 0.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import eig, kp, poisson


def h0_orbitals(prob, n_orb):
    H = kp.assemble_h0(prob)
    return eig.lowest_dense(H, n_orb, mask=prob.mask)


def orbital_overlaps(phi):
    """O[i, o, j, q] = sum_p conj(phi_i(p, o)) phi_j(p, q); phi: [3 Np][n]."""
    N, n = phi.shape
    P = phi.reshape(N // 3, 3, n)
    return np.einsum("poi,pqj->iojq", P.conj(), P)


def one_body(E, O, delta_so):
    n = len(E)
    SO = kp.spin_orbit_matrix(delta_so)
    h = np.zeros((2 * n, 2 * n), dtype=complex)
    for i in range(n):
        for s in range(2):
            for j in range(n):
                for t in range(2):
                    v = E[i] if (i == j and s == t) else 0.0
                    for o in range(3):
                        for q in range(3):
                            v += SO[3 * s + o, 3 * t + q] * O[i, o, j, q]
                    h[2 * i + s, 2 * j + t] = v
    return h


def coulomb_tensor(phi, nx, ny, nz, h, gate_mask, eps_r=poisson.EPS_SI):
    """J[i, j, k, l] = sum_p rho_ik(p) V_jl(p) (eV)."""
    N, n = phi.shape
    P = phi.reshape(N // 3, 3, n)
    rho = np.einsum("poi,pok->pik", P.conj(), P)          # [p][i][k]
    zero = np.zeros(nx * ny * nz)
    V = np.empty_like(rho)
    for j in range(n):
        for l in range(n):
            src = rho[:, j, l] / h ** 3
            V[:, j, l] = (poisson.solve(nx, ny, nz, h, gate_mask, zero, src.real, eps_r)
                          + 1j * poisson.solve(nx, ny, nz, h, gate_mask, zero, src.imag, eps_r))
    return np.einsum("pik,pjl->ijkl", rho, V)


def determinants(n_orb):
    return list(itertools.combinations(range(2 * n_orb), 2))


def _one_body_in_dets(o, dets):
    K = len(dets)
    M = np.zeros((K, K), dtype=complex)
    for x, (a, b) in enumerate(dets):
        for y, (c, d) in enumerate(dets):
            M[x, y] = (o[a, c] * (b == d) + o[b, d] * (a == c) - o[a, d] * (b == c) - o[b, c] * (a == d))
    return M


def ci_matrix(h, J, n_orb):
    dets = determinants(n_orb)
    H = _one_body_in_dets(h, dets)

    def two(a, b, c, d):
        if a % 2 != c % 2 or b % 2 != d % 2:
            return 0.0
        return J[a // 2, b // 2, c // 2, d // 2]

    for x, (a, b) in enumerate(dets):
        for y, (c, d) in enumerate(dets):
            H[x, y] += two(a, b, c, d) - two(a, b, d, c)
    return H, dets


def spin_squared(n_orb):
    """<S^2> operator in the determinant basis: S- S+ + Sz (Sz + 1)."""
    M = 2 * n_orb
    sz = np.diag([0.5 - (a % 2) for a in range(M)]).astype(complex)
    sp = np.zeros((M, M), dtype=complex)
    for i in range(n_orb):
        sp[2 * i, 2 * i + 1] = 1.0          # S+ |i down> = |i up>
    dets = determinants(n_orb)
    Sz = _one_body_in_dets(sz, dets)
    Sp = _one_body_in_dets(sp, dets)
    Sm = _one_body_in_dets(sp.conj().T, dets)
    return Sm @ Sp + Sz @ (Sz + np.eye(len(dets)))


def exchange(Hci, n_orb):
    """(all CI energies, <S^2> per state, J = E_triplet - E_singlet)."""
    w, v = np.linalg.eigh(Hci)
    S2 = spin_squared(n_orb)
    s2 = np.real(np.einsum("ik,ij,jk->k", v.conj(), S2, v))
    singlet = w[np.flatnonzero(s2 < 1.0)[0]]
    triplet = w[np.flatnonzero(s2 > 1.0)[0]]
    return w, s2, triplet - singlet


def truncate_orbitals(E, e_c, T):
    """Number of orbitals kept by the charging-energy filter (Sec. III A: a
    Fermi-Dirac function at E_F = E_C and temperature T applied to the
    orbital energies measured from the lowest): those whose filter value
    1 / (1 + exp((E_i - E_0 - E_C) / kT)) is at least 1/2."""
    kT = poisson.KB_EV * T
    n = 0
    for e in E:
        x = (e - E[0] - e_c) / kT
        w = 0.0 if x > 700 else 1.0 / (1.0 + np.exp(x))
        if w >= 0.5:
            n += 1
    return n


def ci_pipeline(prob, n_orb, gate_mask, eps_r=poisson.EPS_SI, e_c=None, T_c=1.0):
    """H0 orbitals -> one- and two-body integrals -> CI energies and J.
    With e_c, the lowest n_orb orbitals are filtered by truncate_orbitals."""
    E, phi = h0_orbitals(prob, n_orb)
    if e_c is not None:
        k = truncate_orbitals(E, e_c, T_c)
        E, phi = E[:k], phi[:, :k]
        n_orb = k
    O = orbital_overlaps(phi)
    h = one_body(E, O, prob.material["delta_so"])
    J = coulomb_tensor(phi, prob.nx, prob.ny, prob.nz, prob.h, gate_mask, eps_r)
    H, _ = ci_matrix(h, J, n_orb)
    return exchange(H, n_orb) + (E,)
