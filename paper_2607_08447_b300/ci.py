"""Configuration interaction of two holes (Sec. II C, Eqs. 7-15) on the
library's spin-independent H0 orbitals.

Grid-sized work runs in the library: the H0 eigensolve, the orbital-resolved
overlaps and the Coulomb contraction (khp_project_rows on the tensor cores),
the pair densities (khp_pair_densities) and the Poisson solves of the
Coulomb potentials.  The host assembles the K x K two-hole matrix by the
Slater-Condon rules (K = C(2n, 2) <= 120) and diagonalises it.

Spin-orbitals are (i, s) -> 2 i + s, s = 0 up, 1 down.  One-body terms:
H0 energies plus the spin-orbit term (Delta/3)(1 - L.sigma) of the 6x6
operator between the orbital components; two-body terms: spatial Coulomb
integrals sum_p rho_ik(p) V_jl(p) with the spin selection rule of Eq. 14.
"""
from __future__ import annotations

from dataclasses import dataclass
from itertools import combinations

import numpy as np
import torch


def _levi_civita():
    e = np.zeros((3, 3, 3))
    e[0, 1, 2] = e[1, 2, 0] = e[2, 0, 1] = 1.0
    e[0, 2, 1] = e[2, 1, 0] = e[1, 0, 2] = -1.0
    return e


def spin_orbit_6x6(delta):
    """(Delta/3)(1 - L.sigma) on the index 3 s + o, (L_k)_{oq} = -i eps_koq."""
    eps = _levi_civita()
    sig = [np.array([[0, 1], [1, 0]], dtype=complex), np.array([[0, -1j], [1j, 0]]),
           np.array([[1, 0], [0, -1]], dtype=complex)]
    Ldots = np.zeros((6, 6), dtype=complex)
    for k in range(3):
        Lk = -1j * eps[k]
        Ldots += np.kron(sig[k], Lk)          # spin index outer, orbital inner: 3 s + o
    return (delta / 3.0) * (np.eye(6) - Ldots)


def _two_hole_matrix(h1, Jsp, n):
    """Slater-Condon two-hole matrix over determinants a < b of 2n
    spin-orbitals, and the determinant list."""
    dets = list(combinations(range(2 * n), 2))
    index = {d: x for x, d in enumerate(dets)}
    K = len(dets)
    H = np.zeros((K, K), dtype=complex)

    def g(a, b, c, d):          # <ab|cd> with spin selection
        return Jsp[a >> 1, b >> 1, c >> 1, d >> 1] if ((a ^ c) & 1) == 0 and ((b ^ d) & 1) == 0 else 0.0

    for (a, b), x in index.items():
        for (c, d), y in index.items():
            v = 0.0
            if b == d:
                v += h1[a, c]
            if a == c:
                v += h1[b, d]
            if b == c:
                v -= h1[a, d]
            if a == d:
                v -= h1[b, c]
            H[x, y] = v + g(a, b, c, d) - g(a, b, d, c)
    return H, dets


def _total_spin_squared(n, dets):
    """S^2 = S- S+ + Sz (Sz + 1) in the determinant basis."""
    K = len(dets)
    index = {d: x for x, d in enumerate(dets)}
    Sz = np.diag([sum(0.5 - (q & 1) for q in d) for d in dets]).astype(complex)
    Sp = np.zeros((K, K), dtype=complex)
    # S+ = sum_i c+_{i up} c_{i down}: acting on |ab> replaces one down
    # spin-orbital by the up one of the same orbital (with the sign of
    # the reordered pair)
    for (a, b), x in index.items():
        for pos, q in ((0, a), (1, b)):
            if q & 1:
                up = q - 1
                other = b if pos == 0 else a
                if up == other:
                    continue
                pair = (up, other) if pos == 0 else (other, up)
                sign = 1.0
                if pair[0] > pair[1]:
                    pair = (pair[1], pair[0])
                    sign = -1.0
                Sp[index[pair], x] += sign
    Sm = Sp.conj().T
    return Sm @ Sp + Sz @ (Sz + np.eye(K))


@dataclass
class CIResult:
    energies: np.ndarray        # all K two-hole energies (eV), ascending
    spin2: np.ndarray           # <S^2> of each
    exchange: float             # E_triplet - E_singlet (eV)
    orbital_energies: np.ndarray
    coulomb: np.ndarray         # spatial Coulomb integrals J[i, j, k, l] (eV)
    orbitals: object = None     # the H0 orbitals used (device tensor [3 Np][n])


def kept_orbitals(E, e_c, T):
    """How many orbitals pass the charging-energy filter: a Fermi-Dirac
    function at E_C and temperature T of E_i - E_0, kept where >= 1/2."""
    kT = 8.617333262e-5 * T
    x = np.clip((np.asarray(E) - E[0] - e_c) / kT, -700.0, 700.0)
    return int(np.count_nonzero(1.0 / (1.0 + np.exp(x)) >= 0.5))


def ci_exchange(grid, poisson, n_orb, delta_so, solve_kw=None, method=0, e_c=None, T_c=1.0):
    """Two-hole CI on the lowest n_orb orbitals of the spin-independent H0
    handle `grid` (fields set), Coulomb potentials from `poisson` (grounded
    gates).  With e_c (eV), n_orb is the most orbitals solved for and the
    CI keeps those within the charging energy (kept_orbitals, temperature
    T_c in K).  Returns CIResult."""
    if getattr(grid, "bands", 6) != 3:
        raise ValueError("the CI basis comes from the spin-independent H0 (bands = 3)")
    n = int(n_orb)
    if n * n > 64 or 3 * n > 64:
        raise ValueError("n_orb <= 8")
    kw = dict(block_m=max(n + 8, 16), degree=40, tol=1e-11, seed=1)
    kw.update(solve_kw or {})
    r = grid.eigensolve(n, **kw)
    E, psi = r.evals, r.evecs
    if e_c is not None:
        n = kept_orbitals(E, e_c, T_c)
        if n < 1:
            raise ValueError("no orbital within the charging energy")
        E, psi = E[:n], psi[:, :n].contiguous()
    Np = grid.np_
    m_ov = 0 if (method == 0 and 3 * n <= 32) else 1
    m_cb = 0 if (method == 0 and n * n <= 32) else 1
    # orbital-resolved overlaps: psi [3 Np][n] read as [Np][3 n] (column o n + i)
    Gov, _ = grid.project_rows(psi.view(Np, 3 * n), None, method=m_ov)
    O = Gov.reshape(3, n, 3, n).transpose(1, 0, 3, 2)        # [i][o][j][q]
    SO = spin_orbit_6x6(delta_so)
    h1 = np.zeros((2 * n, 2 * n), dtype=complex)
    for s in range(2):
        for t in range(2):
            blk = np.einsum("oq,iojq->ij", SO[3 * s:3 * s + 3, 3 * t:3 * t + 3], O)
            h1[s::2, t::2] = blk
    h1[np.arange(2 * n), np.arange(2 * n)] += np.repeat(E, 2)
    # Coulomb: potentials of every pair density (real and imaginary parts),
    # contracted against the pair densities on the tensor cores
    R = grid.pair_densities(psi)                                # [Np][n n], rho_jl at j n + l
    # the real and imaginary parts of all n^2 pair densities, solved side by
    # side with grounded gates
    rho = torch.cat([R.real.t(), R.imag.t()]).contiguous()     # [2 n^2][Np]
    phi = poisson.solve_many(rho, grounded=True, tol=1e-13)
    V = torch.complex(phi[:n * n].t(), phi[n * n:].t()).contiguous()
    _, S = grid.project_rows(R, V, method=m_cb)
    # S[(k i), (j l)] = sum_p conj(rho_ki) V_jl = sum_p rho_ik V_jl; the
    # potentials were solved for rho (per point), hence the 1 / h^3
    Jsp = S.reshape(n, n, n, n).transpose(1, 2, 0, 3) / grid.h ** 3
    H, dets = _two_hole_matrix(h1, Jsp, n)
    w, v = np.linalg.eigh(H)
    s2 = np.real(np.einsum("ik,ij,jk->k", v.conj(), _total_spin_squared(n, dets), v))
    singlet = w[np.flatnonzero(s2 < 1.0)[0]]
    triplet = w[np.flatnonzero(s2 > 1.0)[0]]
    return CIResult(w, s2, float(triplet - singlet), E, Jsp, psi)


def ci_detuning_sweep(grid, poisson, potentials, n_orb, delta_so, strain=None, solve_kw=None, method=0,
                      e_c=None, T_c=1.0):
    """The CI at every potential of a detuning sweep (Fig. 2(f): the CI
    matrix is rebuilt for each gate configuration).  `potentials` is a
    sequence of V fields for the H0 handle `grid`; each H0 solve after the
    first starts from the previous point's whole Ritz block (orbitals and
    guard columns).  Returns the list of CIResult."""
    out = []
    kw0 = dict(solve_kw or {})
    bm = kw0.get("block_m") or max(int(n_orb) + 8, 16)
    kw0["block_m"] = bm + bm % 2
    blocks = [torch.empty((grid.N, kw0["block_m"]), dtype=torch.complex128, device=grid.device) for _ in range(2)]
    for i, V in enumerate(potentials):
        grid.set_fields(V, strain)
        kw = dict(kw0, block_out=blocks[i % 2])
        if i > 0:
            kw["warm_start"] = blocks[(i - 1) % 2]
        r = ci_exchange(grid, poisson, n_orb, delta_so, solve_kw=kw, method=method, e_c=e_c, T_c=T_c)
        out.append(r)
    return out
