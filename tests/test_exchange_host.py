"""Host arithmetic of the g-tensors and of the magnetic two-hole model
(Sec. III B, Eqs. 16-17): the package's vectorised code against the
oracle's element-by-element code on random inputs (no GPU needed)."""
import numpy as np
import pytest

from oracle import exchange as ex_or
from oracle import gtensor as gt_or
from paper_2607_08447_b300 import exchange as ex
from paper_2607_08447_b300 import gtensor as gt


def _rand_g(rng):
    return rng.standard_normal((3, 3)) * 0.7 + np.diag(rng.uniform(-3, 3, 3))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_g_matrix_and_symmetric_tensor_match_oracle(seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3, 4, 4)) + 1j * rng.standard_normal((3, 4, 4))
    M = (A + np.conj(np.swapaxes(A, 1, 2))) * 1e-4
    q, _ = np.linalg.qr(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
    for c in (q[:, :2], q[:, 2:], np.eye(4)[:, :2]):
        g = gt.g_matrix_of(M, c)
        assert np.abs(g - gt_or.g_matrix(M, c)).max() <= 1e-12 * np.abs(g).max()
        assert np.abs(gt.symmetric_g(g) - gt_or.symmetric_g(g)).max() <= 1e-12 * np.abs(g).max()
    assert gt.MU_B == gt_or.MU_B == ex.MU_B


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_eq16_matrix_matches_oracle(seed):
    rng = np.random.default_rng(10 + seed)
    gL, gR = _rand_g(rng), _rand_g(rng)
    n, th = rng.standard_normal(3), rng.uniform(-1, 1)
    Bs = rng.standard_normal((5, 3))
    bbar, db = ex.zeeman_fields(gL, gR, th, n, Bs)
    H = ex.hamiltonian_b(2e-3, 1.1e-5, bbar, db)
    for k, B in enumerate(Bs):
        bo, do = ex_or.zeeman_fields(gL, gR, th, n, B)
        scale = np.abs(bo).max() + np.abs(do).max()
        assert np.abs(bbar[k] - bo).max() <= 1e-14 * scale and np.abs(db[k] - do).max() <= 1e-14 * scale
        assert np.abs(H[k] - ex_or.hamiltonian_b(2e-3, 1.1e-5, bo, do)).max() <= 1e-14 * scale
    w = ex.magnetic_spectrum(2e-3, 1.1e-5, gL, gR, th, n, Bs)
    assert np.abs(w - np.linalg.eigvalsh(H)).max() <= 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_anisotropic_exchange_matches_oracle(seed):
    rng = np.random.default_rng(20 + seed)
    gL, gR = _rand_g(rng), _rand_g(rng)
    n, th, J = rng.standard_normal(3), rng.uniform(-1, 1), 1e-6
    thetas, phis = np.linspace(0, np.pi, 7), np.linspace(0, 2 * np.pi, 9)
    jp, jl, dz = ex.exchange_maps(J, gL, gR, th, n, 0.5, thetas, phis)
    jpo, jlo, dzo = ex_or.exchange_maps(J, gL, gR, th, n, 0.5, thetas, phis)
    assert np.abs(jp - jpo).max() <= 1e-13 * J
    assert np.abs(jl - jlo).max() <= 1e-13 * J
    assert np.abs(dz - dzo).max() <= 1e-13 * np.abs(dzo).max()
    # n_L along +-z (edge cases of the shortest-arc rotation): for -z the
    # rotation is fixed only up to a turn about z, which |J_perp| and J_par
    # do not see
    for B in (np.linalg.solve(gL, [0, 0, 1.0]), np.linalg.solve(gL, [0, 0, -1.0])):
        Jt, a, b, _ = ex.anisotropic_exchange(J, gL, gR, th, n, B)
        Jto, ao, bo, _ = ex_or.anisotropic_exchange(J, gL, gR, th, n, B)
        assert abs(a - ao) <= 1e-13 * J and abs(b - bo) <= 1e-13 * J
        assert abs(Jt[2, 2] - Jto[2, 2]) <= 1e-13 * J


def test_charging_energy_filter_matches_oracle():
    """The CI truncation filter (Fermi-Dirac at E_C): package and oracle
    keep the same orbitals; at low T exactly those with E_i - E_0 <= E_C."""
    from oracle import ci as ci_or
    from paper_2607_08447_b300.ci import kept_orbitals
    rng = np.random.default_rng(5)
    for _ in range(20):
        E = np.sort(rng.uniform(0.0, 5e-3, 8)) - 0.01
        e_c = rng.uniform(0.0, 5e-3)
        for T in (0.1, 1.5):
            assert kept_orbitals(E, e_c, T) == ci_or.truncate_orbitals(E, e_c, T)
        assert kept_orbitals(E, e_c, 0.01) == int(np.count_nonzero(E - E[0] <= e_c))
        assert ci_or.truncate_orbitals(E, e_c, 0.01) == int(np.count_nonzero(E - E[0] <= e_c))
