"""Host-side arithmetic of the package (the steps that run on small
matrices on the host) against the oracle's separately written versions,
on random inputs: the Fermi level of the SP loop, the spin-orbit block and
the Slater-Condon two-hole matrix of the CI, and the total-spin operator.
No GPU needed."""
import numpy as np
import pytest

from oracle import ci as ci_or
from oracle import kp
from oracle import poisson as po_or
from paper_2607_08447_b300 import ci as ci_pkg
from paper_2607_08447_b300 import poisson as po_pkg


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fermi_level_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    E = np.sort(rng.uniform(-5e-3, 5e-3, 16))
    for T, nh in ((1.5, 2.0), (20.0, 3.0), (0.3, 1.0)):
        kT = 8.617333262e-5 * T
        mu_p = po_pkg.fermi_level(E, nh, kT)
        mu_o = po_or.fermi_level(E, nh, kT)
        assert abs(mu_p - mu_o) <= 1e-12
        assert abs(np.sum(po_or.occupations(E, mu_p, kT)) - nh) <= 1e-9


def test_spin_orbit_block_matches_oracle():
    for delta in (0.044, 0.3):
        assert np.abs(ci_pkg.spin_orbit_6x6(delta) - kp.spin_orbit_matrix(delta)).max() <= 1e-15


@pytest.mark.parametrize("n", [2, 3, 4])
def test_two_hole_matrix_matches_oracle(n):
    rng = np.random.default_rng(10 + n)
    A = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
    h1 = A + A.conj().T
    J = rng.standard_normal((n, n, n, n)) + 1j * rng.standard_normal((n, n, n, n))
    # the symmetries of Coulomb integrals: particle swap and Hermiticity
    J = J + J.transpose(1, 0, 3, 2)
    J = J + J.transpose(2, 3, 0, 1).conj()
    H_pkg, dets_pkg = ci_pkg._two_hole_matrix(h1, J, n)
    H_or, dets_or = ci_or.ci_matrix(h1, J, n)
    assert list(dets_pkg) == list(dets_or)
    assert np.abs(H_pkg - H_or).max() <= 1e-12 * np.abs(H_or).max()
    S_pkg = ci_pkg._total_spin_squared(n, dets_pkg)
    S_or = ci_or.spin_squared(n)
    assert np.abs(S_pkg - S_or).max() <= 1e-12
