"""Two-hole configuration interaction (Sec. II C, Eqs. 7-15) through the
CUDA path (H0 orbitals, overlaps and Coulomb contractions on the tensor
cores, pair densities, Poisson potentials) against the oracle pipeline
(dense H0, direct Poisson solves, the same Slater-Condon rules written
separately).  CI energies and the exchange splitting are invariant under
the phases of the orbitals, so they are compared directly."""
import numpy as np
import pytest

import inputs
from oracle import ci as ci_oracle

pytestmark = pytest.mark.gpu


def _end_gates(p):
    g = np.zeros((p.nz, p.ny, p.nx), dtype=np.uint8)
    g[:, :, 0] = 1
    g[:, :, -1] = 1
    return g


@pytest.mark.parametrize("n_orb", [2, 3])
def test_ci_matches_oracle(khp, n_orb):
    from paper_2607_08447_b300.ci import ci_exchange
    from paper_2607_08447_b300.poisson import Poisson
    p = inputs.small_problem(14, 6, 6, h=0.5, seed=5, strain=True)
    gate = _end_gates(p)
    w_or, s2_or, j_or, E_or = ci_oracle.ci_pipeline(p, n_orb, gate)
    g = khp.KPGrid.from_problem(p, bands=3)
    P = Poisson(p.nx, p.ny, p.nz, p.h, gate, np.zeros_like(p.V))
    r = ci_exchange(g, P, n_orb, p.material["delta_so"], solve_kw=dict(tol=1e-12))
    assert np.abs(r.orbital_energies - E_or).max() <= 1e-10
    assert len(r.energies) == n_orb * (2 * n_orb - 1)
    assert np.abs(r.energies - w_or).max() <= 1e-9
    assert np.abs(r.spin2 - s2_or).max() <= 1e-6
    assert abs(r.exchange - j_or) <= 1e-9
    J = r.coulomb
    assert np.abs(J - J.transpose(1, 0, 3, 2)).max() <= 1e-10 * np.abs(J).max()
    P.close()
    g.close()


def test_ci_rejects_six_band_handle(khp):
    from paper_2607_08447_b300.ci import ci_exchange
    from paper_2607_08447_b300.poisson import Poisson
    p = inputs.small_problem(8, 5, 5, h=0.5, seed=1)
    g = khp.KPGrid.from_problem(p)
    P = Poisson(p.nx, p.ny, p.nz, p.h, _end_gates(p), np.zeros_like(p.V))
    with pytest.raises(ValueError):
        ci_exchange(g, P, 2, 0.044)
    P.close()
    g.close()


def test_ci_charging_energy_truncation_matches_oracle(khp):
    """CI space cut by the charging-energy filter (Fermi-Dirac at E_C):
    E_C between the second and third H0 orbital energies keeps two of the
    four solved orbitals on both sides."""
    from paper_2607_08447_b300.ci import ci_exchange
    from paper_2607_08447_b300.poisson import Poisson
    p = inputs.small_problem(14, 6, 6, h=0.5, seed=5, strain=True)
    gate = _end_gates(p)
    E4, _ = ci_oracle.h0_orbitals(p, 4)
    e_c = 0.5 * ((E4[1] - E4[0]) + (E4[2] - E4[0]))
    w_or, s2_or, j_or, E_or = ci_oracle.ci_pipeline(p, 4, gate, e_c=e_c, T_c=0.5)
    assert len(E_or) == 2
    g = khp.KPGrid.from_problem(p, bands=3)
    P = Poisson(p.nx, p.ny, p.nz, p.h, gate, np.zeros_like(p.V))
    r = ci_exchange(g, P, 4, p.material["delta_so"], solve_kw=dict(tol=1e-12), e_c=e_c, T_c=0.5)
    assert len(r.orbital_energies) == 2 and len(r.energies) == 6
    assert np.abs(r.energies - w_or).max() <= 1e-9
    assert abs(r.exchange - j_or) <= 1e-9
    P.close()
    g.close()


def test_ci_detuning_sweep_matches_oracle(khp):
    """CI along a detuning sweep (three potentials: the double well tilted by
    a linear field of -1, 0, +1 meV across the box), warm-started H0 solves,
    against the oracle pipeline run at each point."""
    from paper_2607_08447_b300.ci import ci_detuning_sweep
    from paper_2607_08447_b300.poisson import Poisson
    p = inputs.small_problem(14, 6, 6, h=0.5, seed=5, strain=True)
    gate = _end_gates(p)
    x = (np.arange(p.nx) - 0.5 * (p.nx - 1)) / (p.nx - 1)
    pots = [p.V + eps * x[None, None, :] for eps in (-1e-3, 0.0, 1e-3)]
    g = khp.KPGrid.from_problem(p, bands=3)
    P = Poisson(p.nx, p.ny, p.nz, p.h, gate, np.zeros_like(p.V))
    rs = ci_detuning_sweep(g, P, pots, 2, p.material["delta_so"], strain=p.strain, solve_kw=dict(tol=1e-12))
    assert len(rs) == 3
    for V, r in zip(pots, rs):
        w_or, s2_or, j_or, E_or = ci_oracle.ci_pipeline(p.with_(V=V), 2, gate)
        assert np.abs(r.orbital_energies - E_or).max() <= 1e-10
        assert np.abs(r.energies - w_or).max() <= 1e-9
        assert abs(r.exchange - j_or) <= 1e-9
    P.close()
    g.close()
