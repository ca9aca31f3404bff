"""g-matrices and left/right g-tensors of a double dot (Sec. III B) through
the CUDA path against the FP64 oracle (`oracle.gtensor`): the position
moments of a block of states, and the basis-independent outputs of the
g-tensor pipeline (energies, g^T g of the bonding, anti-bonding, left and
right doublets, the symmetric g-tensors, det g signs).  The oracle uses a
dense eigensolver and the assembled CSR operator at B = +-d e_j."""
import numpy as np
import pytest
import torch

import inputs
from oracle import gtensor as gt_or

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(7, 5, 4), (33, 9, 7)])
@pytest.mark.parametrize("m", [1, 4, 5, 16])
def test_position_moments_match_oracle(khp, shape, m):
    p = inputs.small_problem(*shape, h=0.5, seed=2, strain=False)
    X = inputs.random_block(6 * p.n_points, m, seed=700 + m)
    g = khp.KPGrid.from_problem(p)
    D = g.position_moments(torch.from_numpy(X).cuda())
    for a in range(3):
        ref = gt_or.position_matrix(p, X, axis=a)
        assert np.abs(D[a] - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.abs(D[a] - D[a].conj().T).max() == 0.0
    # bitwise reproducible
    D2 = g.position_moments(torch.from_numpy(X).cuda())
    assert np.array_equal(D, D2)
    g.close()


def test_position_moments_reject_bad_sizes(khp):
    p = inputs.small_problem(5, 4, 3, h=0.5, seed=2, strain=False)
    g = khp.KPGrid.from_problem(p)
    X = torch.zeros((6 * p.n_points, 17), dtype=torch.complex128, device="cuda")
    with pytest.raises(khp.KHPError):
        g.position_moments(X)
    g.close()


@pytest.mark.parametrize("rot,gauge", [("identity", 0), ("device", 0), ("device", 1)])
def test_g_tensors_match_oracle(khp, rot, gauge):
    from paper_2607_08447_b300.gtensor import g_tensors
    p = inputs.small_problem(12, 6, 6, h=1.0, seed=3, strain=True, rot=rot, B=(0.2, -0.1, 0.3), gauge=gauge)
    ref = gt_or.dqd_g_tensors(p)
    g = khp.KPGrid.from_problem(p)
    r = g_tensors(g, solve_kw=dict(tol=1e-12))
    assert np.array_equal(g.B, p.B)                   # the field is restored
    assert np.abs(r.energies - ref["E"]).max() <= 1e-10
    assert abs(r.delta - ref["delta"]) <= 1e-10
    for key, ours in (("g_bonding", r.g_bonding), ("g_antibonding", r.g_antibonding),
                      ("g_left", r.g_left), ("g_right", r.g_right)):
        G, Gr = ours.T @ ours, ref[key].T @ ref[key]
        assert np.abs(G - Gr).max() <= 1e-7 * max(1.0, np.abs(Gr).max()), key
        assert np.sign(np.linalg.det(ours)) == np.sign(np.linalg.det(ref[key])), key
    assert np.abs(r.gsym_left - ref["gsym_left"]).max() <= 1e-7
    assert np.abs(r.gsym_right - ref["gsym_right"]).max() <= 1e-7
    # the projected position pairs up (Kramers)
    w = np.linalg.eigvalsh(r.position)
    assert abs(w[1] - w[0]) <= 1e-8 and abs(w[3] - w[2]) <= 1e-8
    g.close()


def test_g_tensors_mirror_symmetric_double_dot(khp):
    """Mirror x -> -x of the double dot maps g_L onto g_R: G_R = S G_L S,
    S = diag(1, -1, -1) (B is axial), on the CUDA path alone."""
    from paper_2607_08447_b300.gtensor import g_tensors
    p = inputs.small_problem(20, 8, 8, h=0.8, seed=3, strain=False, noise_mev=0.0, rot="device")
    z, y, x = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    V = p.V + 3e-3 * (y - 3.5) / 8 + 2e-3 * (z - 3.5) / 8 + 1e-3 * (y - 3.5) * (z - 3.5) / 64
    g = khp.KPGrid.from_problem(p.with_(V=V))
    r = g_tensors(g, solve_kw=dict(tol=1e-12))
    S = np.diag([1.0, -1.0, -1.0])
    GL, GR = r.g_left.T @ r.g_left, r.g_right.T @ r.g_right
    assert np.abs(GR - S @ GL @ S).max() <= 1e-7 * np.abs(GL).max()
    assert np.abs(r.gsym_right - S @ r.gsym_left @ S).max() <= 1e-7 * np.abs(GL).max()
    g.close()


@pytest.mark.parametrize("bands,mask", [(3, False), (6, True)])
def test_position_moments_h0_and_masked_grids(khp, bands, mask):
    """The moments kernel on a 3-band H0 handle and on a masked 6-band
    handle (the points a mask excludes still count with whatever X holds
    there) against the plain sum."""
    p = inputs.small_problem(9, 7, 5, h=0.5, seed=4, strain=False, mask=mask)
    nb = bands
    m = 3
    X = inputs.random_block(nb * p.n_points, m, seed=77)
    g = khp.KPGrid.from_problem(p, bands=bands)
    D = g.position_moments(torch.from_numpy(X).cuda())
    z, y, x = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    for a, (c, n_a) in enumerate(((x, p.nx), (y, p.ny), (z, p.nz))):
        r = np.repeat(((c - 0.5 * (n_a - 1)) * p.h).reshape(-1), nb)
        ref = X.conj().T @ (r[:, None] * X)
        assert np.abs(D[a] - ref).max() <= 1e-13 * np.abs(ref).max()
    g.close()
