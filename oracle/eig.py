"""Plain FP64 eigen-solvers for the lowest states of the assembled H.

TEST INFRASTRUCTURE.  Only tests, the smoke check and the CPU-baseline leg
of the benchmark may use this module; the product path never does.

The method of the paper (Sec. II B: all wanted eigenpairs of the discretised
Schroedinger equation) reaches, up to rounding, the exact lowest eigenpairs
of the Hermitian matrix H.  The oracle is that definition:

* `lowest_dense`: the whole matrix densified and handed to LAPACK's
  Hermitian eigensolver (a library primitive) for the lowest n states;
* `lowest_block_lanczos`: thick-restarted block Lanczos with full
  re-orthogonalisation, for grids too large to densify.  Every cycle does an
  explicit Rayleigh-Ritz on the whole basis (T = Q^H H Q), so the Ritz pairs
  are exact for that subspace, and stops when every wanted residual
  ||H y - theta y|| is below `tol`.  A block (not single-vector) Krylov space
  is used so that exactly degenerate pairs (Kramers doublets at B = 0) are
  both found;
* `lowest_arpack`: ARPACK's implicitly restarted Lanczos (SciPy `eigsh`,
  which='SA', a library routine) for the largest grids at B != 0, where no
  level is exactly degenerate (a single-vector Krylov space holds one vector
  of each exactly degenerate eigenspace, so this path is not used at B = 0).
  Its products H x run through a multithreaded CSR product of PyTorch's CPU
  backend; the returned residuals are recomputed from the assembled H.

Masked points are removed from the matrix before solving and the returned
vectors carry zeros there.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _active(H, mask):
    if mask is None:
        return H, None
    bands = H.shape[0] // mask.size          # 6, or 3 for the spin-independent H0
    keep = np.repeat(mask.reshape(-1).astype(bool), bands)
    idx = np.nonzero(keep)[0]
    return H[idx][:, idx], idx


def _embed(vecs, idx, N):
    if idx is None:
        return vecs
    out = np.zeros((N, vecs.shape[1]), dtype=vecs.dtype)
    out[idx] = vecs
    return out


def lowest_dense(H, n, mask=None):
    """Lowest n eigenpairs by dense LAPACK diagonalisation (ascending)."""
    N = H.shape[0]
    Ha, idx = _active(H, mask)
    A = Ha.toarray()
    w, v = sla.eigh(A, subset_by_index=(0, n - 1), driver="evr")
    return w, _embed(v, idx, N)


def all_eigenvalues_dense(H, mask=None):
    Ha, _ = _active(H, mask)
    return sla.eigvalsh(Ha.toarray())


def _orth_against(W, Q):
    # classical Gram-Schmidt against Q, done twice
    for _ in range(2):
        W = W - Q @ (Q.conj().T @ W)
    return W


def lowest_block_lanczos(H, n, block=4, keep=None, basis_max=None, tol=1e-11,
                         max_cycles=400, seed=12345, mask=None, return_residuals=False):
    """Lowest n eigenpairs by thick-restarted block Lanczos (see module doc)."""
    N = H.shape[0]
    Ha, idx = _active(H, mask)
    Na = Ha.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    keep = keep or (n + 2 * block)
    basis_max = basis_max or max(keep + 12 * block, 3 * keep)
    basis_max = min(basis_max, Na)
    keep = min(keep, basis_max - block) if basis_max > block else basis_max

    def fresh_block(Q, W):
        # orthonormal block orthogonal to Q spanning W; directions lost to
        # rank deficiency are refilled with random ones
        Vn, _ = np.linalg.qr(_orth_against(W, Q))
        if np.any(np.linalg.norm(_orth_against(Vn, Q), axis=0) < 0.5):
            Rr = rng.standard_normal((Na, W.shape[1])) + 1j * rng.standard_normal((Na, W.shape[1]))
            Vn, _ = np.linalg.qr(_orth_against(Rr, Q))
        return Vn

    V0 = rng.standard_normal((Na, block)) + 1j * rng.standard_normal((Na, block))
    Q, _ = np.linalg.qr(V0)
    HQ = np.asarray(Ha @ Q)
    res = None
    for cycle in range(max_cycles):
        # block Krylov expansion: the newest block's product is HQ[:, -block:]
        while Q.shape[1] + block <= basis_max:
            Vn = fresh_block(Q, HQ[:, -block:])
            Q = np.hstack([Q, Vn])
            HQ = np.hstack([HQ, np.asarray(Ha @ Vn)])
        # Rayleigh-Ritz on the whole basis
        T = Q.conj().T @ HQ
        T = 0.5 * (T + T.conj().T)
        theta, S = np.linalg.eigh(T)
        Y = Q @ S[:, :keep]
        HY = HQ @ S[:, :keep]
        R = HY - Y * theta[None, :keep]
        res = np.linalg.norm(R, axis=0)
        if np.all(res[:n] <= tol):
            break
        # thick restart: keep the lowest Ritz vectors and continue the
        # Krylov chain from the residuals of the lowest unconverged ones
        unconv = [i for i in range(keep) if res[i] > tol][:block]
        while len(unconv) < block:
            unconv.append(keep - 1 - len(unconv))
        Q, HQ = Y, HY
        Vn = fresh_block(Q, R[:, unconv])
        Q = np.hstack([Q, Vn])
        HQ = np.hstack([HQ, np.asarray(Ha @ Vn)])
    out = (theta[:n], _embed(Y[:, :n], idx, N))
    if return_residuals:
        return out + (res[:n], cycle + 1)
    return out


def lowest_arpack(H, n, tol=1e-13, ncv=None, seed=12345, mask=None, return_residuals=False):
    """Lowest n eigenpairs (ascending) by ARPACK (see module doc).  `tol` is
    ARPACK's relative Ritz-estimate tolerance; the residuals returned with
    `return_residuals` are ||H v - w v|| recomputed from H."""
    import scipy.sparse.linalg as spla
    import torch
    N = H.shape[0]
    Ha, idx = _active(H, mask)
    Ha = Ha.tocsr()
    Na = Ha.shape[0]
    Ht = torch.sparse_csr_tensor(torch.from_numpy(Ha.indptr.astype(np.int64)),
                                 torch.from_numpy(Ha.indices.astype(np.int64)),
                                 torch.from_numpy(np.ascontiguousarray(Ha.data, dtype=np.complex128)),
                                 size=(Na, Na))
    count = [0]

    def mv(x):
        count[0] += 1
        return (Ht @ torch.from_numpy(np.ascontiguousarray(np.asarray(x).reshape(-1), dtype=np.complex128))).numpy()

    op = spla.LinearOperator((Na, Na), matvec=mv, dtype=np.complex128)
    rng = np.random.Generator(np.random.PCG64(seed))
    v0 = rng.standard_normal(Na) + 1j * rng.standard_normal(Na)
    ncv = ncv or min(Na - 1, max(4 * n, 2 * n + 20))
    w, v = spla.eigsh(op, k=n, which="SA", tol=tol, ncv=ncv, v0=v0, maxiter=100000)
    o = np.argsort(w)
    w, v = w[o], v[:, o]
    if not return_residuals:
        return w, _embed(v, idx, N)
    res = np.linalg.norm(Ha @ v - v * w[None, :], axis=0)
    return w, _embed(v, idx, N), res, count[0]
