"""Spectral helpers used to choose the bare mass m0 of the synthetic workloads.

The paper's systems are near-critical (Table 2 lists m0 close to m_crit).
Criticality means that D(m0) = D(0) + m0 has an eigenvalue close to 0.  Since
D(m0) shifts the spectrum of D(0) by m0, the spectrum's left edge
min Re lambda(D(0)) fixes how close to critical a given field can be made.

* ``leftmost_eigenvalues``: the k eigenvalues of D with smallest real part
  (implicitly restarted Arnoldi, scipy's ARPACK wrapper, matrix-vector
  products only).
* ``edge_mass``: m0 = margin - min Re lambda(D(0)), which places the left
  edge of the spectrum of D(m0) at Re = margin.  This is the reading used for
  the benchmark masses: for smooth fields with an antiperiodic time direction
  D(0) has no real eigenvalue at its left edge, so the smallest singular value
  of D(m0) never crosses zero and a bisection on it has no crossing to find.
* ``sigma_min``: the smallest singular value min |lambda(Gamma_5 D)| (Gamma_5 D
  is Hermitian by gamma_5-symmetry) by shift-invert Lanczos with a sparse LU;
  tiny lattices only.

Pins: on a unit gauge field the leftmost eigenvalues are the closed-form
free-field values m0 + sum_mu (1 - cos p_mu) +- i sqrt(sum_mu sin^2 p_mu).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .wilson import WilsonOp


def sparse_matrix(op) -> sp.csr_matrix:
    """The operator as a sparse matrix (row/column = lexicographic site * ndof + dof)."""
    st = op.stencil()
    dims = st.dims
    n = st.ndof
    V = int(np.prod(dims))
    sites = np.arange(V).reshape(dims)
    rows, cols, vals = [], [], []

    def add(blocks, nbr):
        b = blocks.reshape(V, n, n)
        r = (sites.reshape(V)[:, None, None] * n + np.arange(n)[None, :, None])
        c = (nbr.reshape(V)[:, None, None] * n + np.arange(n)[None, None, :])
        r, c = np.broadcast_to(r, b.shape), np.broadcast_to(c, b.shape)
        keep = b != 0
        rows.append(r[keep])
        cols.append(c[keep])
        vals.append(b[keep])

    add(st.diag, sites)
    for mu in range(4):
        add(st.fwd[mu], np.roll(sites, -1, axis=mu))
        add(st.bwd[mu], np.roll(sites, 1, axis=mu))
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(V * n, V * n))
    return M.tocsr()


def leftmost_eigenvalues(op, k: int = 20, ncv: int = 120, tol: float = 1e-10) -> np.ndarray:
    """The k eigenvalues of the operator with the smallest real part, sorted by real part."""
    D = sparse_matrix(op)
    w = spla.eigs(D, k=k, which="SR", ncv=ncv, tol=tol, return_eigenvectors=False)
    return w[np.argsort(w.real)]


def edge_mass(U, csw: float, bc_t: int = -1, margin: float = 1e-3, k: int = 20) -> tuple:
    """(m0, leftmost eigenvalues of D(0)) with m0 = margin - min Re lambda(D(0))."""
    w = leftmost_eigenvalues(WilsonOp.build(U, 0.0, csw, bc_t), k=k)
    return margin - float(w.real.min()), w


def sigma_min(op, k: int = 2) -> float:
    D = sparse_matrix(op)
    g5 = np.tile(op.gamma5, D.shape[0] // op.ndof)
    Q = sp.diags(g5) @ D
    lu = spla.splu(Q.tocsc())
    Op = spla.LinearOperator(Q.shape, matvec=lu.solve, dtype=np.complex128)
    w = spla.eigsh(Q, k=k, sigma=0.0, which="LM", OPinv=Op, return_eigenvectors=False, tol=1e-8)
    return float(np.min(np.abs(w)))
