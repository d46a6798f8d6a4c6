"""Aggregation-based interpolation P_l, restriction R = P_l^dagger and D_{l+1} = P^dagger D P.

Sec. 1 and Sec. 2.2: P groups spins 1, 2 and spins 3, 4 separately (on a
coarse level: the first and the second half of the degrees of freedom), so
the coarse operator stays gamma_5-symmetric.  Aggregates are lattice blocks
(4^4 on level 1, 2^4 on coarser levels, Table 1).

For every aggregate A and chirality s the N test vectors restricted to (A, s)
form a matrix W_{A,s}; its columns are orthonormalised (classical
Gram-Schmidt applied twice, in column order; the paper names no variant) into
Q_{A,s}.  Coarse degree of freedom (A, s, j) is column j of Q_{A,s}, so a
coarse site carries 2N dof: index s*N + j.

P is stored as N fields ``Pf[j, T, Z, Y, X, n]`` (field j holds column j of
every Q_{A,s}); P^dagger P = I.
"""
from __future__ import annotations

import numpy as np

from .lattice import to_blocks, from_blocks, check_blocking, internal_hop_masks, site_axis
from .stencil import Stencil


class RankDeficient(ValueError):
    pass


def cgs2(W: np.ndarray, rank_tol: float = 1e-12) -> np.ndarray:
    """Orthonormalise the columns of W[..., rows, N] in order, classical Gram-Schmidt twice."""
    Q = np.zeros_like(W)
    N = W.shape[-1]
    for j in range(N):
        w = W[..., :, j].copy()
        n0 = np.linalg.norm(w, axis=-1)
        for _ in range(2):
            h = np.einsum("...ri,...r->...i", np.conj(Q[..., :, :j]), w)
            w = w - np.einsum("...ri,...i->...r", Q[..., :, :j], h)
        nrm = np.linalg.norm(w, axis=-1)
        if np.any(nrm <= rank_tol * n0) or np.any(n0 == 0):
            raise RankDeficient(f"test vector {j} is linearly dependent on an aggregate")
        Q[..., :, j] = w / nrm[..., None]
    return Q


def build_interpolation(tv: np.ndarray, agg) -> np.ndarray:
    """P from test vectors tv[N, T, Z, Y, X, n] on aggregates of size agg."""
    N = tv.shape[0]
    dims = tv.shape[1:5]
    n = tv.shape[-1]
    h = n // 2
    check_blocking(dims, agg, "aggregate")
    blk = to_blocks(tv, agg)                       # [N, Tb, Zb, Yb, Xb, vol, n]
    out = np.zeros_like(blk)
    for s in range(2):
        part = blk[..., s * h:(s + 1) * h]         # [N, Tb.., vol, h]
        W = np.moveaxis(part.reshape(part.shape[:-2] + (-1,)), 0, -1)   # [Tb.., vol*h, N]
        Q = cgs2(W)
        out[..., s * h:(s + 1) * h] = np.moveaxis(Q, -1, 0).reshape(part.shape)
    return from_blocks(out, agg)


def restrict(Pf: np.ndarray, agg, f: np.ndarray) -> np.ndarray:
    """(P^dagger f)(A)[s*N + j] = sum_{x in A} sum_{dof in s} conj(Pf[j, x, dof]) f(x, dof)."""
    N = Pf.shape[0]
    n = Pf.shape[-1]
    h = n // 2
    pb = to_blocks(Pf, agg)                        # [N, Tb.., vol, n]
    fb = to_blocks(f, agg)                         # [..., Tb.., vol, n]
    out = np.zeros(fb.shape[:-2] + (2 * N,), dtype=np.complex128)
    for s in range(2):
        out[..., s * N:(s + 1) * N] = np.einsum(
            "jabcdvk,...abcdvk->...abcdj", np.conj(pb[..., s * h:(s + 1) * h]), fb[..., s * h:(s + 1) * h])
    return out


def prolong(Pf: np.ndarray, agg, fc: np.ndarray) -> np.ndarray:
    """(P phi)(x, dof) = sum_j Pf[j, x, dof] phi(A(x))[s(dof)*N + j]."""
    N = Pf.shape[0]
    n = Pf.shape[-1]
    h = n // 2
    pb = to_blocks(Pf, agg)                        # [N, Tb.., vol, n]
    lead = fc.shape[:-5]
    out = np.zeros(lead + pb.shape[1:], dtype=np.complex128)
    for s in range(2):
        out[..., s * h:(s + 1) * h] = np.einsum(
            "jabcdvk,...abcdj->...abcdvk", pb[..., s * h:(s + 1) * h], fc[..., s * N:(s + 1) * N])
    return from_blocks(out, agg)


def interpolation_site_matrices(Pf: np.ndarray) -> np.ndarray:
    """P_x = the rows of P at site x: [T, Z, Y, X, n, 2N], zero across chiralities."""
    N = Pf.shape[0]
    n = Pf.shape[-1]
    h = n // 2
    dims = Pf.shape[1:5]
    Px = np.zeros(tuple(dims) + (n, 2 * N), dtype=np.complex128)
    pf = np.moveaxis(Pf, 0, -1)                    # [T.., n, N]
    Px[..., :h, :N] = pf[..., :h, :]
    Px[..., h:, N:] = pf[..., h:, :]
    return Px


def galerkin(op, Pf: np.ndarray, agg) -> Stencil:
    """D_{l+1} = P^dagger D_l P as a coarse stencil.

    With D_l in stencil form (diag(x), fwd_mu(x), bwd_mu(x)) and P_x the rows
    of P at x:
      S(A)     = sum_{x in A} P_x^+ diag(x) P_x
                 + sum_mu sum_{x in A, x+mu in A} P_x^+ fwd_mu(x) P_{x+mu}
                 + sum_mu sum_{x in A, x-mu in A} P_x^+ bwd_mu(x) P_{x-mu}
      F_mu(A)  = sum_{x in A, x+mu not in A} P_x^+ fwd_mu(x) P_{x+mu}
      B_mu(A)  = sum_{x in A, x-mu not in A} P_x^+ bwd_mu(x) P_{x-mu}
    B_mu is computed directly, not from the gamma_5 relation.
    """
    st = op.stencil()
    dims = st.dims
    check_blocking(dims, agg, "aggregate")
    Px = interpolation_site_matrices(Pf)
    PxH = np.conj(np.swapaxes(Px, -1, -2))
    fint, bint = internal_hop_masks(dims, agg)

    def blocksum(t):                                # t: [T, Z, Y, X, nc, nc] -> per aggregate
        return to_blocks(t.reshape(tuple(dims) + (-1,)), agg).sum(axis=-2).reshape(
            tuple(d // a for d, a in zip(dims, agg)) + t.shape[-2:])

    S = PxH @ st.diag @ Px
    F = []
    B = []
    for mu in range(4):
        ax = mu                                     # site axis of Px [T, Z, Y, X, n, nc]
        tf = PxH @ st.fwd[mu] @ np.roll(Px, -1, axis=ax)
        tb = PxH @ st.bwd[mu] @ np.roll(Px, 1, axis=ax)
        S = S + tf * fint[mu][..., None, None] + tb * bint[mu][..., None, None]
        F.append(blocksum(tf * (~fint[mu])[..., None, None]))
        B.append(blocksum(tb * (~bint[mu])[..., None, None]))
    return Stencil(diag=blocksum(S), fwd=np.stack(F), bwd=np.stack(B))


def coarse_dims(dims, agg):
    return tuple(d // a for d, a in zip(dims, agg))
