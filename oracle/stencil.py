"""Nearest-neighbour block stencils: the coarse operators D_l, l >= 2.

A Galerkin operator built from aggregates of lattice blocks couples each
coarse site only to itself and its 8 nearest neighbours (Sec. 1, Sec. 2), so

  (D_l phi)(A) = S(A) phi(A) + sum_mu [ F_mu(A) phi(A + mu) + B_mu(A) phi(A - mu) ]

with dense n x n blocks.  Where an extent is 2, A + mu = A - mu: both blocks
are kept and both terms are added.  Boundary signs are folded into the
blocks, so coarse shifts are plain periodic rolls.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .gamma import gamma5_signs
from .lattice import site_axis, parity


def matvec(M: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Per-site matrix times vector: (M f)(x) = M(x) f(x), broadcasting over leading axes of f."""
    return (M @ f[..., None])[..., 0]


@dataclass
class Stencil:
    diag: np.ndarray   # S(A):     [T, Z, Y, X, n, n]
    fwd: np.ndarray    # F_mu(A):  [4, T, Z, Y, X, n, n], multiplies phi(A + mu)
    bwd: np.ndarray    # B_mu(A):  [4, T, Z, Y, X, n, n], multiplies phi(A - mu)

    @property
    def dims(self):
        return tuple(self.diag.shape[:4])

    @property
    def ndof(self) -> int:
        return int(self.diag.shape[-1])

    @property
    def gamma5(self) -> np.ndarray:
        return gamma5_signs(self.ndof)

    def apply(self, f: np.ndarray, fwd_mask=None, bwd_mask=None) -> np.ndarray:
        """D f.  With masks, a hop A -> A +/- mu is kept only where the mask is True at A."""
        y = matvec(self.diag, f)
        for mu in range(4):
            ax = site_axis(mu)
            tf = matvec(self.fwd[mu], np.roll(f, -1, axis=ax))
            tb = matvec(self.bwd[mu], np.roll(f, 1, axis=ax))
            if fwd_mask is not None:
                tf = tf * fwd_mask[mu][..., None]
            if bwd_mask is not None:
                tb = tb * bwd_mask[mu][..., None]
            y = y + tf + tb
        return y

    def stencil(self) -> "Stencil":
        return self


class EvenOdd:
    """Even-odd (Schur complement) form of a stencil operator, for the coarsest solve.

    With the sites split by parity, D = [[D_ee, D_eo], [D_oe, D_oo]] where D_ee
    and D_oo are the site-diagonal blocks S(A).  The Schur complement is
    Dhat = D_ee - D_eo D_oo^{-1} D_oe on the even sites; a solution of D z = b
    is z_e = Dhat^{-1} (b_e - D_eo D_oo^{-1} b_o), z_o = D_oo^{-1} (b_o - D_oe z_e).
    Vectors on one parity are full-size fields that vanish on the other parity.
    """

    def __init__(self, op: Stencil):
        self.op = op
        par = parity(op.dims)
        self.even = (par == 0)
        self.odd = (par == 1)
        self.diag_inv = np.linalg.inv(op.diag)

    def restrict_even(self, f):
        return f * self.even[..., None]

    def restrict_odd(self, f):
        return f * self.odd[..., None]

    def diag_solve_odd(self, f):
        return self.restrict_odd(matvec(self.diag_inv, f))

    def schur_apply(self, xe):
        """Dhat x_e = [D x_e]_e - [D (D_oo^{-1} [D x_e]_o)]_e."""
        xe = self.restrict_even(xe)
        y = self.op.apply(xe)
        w = self.diag_solve_odd(self.restrict_odd(y))
        return self.restrict_even(y - self.op.apply(w))

    def schur_rhs(self, b):
        """bhat_e = b_e - D_eo D_oo^{-1} b_o."""
        w = self.diag_solve_odd(self.restrict_odd(b))
        return self.restrict_even(b - self.op.apply(w))

    def back_substitute(self, xe, b):
        """z_o = D_oo^{-1} (b_o - D_oe x_e); returns the full z."""
        xe = self.restrict_even(xe)
        r = self.restrict_odd(b - self.op.apply(xe))
        return xe + self.diag_solve_odd(r)
