"""SAP smoother with minimal-residual block solves (Sec. 1, Table 1).

SAP (the Schwarz alternating procedure) is multiplicative Schwarz over a
red-black colouring of lattice blocks.  D_B is D restricted to block B with
the hops that leave the block dropped.  One application of the smoother to a
residual r is

    e = 0
    for colour c in (red, black):
        rho = r - D e
        for every block B of colour c:  e_B += (block solve of D_B e_B = rho_B)
    return e

and one smoothing iteration of Alg. 1 is z <- z + M(b - D z).  Blocks of one
colour never touch, so the blocks of a colour are solved simultaneously.
Block colour = (sum of block coordinates) mod 2, red = 0 first.  The block
solve is a fixed number of minimal-residual (MR) steps (Table 1: 3 by
default); an exact dense solve is available for the tests.

MR(A, b, k): x = 0, r = b; k times { p = A r; alpha = (p^+ r)/(p^+ p);
x += alpha r; r -= alpha p }.  alpha is taken per block; a block with
p^+ p = 0 keeps alpha = 0 (a zero block right-hand side stays zero).

Block solve on the even-odd Schur complement (schur=True; the paper does not
say which form its block solves use, and the fine operator of the method is
even-odd preconditioned, Sec. 3).  Split the sites of a block by parity,
D_B = [[D_ee, D_eo], [D_oe, D_oo]] with D_ee, D_oo the site-diagonal blocks
(mass + clover; on a coarse level the self blocks).  The block system
D_B e = rho is solved as

    rhohat_e = rho_e - D_eo D_oo^{-1} rho_o
    e_e      = MR(Dhat_B, rhohat_e, k),   Dhat_B = D_ee - D_eo D_oo^{-1} D_oe
    e_o      = D_oo^{-1} (rho_o - D_oe e_e)

with alpha per block over the block's even sites.  With exact=True the Schur
system is solved exactly (dense per block), which equals the exact block solve.
"""
from __future__ import annotations

import numpy as np

from .lattice import (block_colour, internal_hop_masks, to_blocks, from_blocks,
                      check_blocking, parity)


def _block_dot(a, b, bs):
    """Per block, sum over sites in the block and dof of conj(a) * b: [..., Tb, Zb, Yb, Xb]."""
    return np.einsum("...vn,...vn->...", np.conj(to_blocks(a, bs)), to_blocks(b, bs))


def _per_block_scale(alpha, f, bs):
    g = to_blocks(f, bs) * alpha[..., None, None]
    return from_blocks(g, bs)


def _matvec(M, f):
    return (M @ f[..., None])[..., 0]


class SAP:
    def __init__(self, op, block, mr_steps: int, exact: bool = False, schur: bool = False):
        dims = op.dims
        check_blocking(dims, block, "SAP block")
        nb = [d // b for d, b in zip(dims, block)]
        for mu in range(4):
            if nb[mu] != 1 and nb[mu] % 2 != 0:
                raise ValueError(f"red-black SAP needs an even block count per direction, got {nb}")
        self.op = op
        self.block = tuple(block)
        self.k = int(mr_steps)
        self.exact = exact
        self.colour = block_colour(dims, block)
        self.fint, self.bint = internal_hop_masks(dims, block)
        self.schur = schur
        if schur:
            par = parity(dims)
            self.even = (par == 0)[..., None]
            self.odd = (par == 1)[..., None]
            self.diag_inv = np.linalg.inv(op.diag)          # D_oo^{-1}: per-site inverse
        if exact:
            self._block_inverses()

    def apply_block_diag(self, f):
        """D_B f for every block at once (hops leaving a block dropped)."""
        return self.op.apply(f, fwd_mask=self.fint, bwd_mask=self.bint)

    def mr(self, rho):
        """k MR steps on every block in the support of rho (per block alpha)."""
        x = np.zeros_like(rho)
        r = rho.copy()
        for _ in range(self.k):
            p = self.apply_block_diag(r)
            num = _block_dot(p, r, self.block)
            den = _block_dot(p, p, self.block).real
            alpha = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
            x = x + _per_block_scale(alpha, r, self.block)
            r = r - _per_block_scale(alpha, p, self.block)
        return x

    # --- even-odd Schur complement of the block operator --------------------------
    def _dinv_odd(self, f):
        """D_oo^{-1} f_o (zero on even sites)."""
        return _matvec(self.diag_inv, f * self.odd) * self.odd

    def schur_apply(self, xe):
        """Dhat_B x_e = D_ee x_e - D_eo D_oo^{-1} D_oe x_e, every block at once (x_e on even sites)."""
        xe = xe * self.even
        y = self.apply_block_diag(xe)
        return (y - self.apply_block_diag(self._dinv_odd(y))) * self.even

    def schur_rhs(self, rho):
        """rhohat_e = rho_e - D_eo D_oo^{-1} rho_o."""
        return (rho - self.apply_block_diag(self._dinv_odd(rho))) * self.even

    def back_substitute(self, xe, rho):
        """e = e_e + D_oo^{-1} (rho_o - D_oe e_e)."""
        xe = xe * self.even
        return xe + self._dinv_odd(rho - self.apply_block_diag(xe))

    def mr_schur(self, rho):
        """k MR steps on every block's Schur system, then the odd back-substitution."""
        rh = self.schur_rhs(rho)
        x = np.zeros_like(rho)
        r = rh
        for _ in range(self.k):
            p = self.schur_apply(r)
            num = _block_dot(p, r, self.block)
            den = _block_dot(p, p, self.block).real
            alpha = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
            x = x + _per_block_scale(alpha, r, self.block)
            r = r - _per_block_scale(alpha, p, self.block)
        return self.back_substitute(x, rho)

    def _block_inverses(self):
        dims, bs, n = self.op.dims, self.block, self.op.ndof
        vol = int(np.prod(bs))
        nb = tuple(d // b for d, b in zip(dims, bs))
        m = vol * n
        inv = np.zeros(nb + (m, m), dtype=np.complex128)
        # columns of D_B, block by block, from unit vectors placed in every block at once
        for c in range(m):
            e = np.zeros(nb + (vol, n), dtype=np.complex128)
            e[..., c // n, c % n] = 1.0
            col = to_blocks(self.apply_block_diag(from_blocks(e, bs)), bs)
            inv[..., :, c] = col.reshape(nb + (m,))
        self.block_inv = np.linalg.inv(inv)

    def exact_solve(self, rho):
        bs = self.block
        rb = to_blocks(rho, bs)
        shp = rb.shape
        rv = rb.reshape(shp[:-2] + (-1,))
        xv = np.einsum("...ij,...j->...i", self.block_inv, rv)
        return from_blocks(xv.reshape(shp), bs)

    def __call__(self, r):
        """e = M r (one SAP application, both colours)."""
        e = np.zeros_like(r)
        for c in (0, 1):
            mask = (self.colour == c)[..., None]
            if not mask.any():
                continue
            rho = (r - self.op.apply(e)) * mask
            if self.exact:
                e = e + self.exact_solve(rho) * mask
            elif self.schur:
                e = e + self.mr_schur(rho) * mask
            else:
                e = e + self.mr(rho)
        return e

    def smooth(self, b, z, iterations: int):
        """iterations x { z <- z + M (b - D z) }."""
        for _ in range(iterations):
            z = z + self(b - self.op.apply(z))
        return z
