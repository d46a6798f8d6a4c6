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
"""
from __future__ import annotations

import numpy as np

from .lattice import (block_colour, internal_hop_masks, to_blocks, from_blocks,
                      check_blocking)


def _block_dot(a, b, bs):
    """Per block, sum over sites in the block and dof of conj(a) * b: [..., Tb, Zb, Yb, Xb]."""
    return np.einsum("...vn,...vn->...", np.conj(to_blocks(a, bs)), to_blocks(b, bs))


def _per_block_scale(alpha, f, bs):
    g = to_blocks(f, bs) * alpha[..., None, None]
    return from_blocks(g, bs)


class SAP:
    def __init__(self, op, block, mr_steps: int, exact: bool = False):
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
            e = e + (self.exact_solve(rho) * mask if self.exact else self.mr(rho))
        return e

    def smooth(self, b, z, iterations: int):
        """iterations x { z <- z + M (b - D z) }."""
        for _ in range(iterations):
            z = z + self(b - self.op.apply(z))
        return z
