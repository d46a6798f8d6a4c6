"""Lattice geometry for the oracle.

Fields carry the four site axes (t, z, y, x) followed by one degree-of-freedom
axis: ``f[..., T, Z, Y, X, n]``.  Direction mu = 0, 1, 2, 3 is t, z, y, x, so
the paper's N_t x N_s^3 lattices (Table 2) are ``dims = (N_t, N_s, N_s, N_s)``.

Boundary conditions are a sign per direction (+1 periodic, -1 antiperiodic);
the sign multiplies each hop that crosses the face between x_mu = L_mu - 1 and
x_mu = 0.  It is not stored in the links.
"""
from __future__ import annotations

import numpy as np


def site_axis(mu: int) -> int:
    """Axis of direction mu in a field f[..., T, Z, Y, X, n]."""
    return mu - 5


def shift_fwd(f: np.ndarray, mu: int, bc=(1, 1, 1, 1)) -> np.ndarray:
    """g(x) = sign * f(x + mu_hat); the sign is bc[mu] on the hop that wraps around."""
    ax = site_axis(mu)
    g = np.roll(f, -1, axis=ax)
    if bc[mu] != 1:
        idx = [slice(None)] * g.ndim
        idx[ax] = -1
        g[tuple(idx)] *= bc[mu]
    return g


def shift_bwd(f: np.ndarray, mu: int, bc=(1, 1, 1, 1)) -> np.ndarray:
    """g(x) = sign * f(x - mu_hat); the sign is bc[mu] on the hop that wraps around."""
    ax = site_axis(mu)
    g = np.roll(f, 1, axis=ax)
    if bc[mu] != 1:
        idx = [slice(None)] * g.ndim
        idx[ax] = 0
        g[tuple(idx)] *= bc[mu]
    return g


def coords(dims):
    """Integer coordinate arrays (t, z, y, x), each of shape dims."""
    return np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")


def parity(dims) -> np.ndarray:
    """(t + z + y + x) mod 2; even sites have parity 0."""
    c = coords(dims)
    return (c[0] + c[1] + c[2] + c[3]) % 2


def block_index(dims, bs):
    """Per site, the four block coordinates of the lattice block of size bs containing it."""
    c = coords(dims)
    return [c[mu] // bs[mu] for mu in range(4)]


def block_colour(dims, bs) -> np.ndarray:
    """Red-black colour of the block containing each site: (sum of block coordinates) mod 2."""
    b = block_index(dims, bs)
    return (b[0] + b[1] + b[2] + b[3]) % 2


def internal_hop_masks(dims, bs):
    """Masks (fwd[mu], bwd[mu]) that are True where the hop x -> x +/- mu_hat stays in x's block.

    The neighbour is taken with periodic wrap-around, so a block that spans the
    whole extent of a direction keeps its wrap-around hop.
    """
    c = coords(dims)
    fwd, bwd = [], []
    for mu in range(4):
        L, b = dims[mu], bs[mu]
        own = c[mu] // b
        fwd.append(((c[mu] + 1) % L) // b == own)
        bwd.append(((c[mu] - 1) % L) // b == own)
    return fwd, bwd


def to_blocks(f: np.ndarray, bs) -> np.ndarray:
    """f[..., T, Z, Y, X, n] -> g[..., Tb, Zb, Yb, Xb, bT*bZ*bY*bX, n] (block grid, site in block)."""
    *lead, T, Z, Y, X, n = f.shape
    b0, b1, b2, b3 = bs
    g = f.reshape(*lead, T // b0, b0, Z // b1, b1, Y // b2, b2, X // b3, b3, n)
    k = len(lead)
    perm = list(range(k)) + [k + 0, k + 2, k + 4, k + 6, k + 1, k + 3, k + 5, k + 7, k + 8]
    g = g.transpose(perm)
    return g.reshape(*lead, T // b0, Z // b1, Y // b2, X // b3, b0 * b1 * b2 * b3, n)


def from_blocks(g: np.ndarray, bs) -> np.ndarray:
    """Inverse of ``to_blocks``."""
    *lead, Tb, Zb, Yb, Xb, vol, n = g.shape
    b0, b1, b2, b3 = bs
    h = g.reshape(*lead, Tb, Zb, Yb, Xb, b0, b1, b2, b3, n)
    k = len(lead)
    perm = list(range(k)) + [k + 0, k + 4, k + 1, k + 5, k + 2, k + 6, k + 3, k + 7, k + 8]
    h = h.transpose(perm)
    return h.reshape(*lead, Tb * b0, Zb * b1, Yb * b2, Xb * b3, n)


def red_black_block(dims, bs):
    """SAP block of a lattice whose block count must be even (or 1) in every direction.

    The paper's SAP is red-black on a block grid; where the requested extent
    gives an odd block count, the block is widened to the smallest extent
    >= the requested one that divides the lattice into an even count (or one
    block): 6 sites with 2-site blocks become 3-site blocks.
    """
    out = []
    for L, b in zip(dims, bs):
        c = b
        while c < L and (L % c != 0 or (L // c) % 2 != 0):
            c += 1
        out.append(min(c, L))
    return tuple(out)


def check_blocking(dims, bs, what="block"):
    for mu in range(4):
        if bs[mu] <= 0 or dims[mu] % bs[mu] != 0:
            raise ValueError(f"{what} size {tuple(bs)} does not tile lattice {tuple(dims)}")


def vdot(a: np.ndarray, b: np.ndarray) -> complex:
    """a^dagger b over all entries."""
    return complex(np.vdot(a.ravel(), b.ravel()))


def norm(a: np.ndarray) -> float:
    return float(np.linalg.norm(a.ravel()))
