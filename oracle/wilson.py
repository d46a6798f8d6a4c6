"""Wilson-clover Dirac operator D on the fine level.

The paper works with Wilson's discretisation of the Dirac equation (Sec. 1)
and defers its explicit form to the two-level paper.  The form used here is
the standard Wilson-clover operator

  D psi(x) = (m0 + 4) psi(x)
             - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                           + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) ]
             - (c_sw / 32) sum_{mu, nu} (gamma_mu gamma_nu) (x) (Q_mu_nu(x) - Q_nu_mu(x)) psi(x)

with Q_mu_nu(x) the sum of the four plaquette "leaves" at x in the mu-nu plane
(so Q_nu_mu = Q_mu_nu^dagger).  The clover term is Hermitian and commutes with
Gamma_5, so D satisfies the gamma_5-symmetry D Gamma_5 = Gamma_5 D^dagger of
Sec. 1.  Pins (tests): free-field plane waves, gamma_5-symmetry, gauge
covariance, a hand-computed single-link clover, dense LU solves.

The normalisation of the clover term (the factor c_sw/32 with this Q) is a
reading: the paper prints none.  It is pinned only against the hand-computed
case, i.e. it is "parity unpinned" with respect to the paper itself.

Fields are ``psi[..., T, Z, Y, X, 12]`` with index spin*3 + colour, links
``U[T, Z, Y, X, mu, 3, 3]``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .gamma import GAMMA, I4, spin_colour, gamma5_signs
from .lattice import shift_fwd, shift_bwd, site_axis


def matvec(M: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Per-site matrix times vector: (M f)(x) = M(x) f(x), broadcasting over leading axes of f."""
    return (M @ f[..., None])[..., 0]


def dagger(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


def link(U: np.ndarray, mu: int) -> np.ndarray:
    """U_mu(x) as an array [T, Z, Y, X, 3, 3]."""
    return U[..., mu, :, :]


def link_shift(Umu: np.ndarray, nu: int, s: int) -> np.ndarray:
    """A link field evaluated at x + s*nu_hat (periodic; links carry no boundary sign)."""
    return np.roll(Umu, -s, axis=nu)


def plaquette_leaves(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Q_mu_nu(x): the four oriented plaquettes in the mu-nu plane that start and end at x."""
    Um, Un = link(U, mu), link(U, nu)
    sh = link_shift
    # x -> x+mu -> x+mu+nu -> x+nu -> x
    l1 = Um @ sh(Un, mu, 1) @ dagger(sh(Um, nu, 1)) @ dagger(Un)
    # x -> x+nu -> x+nu-mu -> x-mu -> x
    l2 = Un @ dagger(sh(sh(Um, nu, 1), mu, -1)) @ dagger(sh(Un, mu, -1)) @ sh(Um, mu, -1)
    # x -> x-mu -> x-mu-nu -> x-nu -> x
    l3 = (dagger(sh(Um, mu, -1)) @ dagger(sh(sh(Un, mu, -1), nu, -1))
          @ sh(sh(Um, mu, -1), nu, -1) @ sh(Un, nu, -1))
    # x -> x-nu -> x-nu+mu -> x+mu -> x
    l4 = dagger(sh(Un, nu, -1)) @ sh(Um, nu, -1) @ sh(sh(Un, nu, -1), mu, 1) @ dagger(Um)
    return l1 + l2 + l3 + l4


def clover_term(U: np.ndarray, csw: float) -> np.ndarray:
    """C(x) = -(c_sw/32) sum_{mu != nu} (gamma_mu gamma_nu) (x) (Q_mu_nu - Q_nu_mu), as [..., 12, 12]."""
    dims = U.shape[:4]
    C = np.zeros(tuple(dims) + (12, 12), dtype=np.complex128)
    if csw == 0.0:
        return C
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            Q = plaquette_leaves(U, mu, nu)
            F = Q - dagger(Q)                      # Q_mu_nu - Q_nu_mu
            S = GAMMA[mu] @ GAMMA[nu]
            C += np.einsum("st,...ab->...satb", S, F).reshape(tuple(dims) + (12, 12))
    return -(csw / 32.0) * C


def site_diagonal(U: np.ndarray, m0: float, csw: float) -> np.ndarray:
    """The site-local part (m0 + 4) + C(x) of D, as [..., 12, 12]."""
    dims = U.shape[:4]
    A = clover_term(U, csw)
    A = A + (m0 + 4.0) * np.eye(12)
    return A.reshape(tuple(dims) + (12, 12))


def _colour(Umat: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 3x3 matrix per site to the colour index of psi[..., 12]."""
    p = psi.reshape(psi.shape[:-1] + (4, 3))
    return np.swapaxes(Umat @ np.swapaxes(p, -1, -2), -1, -2).reshape(psi.shape)


def _spin(S: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 4x4 spin matrix to psi[..., 12]."""
    p = psi.reshape(psi.shape[:-1] + (4, 3))
    return (S @ p).reshape(psi.shape)


@dataclass
class WilsonOp:
    """The fine-level operator D_1 = D with its links, site-diagonal part and boundary signs."""
    U: np.ndarray            # [T, Z, Y, X, 4, 3, 3]
    diag: np.ndarray         # [T, Z, Y, X, 12, 12]: (m0 + 4) + C(x)
    bc: tuple                # boundary sign per direction, e.g. (-1, 1, 1, 1)

    @staticmethod
    def build(U, m0: float, csw: float, bc_t: int = -1) -> "WilsonOp":
        return WilsonOp(U=U, diag=site_diagonal(U, m0, csw), bc=(int(bc_t), 1, 1, 1))

    @property
    def dims(self):
        return tuple(self.U.shape[:4])

    @property
    def ndof(self) -> int:
        return 12

    @property
    def gamma5(self) -> np.ndarray:
        return gamma5_signs(12)

    def apply(self, psi: np.ndarray, fwd_mask=None, bwd_mask=None) -> np.ndarray:
        """D psi.  With masks, a hop x -> x +/- mu is kept only where the mask is True at x."""
        out = matvec(self.diag, psi)
        for mu in range(4):
            Um = link(self.U, mu)
            fwd = _spin(I4 - GAMMA[mu], _colour(Um, shift_fwd(psi, mu, self.bc)))
            Ub = link_shift(Um, mu, -1)                     # U_mu(x - mu)
            bwd = _spin(I4 + GAMMA[mu], _colour(dagger(Ub), shift_bwd(psi, mu, self.bc)))
            if fwd_mask is not None:
                fwd = fwd * fwd_mask[mu][..., None]
            if bwd_mask is not None:
                bwd = bwd * bwd_mask[mu][..., None]
            out = out - 0.5 * (fwd + bwd)
        return out

    def stencil(self):
        """The same operator written as a block stencil (diag, fwd[mu], bwd[mu]) of 12x12 blocks.

        fwd[mu](x) multiplies psi(x + mu), bwd[mu](x) multiplies psi(x - mu); the
        boundary sign of the wrapping hop is folded into the block.
        """
        from .stencil import Stencil
        dims = self.dims
        fwd = np.zeros((4,) + dims + (12, 12), dtype=np.complex128)
        bwd = np.zeros_like(fwd)
        for mu in range(4):
            Um = link(self.U, mu)
            Ub = link_shift(Um, mu, -1)
            sf = np.ones(dims)
            sb = np.ones(dims)
            if self.bc[mu] != 1:
                idx = [slice(None)] * 4
                idx[mu] = -1
                sf[tuple(idx)] = self.bc[mu]
                idx[mu] = 0
                sb[tuple(idx)] = self.bc[mu]
            Pm = -0.5 * (I4 - GAMMA[mu])
            Pp = -0.5 * (I4 + GAMMA[mu])
            fwd[mu] = np.einsum("st,...ab->...satb", Pm, Um).reshape(dims + (12, 12)) * sf[..., None, None]
            bwd[mu] = (np.einsum("st,...ab->...satb", Pp, dagger(Ub)).reshape(dims + (12, 12))
                       * sb[..., None, None])
        return Stencil(diag=self.diag.copy(), fwd=fwd, bwd=bwd)


def apply_at_sites(build, U: np.ndarray, psi: np.ndarray, bc, sites) -> np.ndarray:
    """(D psi)(x) at each site x of ``sites`` (a list of (t, z, y, x)), for lattices too large for ``apply``.

    D psi(x) reads psi at x and x +/- mu_hat and links at most one hop from x (the
    four clover leaves included), so it is the value at the centre of the operator
    built on the 3^4 neighbourhood of x, taken periodic, applied to the same
    neighbourhood of psi.  The boundary sign of a hop that wraps the lattice
    multiplies the neighbourhood's psi on the far side instead of the hop.
    ``build(U_patch)`` returns the operator of a patch with periodic boundaries
    (e.g. ``lambda Up: WilsonOp.build(Up, m0, csw, 1)``).  Returns psi[..., nsites, 12].
    """
    dims = U.shape[:4]
    out = []
    for s in sites:
        ix = np.ix_(*[(np.arange(-1, 2) + s[mu]) % dims[mu] for mu in range(4)])
        Up = U[ix]
        pp = psi[(Ellipsis,) + ix + (slice(None),)]
        for mu in range(4):
            if bc[mu] == 1:
                continue
            lo = [slice(None)] * pp.ndim
            if s[mu] == 0:                      # the backward neighbour lies across the boundary
                lo[mu - 5] = 0
                pp[tuple(lo)] *= bc[mu]
            if s[mu] == dims[mu] - 1:           # the forward neighbour lies across the boundary
                lo[mu - 5] = 2
                pp[tuple(lo)] *= bc[mu]
        out.append(build(Up).apply(pp)[..., 1, 1, 1, 1, :])
    return np.stack(out, axis=-2)


def dense_matrix(op, dims=None) -> np.ndarray:
    """The operator as a dense matrix, by applying it to every unit vector (small lattices only).

    Row/column index = lexicographic site * ndof + dof.
    """
    dims = op.dims
    n = op.ndof
    V = int(np.prod(dims))
    N = V * n
    M = np.zeros((N, N), dtype=np.complex128)
    chunk = 256
    for c0 in range(0, N, chunk):
        c1 = min(N, c0 + chunk)
        E = np.zeros((c1 - c0, N), dtype=np.complex128)
        E[np.arange(c1 - c0), np.arange(c0, c1)] = 1.0
        Y = op.apply(E.reshape((c1 - c0,) + tuple(dims) + (n,)))
        M[:, c0:c1] = Y.reshape(c1 - c0, N).T
    return M


def gauge_transform(U: np.ndarray, Omega: np.ndarray) -> np.ndarray:
    """U^Omega_mu(x) = Omega(x) U_mu(x) Omega(x + mu)^dagger."""
    out = np.empty_like(U)
    for mu in range(4):
        out[..., mu, :, :] = Omega @ link(U, mu) @ dagger(link_shift(Omega, mu, 1))
    return out


def colour_rotate(Omega: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(Omega psi)(x) = Omega(x) psi(x) on the colour index."""
    return _colour(Omega, psi)
