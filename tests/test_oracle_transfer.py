"""Pins of aggregation, restriction/prolongation and the Galerkin coarse operator."""
import numpy as np
import pytest

import synth
from oracle.lattice import norm, vdot
from oracle.wilson import WilsonOp, dense_matrix
from oracle.spectrum import sparse_matrix
from oracle.transfer import (build_interpolation, restrict, prolong, galerkin, cgs2,
                             RankDeficient, coarse_dims)

DIMS = (4, 4, 4, 4)
AGG = (2, 2, 2, 2)


def _fine(seed=1, csw=1.0, bc=-1):
    return WilsonOp.build(synth.su3_field(DIMS, 0.4, seed), -0.2, csw, bc)


def _P(N=3, seed=5, dims=DIMS, ndof=12, agg=AGG):
    tv = synth.random_fields(N, dims, ndof, seed)
    return build_interpolation(tv, agg), tv


def dense_P(Pf, agg):
    """P as a dense matrix, column by column from prolongation of coarse unit vectors."""
    N = Pf.shape[0]
    dims = Pf.shape[1:5]
    cd = coarse_dims(dims, agg)
    nc = 2 * N
    Vc = int(np.prod(cd))
    cols = []
    for k in range(Vc * nc):
        e = np.zeros(Vc * nc, dtype=complex)
        e[k] = 1
        cols.append(prolong(Pf, agg, e.reshape(cd + (nc,))).ravel())
    return np.array(cols).T


def test_cgs2_matches_qr_up_to_phases():
    rng = np.random.default_rng(0)
    W = rng.standard_normal((40, 6)) + 1j * rng.standard_normal((40, 6))
    Q = cgs2(W)
    q, r = np.linalg.qr(W)
    d = np.diag(r) / np.abs(np.diag(r))          # QR unique up to the column phases
    assert np.allclose(Q, q * d[None, :], atol=1e-13)


def test_cgs2_rank_deficiency_is_reported():
    rng = np.random.default_rng(1)
    W = rng.standard_normal((20, 3)) + 0j
    W[:, 2] = W[:, 0] - 2 * W[:, 1]
    with pytest.raises(RankDeficient):
        cgs2(W)


def test_interpolation_orthonormal_and_chiral():
    Pf, tv = _P()
    Pd = dense_P(Pf, AGG)
    assert np.allclose(Pd.conj().T @ Pd, np.eye(Pd.shape[1]), atol=1e-13)
    # Gamma_5 P = P Gamma_5^c (spins 1,2 and 3,4 grouped separately, Sec. 1)
    V = int(np.prod(DIMS))
    g5 = np.tile(np.array([1.0] * 6 + [-1.0] * 6), V)
    g5c = np.tile(np.array([1.0] * 3 + [-1.0] * 3), Pd.shape[1] // 6)
    assert np.allclose(g5[:, None] * Pd, Pd * g5c[None, :], atol=1e-14)
    # every test vector lies in the range of P (P P^+ v = v)
    for j in range(tv.shape[0]):
        v = tv[j]
        assert norm(prolong(Pf, AGG, restrict(Pf, AGG, v)) - v) <= 1e-12 * norm(v)


def test_restrict_is_adjoint_of_prolong():
    Pf, _ = _P()
    f = synth.random_spinors(1, DIMS, 7)[0]
    g = synth.random_fields(1, coarse_dims(DIMS, AGG), 6, 8)[0]
    assert abs(vdot(restrict(Pf, AGG, f), g) - vdot(f, prolong(Pf, AGG, g))) < 1e-12 * norm(f) * norm(g)
    Pd = dense_P(Pf, AGG)
    assert np.allclose(restrict(Pf, AGG, f).ravel(), Pd.conj().T @ f.ravel(), atol=1e-13)


@pytest.mark.parametrize("bc", [-1, 1])
def test_galerkin_equals_dense_PtDP(bc):
    # 4^4 -> 2^4: every coarse extent is 2, so A + mu = A - mu and both blocks must be summed
    op = _fine(bc=bc)
    Pf, _ = _P()
    Dc = galerkin(op, Pf, AGG)
    Pd = dense_P(Pf, AGG)
    ref = Pd.conj().T @ dense_matrix(op) @ Pd
    assert np.abs(sparse_matrix(Dc).toarray() - ref).max() < 1e-12


def test_galerkin_non_cubic_aggregates_and_coarse_of_coarse():
    dims = (8, 4, 4, 4)
    op = WilsonOp.build(synth.su3_field(dims, 0.4, 3), -0.1, 1.0, -1)
    agg1 = (2, 2, 2, 2)
    tv = synth.random_fields(3, dims, 12, 4)
    P1 = build_interpolation(tv, agg1)
    D2 = galerkin(op, P1, agg1)                                     # 4 x 2 x 2 x 2
    assert np.allclose(sparse_matrix(D2).toarray(),
                       dense_P(P1, agg1).conj().T @ sparse_matrix(op).toarray() @ dense_P(P1, agg1),
                       atol=1e-12)
    agg2 = (2, 1, 2, 1)
    tv2 = synth.random_fields(4, D2.dims, D2.ndof, 5)
    P2 = build_interpolation(tv2, agg2)
    D3 = galerkin(D2, P2, agg2)                                     # 2 x 2 x 1 x 2
    ref = dense_P(P2, agg2).conj().T @ sparse_matrix(D2).toarray() @ dense_P(P2, agg2)
    assert np.abs(sparse_matrix(D3).toarray() - ref).max() < 1e-12


def test_coarse_gamma5_symmetry_on_every_level():
    op = _fine()
    Pf, _ = _P()
    Dc = galerkin(op, Pf, AGG)
    for D in (op, Dc):
        M = sparse_matrix(D).toarray()
        g5 = np.tile(D.gamma5, M.shape[0] // D.ndof)
        assert np.abs(g5[:, None] * M * g5[None, :] - M.conj().T).max() < 1e-12
    # the block relation B_mu(A + mu) = Gamma_5 F_mu(A)^+ Gamma_5 the CUDA path relies on
    g = Dc.gamma5
    for mu in range(4):
        lhs = np.roll(Dc.bwd[mu], -1, axis=mu)                      # B_mu(A + mu)
        rhs = g[:, None] * np.conj(np.swapaxes(Dc.fwd[mu], -1, -2)) * g[None, :]
        assert np.abs(lhs - rhs).max() < 1e-12


def test_galerkin_free_field_constant_vectors():
    """U = 1, periodic: constant spinors are zero modes of D - m0, so D_c 1_c = m0 1_c."""
    m0 = 0.37
    op = WilsonOp.build(synth.unit_gauge(DIMS), m0, 1.0, bc_t=1)
    tv = np.zeros((6,) + DIMS + (12,), dtype=complex)
    for j in range(6):
        tv[j, ..., j] = 1.0
        tv[j, ..., 6 + j] = 1.0
    Pf = build_interpolation(tv, AGG)
    Dc = galerkin(op, Pf, AGG)
    one = np.ones(coarse_dims(DIMS, AGG) + (12,), dtype=complex)
    assert norm(Dc.apply(one) - m0 * one) < 1e-13 * norm(one)
