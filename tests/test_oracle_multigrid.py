"""Pins of the multilevel cycle (Alg. 1/2, the E_2g form of Sec. 1) and of the setup (Alg. 3/4)."""
import numpy as np
import pytest

import synth
from oracle.lattice import norm
from oracle.wilson import WilsonOp
from oracle.spectrum import sparse_matrix
from oracle.smoother import SAP
from oracle.transfer import build_interpolation, galerkin, prolong, restrict, coarse_dims
from oracle.multigrid import Params, Hierarchy, build_hierarchy
from oracle.stencil import EvenOdd

DIMS = (4, 4, 4, 4)


def _dense_P(Pf, agg):
    dims = Pf.shape[1:5]
    cd = coarse_dims(dims, agg)
    nc = 2 * Pf.shape[0]
    I = np.eye(int(np.prod(cd)) * nc)
    return np.stack([prolong(Pf, agg, e.reshape(cd + (nc,))).ravel() for e in I], axis=1)


def _two_level(nu, exact_sap):
    op = WilsonOp.build(synth.su3_field(DIMS, 0.4, 1), -0.2, 1.0, -1)
    p = Params(levels=2, agg=((2, 2, 2, 2),), n_tv=(3,), sap_block=((2, 2, 2, 2), None),
               mr_steps=3, nu=nu, mu=0, coarse_tol=1e-15, coarse_restart=100, coarse_cycles=5)
    h = Hierarchy(op, p)
    h.levels[0].tv = synth.random_fields(3, DIMS, 12, 2)
    h.rebuild(0)
    h.levels[0].sap = SAP(op, (2, 2, 2, 2), 3, exact=exact_sap)
    return op, h


def test_two_level_cycle_without_smoothing_is_coarse_correction():
    op, h = _two_level(nu=0, exact_sap=False)
    b = synth.random_spinors(1, DIMS, 3)[0]
    z = h.kcycle(0, b)
    Pd = _dense_P(h.levels[0].P, (2, 2, 2, 2))
    D = sparse_matrix(op).toarray()
    Dc = Pd.conj().T @ D @ Pd
    ref = Pd @ np.linalg.solve(Dc, Pd.conj().T @ b.ravel())
    assert norm(z.ravel() - ref) <= 1e-11 * norm(ref)
    # I - P Dc^{-1} P^+ D is a projector
    C = np.eye(D.shape[0]) - Pd @ np.linalg.solve(Dc, Pd.conj().T @ D)
    assert np.abs(C @ C - C).max() < 1e-10


def test_two_level_error_propagator_E2g():
    """With exact block solves (linear M) and exact coarse solve, e -> e - z(De) equals
    E_2g e = (I - M D)^nu (I - P Dc^{-1} P^+ D) e  (Sec. 1, mu = 0)."""
    nu = 2
    op, h = _two_level(nu=nu, exact_sap=True)
    D = sparse_matrix(op).toarray()
    e = synth.random_spinors(1, DIMS, 4)[0]
    b = op.apply(e)
    z = h.kcycle(0, b)
    Pd = _dense_P(h.levels[0].P, (2, 2, 2, 2))
    Dc = Pd.conj().T @ D @ Pd
    n = D.shape[0]
    M = np.stack([h.levels[0].sap(col.reshape(DIMS + (12,))).ravel() for col in np.eye(n)], axis=1)
    E = np.linalg.matrix_power(np.eye(n) - M @ D, nu) @ (np.eye(n) - Pd @ np.linalg.solve(Dc, Pd.conj().T @ D))
    assert norm((e - z).ravel() - E @ e.ravel()) <= 1e-10 * norm(e)


def test_setup_call_sequence_replays_alg3_alg4():
    """The setup's steps in order, replayed by hand from Alg. 3 and Alg. 4 (L = 3, n_inv = 2)."""
    dims = (8, 4, 4, 4)
    op = WilsonOp.build(synth.su3_field(dims, 0.3, 1), -0.1, 0.0, -1)
    N0, N1 = 2, 3
    p = Params(levels=3, agg=((2, 2, 2, 2), (2, 1, 1, 1)), n_tv=(N0, N1),
               sap_block=((2, 2, 2, 2), (2, 2, 2, 2), None), mr_steps=2, nu=1, n_inv=2)
    c1 = coarse_dims(dims, (2, 2, 2, 2))
    rtv = [synth.random_fields(N0, dims, 12, 2), synth.random_fields(N1 - N0, c1, 2 * N0, 3)]
    h = build_hierarchy(op, p, rtv, trace=True)
    got = [e for e in h.trace.events if e[0] != "kcycle"]
    exp = []
    # Alg. 3 on level 0, then on level 1
    for lvl, N in ((0, N0), (1, N1)):
        for eta in (1, 2, 3):
            for j in range(N):
                exp.append(("smooth", lvl, eta, j))
        exp.append(("build", lvl))
    # Alg. 4: for i = 1..n_inv: iterative_setup_phase(0, i)
    for i in (1, 2):
        exp += [("iterate", 0, i, j) for j in range(N0)]
        exp += [("build", 0), ("build", 1)]
        for q in range(1, i + 1):                      # iterative_setup_phase(1, q)
            exp += [("iterate", 1, q, j) for j in range(N1)]
            exp += [("build", 1)]
    assert got == exp
    # the updated test vectors are normalised and P stays orthonormal
    for lvl in (0, 1):
        for v in h.levels[lvl].tv:
            assert abs(norm(v) - 1.0) < 1e-12


def test_alg4_pass_applies_the_fixed_two_level_cycle_to_every_test_vector():
    """One pass of Alg. 4 on a two-level hierarchy with exact block solves and an exact coarse
    solve: every test vector becomes M v_j / ||M v_j||, M the linear two-level cycle of the P
    built before the pass (z_0 = P Dc^{-1} P^+ b, then nu steps z <- z + S (b - D z)), written out
    densely here; then P is rebuilt from the new vectors.  Rebuilding P inside the pass, taking
    another iterate than the cycle's result, or skipping the normalisation all fail this."""
    nu = 2
    op, h = _two_level(nu=nu, exact_sap=True)
    h.p.n_inv = 1
    D = sparse_matrix(op).toarray()
    n = D.shape[0]
    Pd = _dense_P(h.levels[0].P, (2, 2, 2, 2))
    Dc = Pd.conj().T @ D @ Pd
    S = np.stack([h.levels[0].sap(col.reshape(DIMS + (12,))).ravel() for col in np.eye(n)], axis=1)
    C = Pd @ np.linalg.solve(Dc, Pd.conj().T)
    G = np.eye(n) - S @ D
    M = np.linalg.matrix_power(G, nu) @ C + sum(np.linalg.matrix_power(G, k) @ S for k in range(nu))
    old = [v.copy() for v in h.levels[0].tv]
    h.trace = None
    h.iterative_setup_phase(0, 1)
    for v_old, v_new in zip(old, h.levels[0].tv):
        ref = M @ v_old.ravel()
        ref = ref / norm(ref)
        assert norm(v_new.ravel() - ref) <= 1e-10, norm(v_new.ravel() - ref)
    # P of the new vectors: the coarse operator equals P^+ D P of the dense interpolation
    Pn = _dense_P(h.levels[0].P, (2, 2, 2, 2))
    assert np.abs(Pn.conj().T @ Pn - np.eye(Pn.shape[1])).max() < 1e-12
    cd = coarse_dims(DIMS, (2, 2, 2, 2))
    nc = Pn.shape[1] // int(np.prod(cd))
    Dc_new = np.stack([h.levels[1].op.apply(e.reshape(cd + (nc,))).ravel() for e in np.eye(Pn.shape[1])], axis=1)
    assert np.abs(Dc_new - Pn.conj().T @ D @ Pn).max() <= 1e-12 * np.abs(D).max()


def test_two_level_solve_matches_dense_lu():
    op = WilsonOp.build(synth.su3_field(DIMS, 0.3, 0), -0.35, 0.0, -1)
    p = Params(levels=2, agg=((2, 2, 2, 2),), n_tv=(6,), sap_block=((2, 2, 2, 2), None),
               mr_steps=4, nu=3, n_inv=2, outer_restart=25)
    h = build_hierarchy(op, p, [synth.random_fields(6, DIMS, 12, 5)])
    b = synth.random_spinors(1, DIMS, 1)[0]
    x, info = h.solve(b, tol=1e-10)
    D = sparse_matrix(op).toarray()
    xd = np.linalg.solve(D, b.ravel())
    s = np.linalg.svd(D, compute_uv=False)
    assert info.converged and norm(op.apply(x) - b) <= 1e-10 * norm(b)
    assert norm(x.ravel() - xd) <= (s[0] / s[-1]) * 1e-10 * norm(xd)


def test_three_level_solve_converges():
    dims = (8, 4, 4, 4)
    op = WilsonOp.build(synth.su3_field(dims, 0.4, 2), -0.4, 1.0, -1)
    p = Params(levels=3, agg=((2, 2, 2, 2), (2, 1, 1, 1)), n_tv=(4, 6),
               sap_block=((2, 2, 2, 2), (2, 2, 2, 2), None), mr_steps=3, nu=2, n_inv=1)
    c1 = coarse_dims(dims, (2, 2, 2, 2))
    h = build_hierarchy(op, p, [synth.random_fields(4, dims, 12, 2), synth.random_fields(2, c1, 8, 3)])
    b = synth.random_spinors(1, dims, 4)[0]
    x, info = h.solve(b, tol=1e-10)
    assert info.converged and norm(op.apply(x) - b) <= 1e-10 * norm(b)


def test_red_black_block_reading():
    from oracle.lattice import red_black_block
    # the worked cases of the reading: 6-site extents with 2-site blocks -> 3-site blocks
    assert red_black_block((12, 6, 6, 6), (2, 2, 2, 2)) == (2, 3, 3, 3)
    assert red_black_block((12, 6, 6, 6), (3, 3, 3, 3)) == (3, 3, 3, 3)
    assert red_black_block((8, 8, 8, 8), (2, 2, 2, 2)) == (2, 2, 2, 2)        # unchanged when even
    assert red_black_block((4, 2, 2, 2), (2, 2, 2, 2)) == (2, 2, 2, 2)        # one block: no colouring needed
    assert red_black_block((5, 3, 3, 6), (2, 2, 2, 2)) == (5, 3, 3, 3)        # falls back to one block
    for dims in [(12, 6, 6, 6), (24, 12, 6, 10), (14, 14, 6, 6)]:
        bs = red_black_block(dims, (2, 2, 2, 2))
        for L, b in zip(dims, bs):
            assert L % b == 0 and ((L // b) % 2 == 0 or L // b == 1)


def test_odd_coarsest_uses_plain_gmres_and_solves():
    """A three-level hierarchy whose coarsest lattice has odd extents (plain GMRES there)
    and whose level-1 SAP blocks are widened to 3 sites: the K-cycle preconditioned
    solve still reaches 1e-10 against the fine operator."""
    import synth
    from oracle.wilson import WilsonOp
    from oracle.multigrid import Hierarchy, Params
    dims = (8, 12, 12, 12)
    U = synth.su3_field(dims, 0.3, 1)
    op = WilsonOp.build(U, -0.2, 1.0)
    p = Params(levels=3, agg=((2, 2, 2, 2), (2, 2, 2, 2)), n_tv=(4, 5),
               sap_block=((2, 2, 2, 2), (2, 2, 2, 2), None), mr_steps=2, nu=2, n_inv=0, eta_passes=1,
               outer_restart=10)
    ld = [dims, (4, 6, 6, 6), (2, 3, 3, 3)]
    tv = synth.random_test_vectors(ld, (4, 5), 3)
    h = Hierarchy(op, p).setup(tv)
    assert h.levels[2].eo is None
    assert h.levels[1].sap.block == (2, 3, 3, 3)
    b = synth.random_spinors(1, dims, 2)[0]
    x, info = h.solve(b, tol=1e-10)
    assert info.converged
    assert np.linalg.norm(b - op.apply(x)) <= 1e-10 * np.linalg.norm(b)


# ---------------------------------------------------------------------------
# The recursive K-cycle (Alg. 2 over Alg. 1): an inner FGMRES on level 1 whose
# preconditioner is the K-cycle at level 1, which ends in the coarsest solve.
# Exact SAP block solves and an exact coarsest solve make every cycle linear,
# so each expected value below is written with dense matrices only.

def _three_level_exact(nu, kcycle_len, kcycle_cycles, kcycle_tol):
    """4^4 -> 2^4 (aggregates 2^4, N0 = 3) -> 1x1x2x2 (aggregates 2x2x1x1, N1 = 4)."""
    op = WilsonOp.build(synth.su3_field(DIMS, 0.4, 5), -0.25, 1.0, -1)
    p = Params(levels=3, agg=((2, 2, 2, 2), (2, 2, 1, 1)), n_tv=(3, 4),
               sap_block=((2, 2, 2, 2), (1, 1, 2, 2), None), mr_steps=3, nu=nu, mu=0,
               kcycle_len=kcycle_len, kcycle_cycles=kcycle_cycles, kcycle_tol=kcycle_tol,
               coarse_tol=1e-15, coarse_restart=64, coarse_cycles=4)
    h = Hierarchy(op, p)
    h.levels[0].tv = synth.random_fields(3, DIMS, 12, 6)
    h.rebuild(0)
    h.levels[1].tv = synth.random_fields(4, coarse_dims(DIMS, (2, 2, 2, 2)), 6, 7)
    h.rebuild(1)
    h.levels[0].sap = SAP(op, (2, 2, 2, 2), 3, exact=True)
    h.levels[1].sap = SAP(h.levels[1].op, (1, 1, 2, 2), 3, exact=True)
    return op, h


def _dense_op(f_apply, shape):
    n = int(np.prod(shape))
    return np.stack([f_apply(e.reshape(shape)).ravel() for e in np.eye(n, dtype=np.complex128)], axis=1)


def _dense_levels(op, h):
    """Dense D0, P0, D1 = P0^+ D0 P0, P1, D2 = P1^+ D1 P1, and the exact SAP maps M0 (as a
    callable) and M1 (dense), all from the fine operator, the interpolations and SAP."""
    D0 = sparse_matrix(op).toarray()
    P0 = _dense_P(h.levels[0].P, (2, 2, 2, 2))
    D1 = P0.conj().T @ D0 @ P0
    P1 = _dense_P(h.levels[1].P, (2, 2, 1, 1))
    D2 = P1.conj().T @ D1 @ P1
    shape1 = coarse_dims(DIMS, (2, 2, 2, 2)) + (6,)
    M1 = _dense_op(h.levels[1].sap, shape1)
    return D0, P0, D1, P1, D2, M1


def _smooth(M_apply, D_apply, b, z, nu):
    for _ in range(nu):
        z = z + M_apply(b - D_apply(z))
    return z


def _dense_cycle_level1(D1, P1, D2, M1, nu):
    """The K-cycle at level 1 as a matrix: Z = P1 D2^{-1} P1^+, then nu times Z += M1 (I - D1 Z)."""
    Z = P1 @ np.linalg.solve(D2, P1.conj().T)
    for _ in range(nu):
        Z = Z + M1 @ (np.eye(D1.shape[0]) - D1 @ Z)
    return Z


def test_recursive_kcycle_converged_inner_solve_is_exact_coarse_correction():
    """kcycle_tol = 1e-14 with enough inner iterations: the level-1 FGMRES solves D1 y = P0^+ b
    exactly, so the cycle from level 0 is z = P0 D1^{-1} P0^+ b followed by the nu level-0 SAP
    iterations (Alg. 2; D1 = P0^+ D0 P0 of Sec. 1)."""
    nu = 1
    op, h = _three_level_exact(nu, kcycle_len=40, kcycle_cycles=6, kcycle_tol=1e-14)
    D0, P0, D1, P1, D2, M1 = _dense_levels(op, h)
    b = synth.random_spinors(1, DIMS, 8)[0]
    z = h.kcycle(0, b)
    y = P0 @ np.linalg.solve(D1, P0.conj().T @ b.ravel())
    D0a = lambda v: (D0 @ v.ravel()).reshape(v.shape)
    ref = _smooth(h.levels[0].sap, D0a, b, y.reshape(b.shape), nu)
    assert norm(z - ref) <= 1e-10 * norm(ref)


def test_recursive_kcycle_one_inner_step_is_scaled_level1_cycle():
    """One inner FGMRES step (kcycle_len = kcycle_cycles = 1): with b1 = P0^+ b and K1 the dense
    K-cycle at level 1 (coarsest solve plus nu SAP iterations there), the step's minimal-residual
    coefficient is alpha = <D1 K1 b1, b1> / ||D1 K1 b1||^2 and z = P0 (alpha K1 b1), followed by
    the nu level-0 SAP iterations.  This exercises the recursive preconditioner itself."""
    nu = 2
    op, h = _three_level_exact(nu, kcycle_len=1, kcycle_cycles=1, kcycle_tol=1e-14)
    D0, P0, D1, P1, D2, M1 = _dense_levels(op, h)
    K1 = _dense_cycle_level1(D1, P1, D2, M1, nu)
    b = synth.random_spinors(1, DIMS, 9)[0]
    b1 = P0.conj().T @ b.ravel()
    y = K1 @ b1
    w = D1 @ y
    alpha = np.vdot(w, b1) / np.vdot(w, w).real
    D0a = lambda v: (D0 @ v.ravel()).reshape(v.shape)
    ref = _smooth(h.levels[0].sap, D0a, b, (P0 @ (alpha * y)).reshape(b.shape), nu)
    z = h.kcycle(0, b)
    assert norm(z - ref) <= 1e-10 * norm(ref)
    # the level-1 iterate the setup reads (Alg. 4's z_l) is alpha K1 b1
    assert norm(h.last_iterate[1].ravel() - alpha * y) <= 1e-10 * norm(alpha * y)


def test_recursive_kcycle_two_inner_steps_minimise_over_two_directions():
    """kcycle_len = 2, kcycle_cycles = 1: with a linear K-cycle at level 1 the inner FGMRES is
    right-preconditioned GMRES(2), so y1 = K1 u with u minimising ||b1 - D1 K1 u|| over
    span{b1, D1 K1 b1}.  Swapping the length and the number of cycles (two restarted one-step
    cycles) gives a different vector, which this pin rejects."""
    nu = 1
    op, h = _three_level_exact(nu, kcycle_len=2, kcycle_cycles=1, kcycle_tol=1e-14)
    D0, P0, D1, P1, D2, M1 = _dense_levels(op, h)
    K1 = _dense_cycle_level1(D1, P1, D2, M1, nu)
    A = D1 @ K1
    b = synth.random_spinors(1, DIMS, 10)[0]
    b1 = P0.conj().T @ b.ravel()
    B = np.stack([b1, A @ b1], axis=1)
    c, *_ = np.linalg.lstsq(A @ B, b1, rcond=None)
    y1 = K1 @ (B @ c)
    D0a = lambda v: (D0 @ v.ravel()).reshape(v.shape)
    ref = _smooth(h.levels[0].sap, D0a, b, (P0 @ y1).reshape(b.shape), nu)
    z = h.kcycle(0, b)
    assert norm(z - ref) <= 1e-10 * norm(ref)
    # two restarted one-step cycles differ from the two-step cycle by far more than rounding
    _, h2 = _three_level_exact(nu, kcycle_len=1, kcycle_cycles=2, kcycle_tol=1e-14)
    z2 = h2.kcycle(0, b)
    assert norm(z2 - ref) > 1e-6 * norm(ref)
