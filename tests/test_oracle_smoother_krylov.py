"""Pins of the MR block solver, SAP, (F)GMRES and the even-odd coarsest solve."""
import numpy as np
import pytest

import synth
from oracle.lattice import norm, block_colour, coords
from oracle.wilson import WilsonOp
from oracle.spectrum import sparse_matrix
from oracle.smoother import SAP
from oracle.krylov import fgmres, gmres, coarsest_solve
from oracle.stencil import EvenOdd
from oracle.transfer import build_interpolation, galerkin

DIMS = (4, 4, 4, 4)
BS = (2, 2, 2, 2)


def _op(seed=1, m0=-0.1, csw=1.0):
    return WilsonOp.build(synth.su3_field(DIMS, 0.4, seed), m0, csw, -1)


def _site_index_sets(dims, bs):
    """For every block (lexicographic over the block grid): its dof indices, and its colour."""
    c = coords(dims)
    lex = ((c[0] * dims[1] + c[1]) * dims[2] + c[2]) * dims[3] + c[3]
    col = block_colour(dims, bs)
    bid = [c[mu] // bs[mu] for mu in range(4)]
    nb = [d // b for d, b in zip(dims, bs)]
    blin = ((bid[0] * nb[1] + bid[1]) * nb[2] + bid[2]) * nb[3] + bid[3]
    out = []
    for b in range(int(np.prod(nb))):
        sites = np.sort(lex[blin == b])
        colour = int(col[blin == b].ravel()[0])
        out.append((sites, colour))
    return out


def _dofs(sites, n):
    return (sites[:, None] * n + np.arange(n)[None, :]).ravel()


def test_mr_residual_monotone_and_alpha_optimal():
    rng = np.random.default_rng(0)
    A = np.eye(30) * 3 + 0.5 * (rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30)))
    r = rng.standard_normal(30) + 0j
    prev = np.linalg.norm(r)
    for _ in range(6):
        p = A @ r
        alpha = np.vdot(p, r) / np.vdot(p, p)
        new = r - alpha * p
        for da in (1e-3, -1e-3, 1e-3j, -1e-3j):
            assert np.linalg.norm(new) <= np.linalg.norm(r - (alpha + da) * p)
        assert np.linalg.norm(new) <= prev + 1e-14
        prev = np.linalg.norm(new)
        r = new


def test_sap_mr_equals_blockwise_brute_force():
    """SAP with k MR steps == an explicit loop over blocks with dense D_B and scalar MR."""
    op = _op()
    sap = SAP(op, BS, mr_steps=3)
    r = synth.random_spinors(1, DIMS, 3)[0]
    D = sparse_matrix(op).toarray()
    n = 12
    e = np.zeros(D.shape[0], dtype=complex)
    rv = r.ravel()
    blocks = _site_index_sets(DIMS, BS)
    for colour in (0, 1):
        rho = rv - D @ e
        for sites, c in blocks:
            if c != colour:
                continue
            idx = _dofs(sites, n)
            DB = D[np.ix_(idx, idx)]
            x = np.zeros(len(idx), dtype=complex)
            rr = rho[idx].copy()
            for _ in range(3):
                p = DB @ rr
                a = np.vdot(p, rr) / np.vdot(p, p)
                x += a * rr
                rr -= a * p
            e[idx] += x
    got = sap(r).ravel()
    assert norm(got - e) <= 1e-13 * norm(e)


def test_sap_exact_block_solves_equal_block_gauss_seidel():
    op = _op(seed=2)
    sap = SAP(op, BS, mr_steps=0, exact=True)
    r = synth.random_spinors(1, DIMS, 4)[0]
    D = sparse_matrix(op).toarray()
    blocks = _site_index_sets(DIMS, BS)
    R = np.concatenate([_dofs(s, 12) for s, c in blocks if c == 0])
    B = np.concatenate([_dofs(s, 12) for s, c in blocks if c == 1])
    rv = r.ravel()
    e = np.zeros_like(rv)
    e[R] = np.linalg.solve(D[np.ix_(R, R)], rv[R])
    e[B] = np.linalg.solve(D[np.ix_(B, B)], rv[B] - D[np.ix_(B, R)] @ e[R])
    assert norm(sap(r).ravel() - e) <= 1e-12 * norm(e)


def test_sap_zero_block_rhs_stays_zero():
    op = _op()
    sap = SAP(op, BS, mr_steps=4)
    r = np.zeros(DIMS + (12,), dtype=complex)
    r[0, 0, 0, 0, 5] = 1.0                  # point source: most blocks see a zero residual
    e = sap(r)
    assert np.all(np.isfinite(e)) and norm(e) > 0


def test_gmres_minimises_residual_over_krylov_space():
    rng = np.random.default_rng(3)
    n = 25
    A = np.eye(n) * 2 + 0.4 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for j in (1, 3, 7):
        x, info = gmres(lambda v: A @ v, b, m=j, tol=1e-30, max_cycles=1)
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(j)], axis=1)
        y = np.linalg.lstsq(A @ K, b, rcond=None)[0]
        best = np.linalg.norm(b - A @ K @ y)
        assert abs(np.linalg.norm(b - A @ x) - best) < 1e-10 * np.linalg.norm(b)
        assert abs(info.true_residual - best / np.linalg.norm(b)) < 1e-10


def test_gmres_exact_in_n_steps_and_fgmres_with_exact_preconditioner():
    rng = np.random.default_rng(4)
    n = 12
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    b = rng.standard_normal(n) + 0j
    x, info = gmres(lambda v: A @ v, b, m=n, tol=1e-14, max_cycles=1)
    assert np.linalg.norm(A @ x - b) < 1e-11 * np.linalg.norm(b)
    Ainv = np.linalg.inv(A)
    x, info = fgmres(lambda v: A @ v, b, M=lambda v: Ainv @ v, m=5, tol=1e-12)
    assert info.iterations == 1 and info.converged


def test_fgmres_with_sap_matches_dense_lu():
    op = _op(seed=5, m0=-0.3)
    sap = SAP(op, BS, mr_steps=4)
    b = synth.random_spinors(1, DIMS, 6)[0]
    x, info = fgmres(op.apply, b, M=sap, m=10, tol=1e-10)
    D = sparse_matrix(op).toarray()
    xd = np.linalg.solve(D, b.ravel())
    s = np.linalg.svd(D, compute_uv=False)
    kappa = s[0] / s[-1]
    assert info.converged and info.true_residual <= 1e-10
    assert norm(op.apply(x) - b) <= 1e-10 * norm(b)
    assert norm(x.ravel() - xd) <= kappa * 1e-10 * norm(xd)


def test_even_odd_schur_solve_equals_dense_lu():
    op = _op(seed=7)
    Pf = build_interpolation(synth.random_fields(3, DIMS, 12, 8), BS)
    Dc = galerkin(op, Pf, BS)                      # 2^4 coarse lattice, 6 dof
    eo = EvenOdd(Dc)
    b = synth.random_fields(1, Dc.dims, 6, 9)[0]
    M = sparse_matrix(Dc).toarray()
    xd = np.linalg.solve(M, b.ravel())
    # Schur complement solved densely, then the odd back-substitution
    ev = np.repeat(eo.even.ravel(), 6)
    S = np.stack([eo.schur_apply(e.reshape(b.shape)).ravel() for e in np.eye(M.shape[0])], axis=1)
    bh = eo.schur_rhs(b).ravel()
    xe = np.zeros_like(bh)
    xe[ev] = np.linalg.solve(S[np.ix_(ev, ev)], bh[ev])
    z = eo.back_substitute(xe.reshape(b.shape), b)
    assert norm(z.ravel() - xd) <= 1e-12 * norm(xd)
    # and the GMRES-based coarsest solve to a tight tolerance
    z2, info = coarsest_solve(eo, b, tol=1e-13, m=50, max_cycles=10)
    assert norm(z2.ravel() - xd) <= 1e-10 * norm(xd)


def _parity_of(sites, dims):
    t = sites // (dims[1] * dims[2] * dims[3])
    z = (sites // (dims[2] * dims[3])) % dims[1]
    y = (sites // dims[3]) % dims[2]
    x = sites % dims[3]
    return (t + z + y + x) % 2


def test_sap_schur_mr_equals_blockwise_dense_schur():
    """The block solve on the even-odd Schur complement (rhohat_e = rho_e - D_eo D_oo^-1 rho_o, k MR
    steps on Dhat = D_ee - D_eo D_oo^-1 D_oe, e_o = D_oo^-1 (rho_o - D_oe e_e)) == the same steps
    written with dense sub-matrices of each block of the dense operator."""
    op = _op(seed=3)
    n = 12
    D = sparse_matrix(op).toarray()
    k = 3
    sap = SAP(op, BS, k, schur=True)
    rho = synth.random_spinors(1, DIMS, 4)[0]
    mask = (block_colour(DIMS, BS) == 0)[..., None]
    got = sap.mr_schur(rho * mask).reshape(-1)
    ref = np.zeros_like(got)
    rv = (rho * mask).reshape(-1)
    for sites, colour in _site_index_sets(DIMS, BS):
        if colour != 0:
            continue
        par = _parity_of(sites, DIMS)
        de, do = _dofs(sites[par == 0], n), _dofs(sites[par == 1], n)
        Dee, Deo, Doe, Doo = D[np.ix_(de, de)], D[np.ix_(de, do)], D[np.ix_(do, de)], D[np.ix_(do, do)]
        S = Dee - Deo @ np.linalg.solve(Doo, Doe)
        rh = rv[de] - Deo @ np.linalg.solve(Doo, rv[do])
        x = np.zeros_like(rh)
        r = rh.copy()
        for _ in range(k):
            p = S @ r
            a = np.vdot(p, r) / np.vdot(p, p).real
            x = x + a * r
            r = r - a * p
        ref[de] = x
        ref[do] = np.linalg.solve(Doo, rv[do] - Doe @ x)
    assert norm(got - ref) <= 1e-12 * norm(ref)


def test_sap_schur_mr_converges_to_the_exact_block_solve():
    """Many MR steps on the Schur system plus the back-substitution reach D_B^-1 rho (the exact block
    solves, pinned against dense block Gauss-Seidel above); a wrong sign in rhohat or in the
    back-substitution would converge elsewhere."""
    op = _op(seed=5, m0=0.3)
    rho = synth.random_spinors(1, DIMS, 6)[0]
    mask = (block_colour(DIMS, BS) == 1)[..., None]
    ex = SAP(op, BS, 3, exact=True).exact_solve(rho * mask) * mask
    got = SAP(op, BS, 120, schur=True).mr_schur(rho * mask)
    assert norm(got - ex) <= 1e-9 * norm(ex)
    # the Schur iteration converges faster per step than MR on the whole block
    e8s = norm(SAP(op, BS, 8, schur=True).mr_schur(rho * mask) - ex)
    e8 = norm(SAP(op, BS, 8).mr(rho * mask) - ex)
    assert e8s < e8


def test_sap_schur_application_uses_schur_block_solves():
    """One SAP application with Schur block solves: red blocks from r, black blocks from r - D e."""
    op = _op(seed=7)
    sap = SAP(op, BS, 2, schur=True)
    r = synth.random_spinors(1, DIMS, 8)[0]
    red = (block_colour(DIMS, BS) == 0)[..., None]
    e = sap.mr_schur(r * red) * red
    e = e + sap.mr_schur((r - op.apply(e)) * ~red) * ~red
    assert norm(sap(r) - e) <= 1e-13 * norm(e)


def test_cgls_solves_dense_system():
    """CGNR (CGLS form) on a small complex system: the solution of the dense solve, and finite
    termination within the dimension on a 24 x 24 matrix."""
    from oracle.krylov import cgls
    rng = np.random.default_rng(11)
    A = np.eye(24) * 2 + 0.4 * (rng.standard_normal((24, 24)) + 1j * rng.standard_normal((24, 24)))
    b = rng.standard_normal(24) + 1j * rng.standard_normal(24)
    x, info = cgls(lambda v: A @ v, lambda v: A.conj().T @ v, b, tol=1e-12, max_iter=200)
    assert info.converged and info.iterations <= 40
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)


def test_cgnr_on_the_wilson_operator_matches_dense_lu():
    from oracle.krylov import cgls
    op = _op(seed=2, m0=0.2)
    g5 = op.gamma5
    b = synth.random_spinors(1, DIMS, 3)[0]
    x, info = cgls(op.apply, lambda v: g5 * op.apply(g5 * v), b, tol=1e-10)
    assert info.converged
    D = sparse_matrix(op).toarray()
    xd = np.linalg.solve(D, b.ravel())
    s = np.linalg.svd(D, compute_uv=False)
    assert np.linalg.norm(x.ravel() - xd) <= (s[0] / s[-1]) * 1e-10 * np.linalg.norm(xd)


def test_cg_lanczos_ritz_values():
    """After n CG steps on an n x n Hermitian positive definite matrix the Lanczos matrix built from
    the CG coefficients has the matrix's eigenvalues; after fewer steps its extreme Ritz values lie
    inside the spectrum and approach its ends."""
    from oracle.krylov import cg_lanczos_coefficients, lanczos_tridiagonal
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30)))
    ev = np.linspace(0.05, 4.0, 30)
    A = (Q * ev) @ Q.conj().T
    v = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    a, bt = cg_lanczos_coefficients(lambda u: A @ u, v, 30)
    rz = np.linalg.eigvalsh(lanczos_tridiagonal(a, bt))
    assert np.allclose(np.sort(rz), ev, rtol=1e-6, atol=1e-8)
    a, bt = cg_lanczos_coefficients(lambda u: A @ u, v, 12)
    rz = np.linalg.eigvalsh(lanczos_tridiagonal(a, bt))
    assert ev[0] - 1e-12 <= rz[0] and rz[-1] <= ev[-1] + 1e-12
