"""Pins of the oracle's fine operator against the paper's structure and closed forms."""
import numpy as np
import pytest

import synth
from oracle.gamma import GAMMA, GAMMA5, GAMMA_X, GAMMA_Y, GAMMA_Z, GAMMA_T, spin_colour
from oracle.lattice import vdot, norm, internal_hop_masks
from oracle.wilson import WilsonOp, clover_term, gauge_transform, colour_rotate, dense_matrix, apply_at_sites
from oracle.spectrum import sparse_matrix, leftmost_eigenvalues

DIMS = (4, 4, 4, 4)


def test_gamma_algebra():
    # Hermitian, Clifford algebra, and Gamma_5 = diag(1,1,-1,-1) (Sec. 1: +1 on spins 1,2)
    for mu in range(4):
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T)
        for nu in range(4):
            ac = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4))
    assert np.allclose(GAMMA_X @ GAMMA_Y @ GAMMA_Z @ GAMMA_T, np.diag([1, 1, -1, -1]))
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))


def _plane_wave(dims, n, u):
    """exp(i p.x) u with p_t = (2 n_t + 1) pi / T (antiperiodic) and p_k = 2 pi n_k / L."""
    T = dims[0]
    p = [(2 * n[0] + 1) * np.pi / T] + [2 * np.pi * n[k] / dims[k] for k in (1, 2, 3)]
    c = np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")
    phase = np.exp(1j * sum(p[mu] * c[mu] for mu in range(4)))
    return phase[..., None] * u, np.array(p)


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 1, 0, 3), (3, 2, 1, 1)])
def test_free_field_plane_waves(n):
    m0 = 0.17
    op = WilsonOp.build(synth.unit_gauge(DIMS), m0, 1.3, bc_t=-1)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    psi, p = _plane_wave(DIMS, n, u)
    Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
    expect = psi.reshape(DIMS + (4, 3))
    expect = np.einsum("st,...tc->...sc", Dp, expect).reshape(psi.shape)
    assert norm(op.apply(psi) - expect) <= 1e-13 * norm(expect)


def test_free_field_spectrum_closed_form():
    dims = (4, 2, 2, 2)
    m0 = -0.3
    op = WilsonOp.build(synth.unit_gauge(dims), m0, 0.0, bc_t=-1)
    ev = np.linalg.eigvals(dense_matrix(op))
    expect = []
    for nt in range(dims[0]):
        for nz in range(dims[1]):
            for ny in range(dims[2]):
                for nx in range(dims[3]):
                    p = [(2 * nt + 1) * np.pi / dims[0], 2 * np.pi * nz / dims[1],
                         2 * np.pi * ny / dims[2], 2 * np.pi * nx / dims[3]]
                    re = m0 + sum(1 - np.cos(q) for q in p)
                    im = np.sqrt(sum(np.sin(q) ** 2 for q in p))
                    expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    key = lambda z: (round(z.real, 8), round(z.imag, 8))
    assert np.allclose(sorted(ev, key=key), sorted(expect, key=key), atol=1e-10)


def test_leftmost_eigenvalues_free_field():
    # closed form: smallest real part at p = (pi/T, 0, 0, 0): m0 + 1 - cos(pi/T) +- i sin(pi/T)
    op = WilsonOp.build(synth.unit_gauge(DIMS), 0.0, 0.0, bc_t=-1)
    w = leftmost_eigenvalues(op, k=6, ncv=60)
    assert np.allclose(w.real.min(), 1 - np.cos(np.pi / 4), atol=1e-9)
    assert np.allclose(np.abs(w.imag[np.argmin(w.real)]), np.sin(np.pi / 4), atol=1e-9)


@pytest.mark.parametrize("csw,bc", [(0.0, -1), (1.0, -1), (1.7, 1)])
def test_gamma5_symmetry(csw, bc):
    U = synth.su3_field(DIMS, 0.4, 11)
    op = WilsonOp.build(U, -0.2, csw, bc)
    f = synth.random_spinors(2, DIMS, 12)
    g5 = op.gamma5
    lhs = vdot(f[0], g5 * op.apply(g5 * f[1]))
    rhs = vdot(op.apply(f[0]), f[1])
    assert abs(lhs - rhs) <= 1e-14 * abs(rhs)


def test_gauge_covariance():
    U = synth.su3_field(DIMS, 0.5, 21)
    Om = synth.su3_matrices(DIMS, 1.0, np.random.default_rng(22))
    psi = synth.random_spinors(1, DIMS, 23)[0]
    op = WilsonOp.build(U, 0.1, 1.0, -1)
    opg = WilsonOp.build(gauge_transform(U, Om), 0.1, 1.0, -1)
    lhs = opg.apply(colour_rotate(Om, psi))
    rhs = colour_rotate(Om, op.apply(psi))
    assert norm(lhs - rhs) <= 1e-13 * norm(rhs)


def test_clover_hermitian_and_chiral():
    C = clover_term(synth.su3_field(DIMS, 0.6, 3), 1.0)
    assert np.abs(C - np.conj(np.swapaxes(C, -1, -2))).max() < 1e-14
    # commutes with Gamma_5 <=> no coupling between spins {0,1} and {2,3}
    assert np.abs(C[..., :6, 6:]).max() == 0.0 and np.abs(C[..., 6:, :6]).max() == 0.0


def test_clover_single_link_hand_computed():
    """Unit links except U_mu(x0) = diag(e^{i phi}, e^{-i phi}, 1).

    Worked by hand: the link enters one leaf of Q_mu_nu at x0 + nu and at
    x0 + mu + nu (as W), and one leaf at x0 - nu and x0 + mu - nu (as W^+);
    at x0 and x0 + mu it enters as W + W^+, which is Hermitian and cancels.
    Hence C(x0 + nu) = -(c_sw/16) gamma_mu gamma_nu (x) (W - W^+)
                     = -(c_sw/8) i sin(phi) gamma_mu gamma_nu (x) diag(1, -1, 0).
    """
    phi, csw, mu = 0.7, 1.3, 1
    x0 = (1, 1, 1, 1)
    U = synth.unit_gauge(DIMS)
    W = np.diag([np.exp(1j * phi), np.exp(-1j * phi), 1.0])
    U[x0 + (mu,)] = W
    C = clover_term(U, csw)

    def site(base, steps):
        c = list(base)
        for d, s in steps:
            c[d] = (c[d] + s) % DIMS[d]
        return tuple(c)

    total = np.zeros((12, 12), dtype=complex)
    for nu in range(4):
        if nu == mu:
            continue
        e = -(csw / 8.0) * 1j * np.sin(phi) * spin_colour(GAMMA[mu] @ GAMMA[nu], np.diag([1.0, -1.0, 0.0]))
        assert np.allclose(C[site(x0, [(nu, 1)])], e, atol=1e-14)
        assert np.allclose(C[site(x0, [(mu, 1), (nu, 1)])], e, atol=1e-14)
        assert np.allclose(C[site(x0, [(nu, -1)])], -e, atol=1e-14)
        assert np.allclose(C[site(x0, [(mu, 1), (nu, -1)])], -e, atol=1e-14)
        total += np.abs(e)
    assert np.abs(C[x0]).max() < 1e-14 and np.abs(C[site(x0, [(mu, 1)])]).max() < 1e-14
    nonzero = np.argwhere(np.abs(C).reshape(-1, 144).max(axis=1) > 1e-14)
    assert len(nonzero) == 12          # 3 planes x 4 sites


def test_stencil_form_matches_direct_apply():
    U = synth.su3_field(DIMS, 0.4, 31)
    op = WilsonOp.build(U, 0.05, 1.0, -1)
    st = op.stencil()
    f = synth.random_spinors(2, DIMS, 32)
    assert norm(st.apply(f) - op.apply(f)) <= 1e-14 * norm(op.apply(f))
    fm, bm = internal_hop_masks(DIMS, (2, 2, 2, 2))
    a = op.apply(f, fwd_mask=fm, bwd_mask=bm)
    b = st.apply(f, fwd_mask=fm, bwd_mask=bm)
    assert norm(a - b) <= 1e-14 * norm(a)


def test_dense_matrix_from_apply_matches_sparse_assembly():
    dims = (2, 2, 4, 2)
    op = WilsonOp.build(synth.su3_field(dims, 0.4, 41), -0.1, 1.0, -1)
    assert np.abs(dense_matrix(op) - sparse_matrix(op).toarray()).max() < 1e-14


@pytest.mark.parametrize("dims,bc", [((4, 4, 4, 4), -1), ((2, 3, 4, 1), -1), ((3, 2, 1, 4), 1)])
def test_apply_at_sites_matches_full_apply(dims, bc):
    """Site-by-site evaluation on 3^4 neighbourhoods equals the whole-lattice operator, including
    extents 1 and 2 (the neighbourhood repeats sites) and the antiperiodic time boundary."""
    U = synth.su3_field(dims, 0.4, 3)
    op = WilsonOp.build(U, -0.3, 1.2, bc)
    f = synth.random_fields(2, dims, 12, 5)
    sites = list(np.ndindex(*dims))
    got = apply_at_sites(lambda Up: WilsonOp.build(Up, -0.3, 1.2, 1), U, f, op.bc, sites)
    ref = op.apply(f).reshape(2, -1, 12)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_apply_at_sites_free_field_plane_wave_large_lattice():
    """On a 16^3x32 unit-link lattice, sampled sites (time boundaries included) give the closed form
    (m0 + sum_mu (1 - cos p_mu)) + i sum_mu gamma_mu sin p_mu of an antiperiodic plane wave."""
    dims = (32, 16, 16, 16)
    m0 = 0.13
    U = synth.unit_gauge(dims)
    p = np.array([5 * np.pi / 32, 2 * np.pi * 3 / 16, 2 * np.pi / 16, 0.0])
    co = np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")
    u = np.random.default_rng(4).standard_normal(12) + 1j * np.random.default_rng(5).standard_normal(12)
    psi = np.exp(1j * sum(p[m] * co[m] for m in range(4)))[..., None] * u
    rng = np.random.default_rng(6)
    sites = [(0, 3, 4, 5), (31, 15, 0, 7)] + [tuple(int(rng.integers(0, d)) for d in dims) for _ in range(10)]
    got = apply_at_sites(lambda Up: WilsonOp.build(Up, m0, 1.0, 1), U, psi, (-1, 1, 1, 1), sites)
    Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
    for k, s in enumerate(sites):
        expect = (Dp @ psi[s].reshape(4, 3)).reshape(12)
        assert np.abs(got[k] - expect).max() <= 1e-13
