"""Parity of the CUDA library with the FP64 oracle, element by element on the same seeded inputs.

Tolerances (relative 2-norm error): FP64 operator applications <= 1e-12, FP32
applications <= 2e-6 (against the FP64 oracle on the same FP64 inputs), solves:
final true relative residual <= 1e-10 measured with the oracle's own D.
Iterative building blocks whose stopping decisions depend on rounding
(coarsest GMRES, K-cycle, setup) are compared at 1e-9 in FP64.
"""
import numpy as np
import pytest

import synth
from cases import Case, rel, SMALL2, RAGGED2, THREE, ODD3, FOUR, C1, SAP4, SAP4W, BIG2, BIG3, ODDBIG, golden_mass

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-6


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1307_6101_gb300 as m
    return m


def _pair(spec, precision=0, **kw):
    c = Case(**{**spec, **kw})
    U = c.gauge()
    tv = c.random_tv()
    return c, c.gpu(precision, U, tv), c.oracle(U, tv)


def _fields(n, dims, ndof, seed):
    return np.ascontiguousarray(synth.random_fields(n, dims, ndof, seed))


@pytest.mark.parametrize("spec,csw,bc", [(SMALL2, 0.0, -1), (SMALL2, 1.0, -1), (SMALL2, 1.3, 1), (RAGGED2, 1.0, -1)])
def test_fine_apply(dd, spec, csw, bc):
    c, h, o = _pair(spec, csw=csw, bc_t=bc)
    f = _fields(3, c.dims, 12, 7)
    ref = o.levels[0].op.apply(f)
    for prec, tol in ((0, TOL64), (1, TOL32)):
        out = np.zeros_like(f)
        dd.ddamg_apply(h, 0, prec, f, out, 3)
        assert rel(out, ref) <= tol, (prec, rel(out, ref))
    # gamma_5-symmetry of the GPU operator: x^+ G5 D G5 y = (D x)^+ y
    g5 = np.array([1.0] * 6 + [-1.0] * 6)
    a = np.zeros_like(f)
    dd.ddamg_apply(h, 0, 0, np.ascontiguousarray(g5 * f), a, 3)
    lhs = np.vdot(f[0], g5 * a[1])
    dx = np.zeros_like(f)
    dd.ddamg_apply(h, 0, 0, f, dx, 3)
    assert abs(lhs - np.vdot(dx[0], f[1])) <= 1e-13 * abs(lhs)


def test_fine_apply_free_field_closed_form(dd):
    c = Case(**SMALL2, csw=1.0, m0=0.21)
    h = c.gpu(0, U=synth.unit_gauge(c.dims))
    T = c.dims[0]
    p = np.array([3 * np.pi / T, 2 * np.pi / 4, 0.0, 2 * np.pi * 3 / 4])
    co = np.meshgrid(*[np.arange(d) for d in c.dims], indexing="ij")
    u = np.random.default_rng(1).standard_normal(12) + 0j
    psi = np.exp(1j * sum(p[m] * co[m] for m in range(4)))[..., None] * u
    out = np.zeros((1,) + psi.shape, dtype=complex)
    dd.ddamg_apply(h, 0, 0, np.ascontiguousarray(psi[None]), out, 1)
    from oracle.gamma import GAMMA
    Dp = (0.21 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
    expect = np.einsum("st,...tc->...sc", Dp, psi.reshape(c.dims + (4, 3))).reshape(psi.shape)
    assert rel(out[0], expect) <= TOL64


@pytest.mark.parametrize("spec", [SMALL2, RAGGED2])
def test_fine_sap(dd, spec):
    c, h, o = _pair(spec, mr_steps=4)
    b = _fields(2, c.dims, 12, 8)
    z0 = _fields(2, c.dims, 12, 9)
    for prec, tol, it in ((0, TOL64, 2), (1, TOL32, 1)):
        ref = np.stack([o.levels[0].sap.smooth(b[i], z0[i], it) for i in range(2)])
        z = z0.copy()
        dd.ddamg_smooth(h, 0, prec, b, z, 2, it)
        assert rel(z, ref) <= tol, (prec, rel(z, ref))


@pytest.mark.parametrize("spec", [SAP4, SAP4W])
def test_fine_sap_4x4_blocks(dd, spec):
    """The 4^4-block SAP sweep kernel: FP32 arithmetic on FP32 and on FP16 storage, three right-hand
    sides in one sweep (the block's z is staged once per right-hand side)."""
    from oracle.precision import fine_op_half
    from oracle.smoother import SAP
    c, h, o = _pair(spec, mr_steps=4)
    b = _fields(3, c.dims, 12, 8)
    z0 = _fields(3, c.dims, 12, 9)
    for prec, tol, it in ((0, TOL64, 2), (1, TOL32, 1)):
        ref = np.stack([o.levels[0].sap.smooth(b[i], z0[i], it) for i in range(3)])
        z = z0.copy()
        dd.ddamg_smooth(h, 0, prec, b, z, 3, it)
        assert rel(z, ref) <= tol, (prec, rel(z, ref))
    dd.ddamg_set_option(h, dd.DDAMG_OPT_HALF_STORAGE, 1)
    sap = SAP(fine_op_half(c.gauge(), c.m0, c.csw, c.bc_t), c.sap[0], c.mr_steps)
    ref = np.stack([sap.smooth(b[i], z0[i], 1) for i in range(3)])
    z = z0.copy()
    dd.ddamg_smooth(h, 0, 1, b, z, 3, 1)
    assert rel(z, ref) <= TOL32, rel(z, ref)


@pytest.mark.parametrize("spec", [SMALL2, RAGGED2, THREE, ODD3, FOUR])
def test_interpolation_and_coarse_operators(dd, spec):
    c, h, o = _pair(spec)
    for l in range(c.levels - 1):
        dims, n, N = h.level_info(l)
        P = np.zeros((N,) + dims + (n,), dtype=complex)
        dd.ddamg_get_interpolation(h, l, P)
        assert rel(P, o.levels[l].P) <= TOL64
    for l in range(1, c.levels):
        dims, n, _ = h.level_info(l)
        blk = np.zeros(dims + (9, n, n), dtype=complex)
        dd.ddamg_get_coarse_operator(h, l, blk)
        st = o.levels[l].op
        ref = np.concatenate([st.diag[..., None, :, :], np.moveaxis(st.fwd, 0, -3), np.moveaxis(st.bwd, 0, -3)],
                             axis=-3)
        assert rel(blk, ref) <= TOL64, (l, rel(blk, ref))
        # the gamma_5 relation between backward and forward blocks, on the GPU's blocks
        g = np.array([1.0] * (n // 2) + [-1.0] * (n // 2))
        for mu in range(4):
            lhs = np.roll(blk[..., 5 + mu, :, :], -1, axis=mu)
            rhs = g[:, None] * np.conj(np.swapaxes(blk[..., 1 + mu, :, :], -1, -2)) * g[None, :]
            if np.linalg.norm(rhs) == 0:     # extent-1 direction: every hop stays in the aggregate
                assert np.linalg.norm(lhs) == 0
            else:
                assert rel(lhs, rhs) <= 1e-12


@pytest.mark.parametrize("spec", [SMALL2, RAGGED2, THREE, ODD3])
def test_restrict_prolong(dd, spec):
    from oracle.transfer import restrict, prolong
    c, h, o = _pair(spec)
    for l in range(c.levels - 1):
        dims, n, N = h.level_info(l)
        cdims, nc, _ = h.level_info(l + 1)
        f = _fields(2, dims, n, 10 + l)
        g = _fields(2, cdims, nc, 20 + l)
        rref = restrict(o.levels[l].P, c.agg[l], f)
        pref = prolong(o.levels[l].P, c.agg[l], g)
        for prec, tol in ((0, TOL64), (1, TOL32)):
            out = np.zeros_like(g)
            dd.ddamg_restrict(h, l, prec, f, out, 2)
            assert rel(out, rref) <= tol
            out = np.zeros_like(f)
            dd.ddamg_prolong(h, l, prec, g, out, 2)
            assert rel(out, pref) <= tol


@pytest.mark.parametrize("cluster", [1, 0])
@pytest.mark.parametrize("spec", [SMALL2, THREE, ODD3, FOUR])
def test_coarse_apply_and_sap(dd, spec, cluster):
    c, h, o = _pair(spec)
    dd.ddamg_set_option(h, dd.DDAMG_OPT_SAP_CLUSTER, cluster)
    for l in range(1, c.levels):
        dims, n, _ = h.level_info(l)
        f = _fields(3, dims, n, 30 + l)
        ref = o.levels[l].op.apply(f)
        for prec, tol in ((0, TOL64), (1, TOL32)):
            out = np.zeros_like(f)
            dd.ddamg_apply(h, l, prec, f, out, 3)
            assert rel(out, ref) <= tol
        if l < c.levels - 1:
            b = _fields(2, dims, n, 40 + l)
            z0 = _fields(2, dims, n, 50 + l)
            for prec, tol, it in ((0, TOL64, 2), (1, TOL32, 1)):
                zref = np.stack([o.levels[l].sap.smooth(b[i], z0[i], it) for i in range(2)])
                z = z0.copy()
                dd.ddamg_smooth(h, l, prec, b, z, 2, it)
                assert rel(z, zref) <= tol, (l, prec, rel(z, zref))


def test_coarse_sap_large_blocks(dd):
    """Coarse SAP on 2x3x3x3-site blocks of 56 dof (3024 rows per block, not nested in the aggregates):
    the one-CTA-per-block kernel takes eight rows per thread to stay within its register budget.  FP64,
    FP32, and FP32 on FP16 blocks against the oracle."""
    from oracle.precision import stencil_half
    from oracle.smoother import SAP
    c, h, o = _pair(ODDBIG, mr_steps=3)
    dims, n, _ = h.level_info(1)
    assert n == 56 and o.levels[1].sap.block == (2, 3, 3, 3)
    f = _fields(2, dims, n, 31)
    out = np.zeros_like(f)
    dd.ddamg_apply(h, 1, 1, f, out, 2)                  # one FP32 application: the 2e-6 bound
    assert rel(out, o.levels[1].op.apply(f)) <= TOL32
    # one FP32 SAP iteration chains about eight such applications (two colours, each a residual and
    # three MR steps; 9 * 56 = 504-term sums per row) and block reductions over 3024 rows: bound 1e-5
    TOL_SAP32 = 1e-5
    b = _fields(2, dims, n, 41)
    z0 = _fields(2, dims, n, 51)
    for prec, tol, it in ((0, TOL64, 2), (1, TOL_SAP32, 1)):
        zref = np.stack([o.levels[1].sap.smooth(b[i], z0[i], it) for i in range(2)])
        z = z0.copy()
        dd.ddamg_smooth(h, 1, prec, b, z, 2, it)
        assert rel(z, zref) <= tol, (prec, rel(z, zref))
    dd.ddamg_set_option(h, dd.DDAMG_OPT_HALF_STORAGE, 1)
    sap = SAP(stencil_half(o.levels[1].op), o.levels[1].sap.block, 3)
    zref = np.stack([sap.smooth(b[i], z0[i], 1) for i in range(2)])
    z = z0.copy()
    dd.ddamg_smooth(h, 1, 1, b, z, 2, 1)
    assert rel(z, zref) <= TOL_SAP32, rel(z, zref)


@pytest.mark.parametrize("cluster", [1, 0])
@pytest.mark.parametrize("spec", [SMALL2, THREE])
def test_coarsest_even_odd_gmres(dd, spec, cluster):
    """Coarsest odd-even GMRES: thread-block-cluster kernel and the host-driven loop, vs the oracle."""
    from oracle.krylov import coarsest_solve
    c, h, o = _pair(spec, max_rhs=2)
    dd.ddamg_set_option(h, dd.DDAMG_OPT_COARSEST_CLUSTER, cluster)
    L = c.levels - 1
    dims, n, _ = h.level_info(L)
    b = _fields(2, dims, n, 60)
    z = np.zeros_like(b)
    dd.ddamg_coarse_solve(h, 0, b, z, 2)
    for i in range(2):
        zr, info = coarsest_solve(o.levels[L].eo, b[i], 5e-2, 50, 20)
        assert rel(z[i], zr) <= 1e-9
        eo = o.levels[L].eo
        rh = eo.schur_rhs(b[i]) - eo.schur_apply(eo.restrict_even(z[i]))
        assert np.linalg.norm(rh) <= 5e-2 * np.linalg.norm(eo.schur_rhs(b[i])) * (1 + 1e-9)
    z32 = np.zeros_like(b)
    dd.ddamg_coarse_solve(h, 1, b, z32, 2)
    eo = o.levels[L].eo
    for i in range(2):
        rh = eo.schur_rhs(b[i]) - eo.schur_apply(eo.restrict_even(z32[i]))
        assert np.linalg.norm(rh) <= 5e-2 * np.linalg.norm(eo.schur_rhs(b[i])) * 1.01


@pytest.mark.parametrize("graphs", [1, 0])
@pytest.mark.parametrize("spec", [SMALL2, THREE])
def test_kcycle(dd, spec, graphs):
    """One K-cycle (Alg. 2) vs the oracle: captured CUDA graph with device-driven inner solves, and eager."""
    c, h, o = _pair(spec)
    dd.ddamg_set_option(h, dd.DDAMG_OPT_GRAPHS, graphs)
    b = _fields(1, c.dims, 12, 70)
    z = np.zeros_like(b)
    dd.ddamg_kcycle(h, 0, 0, b, z, 1)
    assert rel(z[0], o.kcycle(0, b[0])) <= 1e-9
    z32 = np.zeros_like(b)
    dd.ddamg_kcycle(h, 0, 1, b, z32, 1)
    assert rel(z32[0], z[0]) <= 1e-3     # FP32 cycle vs FP64 cycle (inner stopping tolerances are 0.1 / 5e-2)


@pytest.mark.parametrize("spec", [BIG2, BIG3])
def test_kcycle_split_arnoldi(dd, spec):
    """K-cycle through the captured graph with Krylov vectors long enough for the cluster-split Arnoldi
    step (coarsest solve by the device-driven GMRES: coarsest cluster kernel off); two right-hand sides,
    and one of them alone gives the same bits."""
    c, h, o = _pair(spec, max_rhs=2)
    dd.ddamg_set_option(h, dd.DDAMG_OPT_COARSEST_CLUSTER, 0)
    dd.ddamg_set_option(h, dd.DDAMG_OPT_GRAPHS, 1)
    b = _fields(2, c.dims, 12, 71)
    z = np.zeros_like(b)
    dd.ddamg_kcycle(h, 0, 0, b, z, 2)
    for i in range(2):
        assert rel(z[i], o.kcycle(0, b[i])) <= 1e-9, rel(z[i], o.kcycle(0, b[i]))
    z1 = np.zeros_like(b[:1])
    dd.ddamg_kcycle(h, 0, 0, np.ascontiguousarray(b[1:2]), z1, 1)
    assert np.array_equal(z1[0], z[1])
    z32 = np.zeros_like(b)
    dd.ddamg_kcycle(h, 0, 1, b, z32, 2)
    assert rel(z32, z) <= 1e-3


def test_setup_initial_phase_alg3(dd):
    c, h, o = _pair(THREE, eta_passes=3, mr_steps=3)
    for l in range(c.levels - 1):
        dims, n, N = h.level_info(l)
        tv = np.zeros((N,) + dims + (n,), dtype=complex)
        dd.ddamg_get_testvectors(h, l, tv, N)
        assert rel(tv, o.levels[l].tv) <= 1e-11
        P = np.zeros_like(tv)
        dd.ddamg_get_interpolation(h, l, P)
        assert rel(P, o.levels[l].P) <= 1e-10


def test_setup_iterative_phase_alg4(dd):
    c, h, o = _pair(THREE, eta_passes=1, n_inv=2, mr_steps=2, nu=1)
    for l in range(c.levels - 1):
        dims, n, N = h.level_info(l)
        tv = np.zeros((N,) + dims + (n,), dtype=complex)
        dd.ddamg_get_testvectors(h, l, tv, N)
        assert rel(tv, o.levels[l].tv) <= 1e-8, (l, rel(tv, o.levels[l].tv))


def test_set_testvectors_and_rebuild(dd):
    from oracle.transfer import build_interpolation, galerkin
    c, h, o = _pair(SMALL2)
    tv = _fields(3, c.dims, 12, 80)
    dd.ddamg_set_testvectors(h, 0, tv, 3)
    dd.ddamg_rebuild(h, 0)
    P = np.zeros_like(tv)
    dd.ddamg_get_interpolation(h, 0, P)
    Pr = build_interpolation(tv, c.agg[0])
    assert rel(P, Pr) <= TOL64
    dims, n, _ = h.level_info(1)
    blk = np.zeros(dims + (9, n, n), dtype=complex)
    dd.ddamg_get_coarse_operator(h, 1, blk)
    st = galerkin(o.levels[0].op, Pr, c.agg[0])
    assert rel(blk[..., 0, :, :], st.diag) <= TOL64


def test_rank_deficient_test_vectors_are_reported(dd):
    c, h, o = _pair(SMALL2)
    tv = _fields(3, c.dims, 12, 81)
    tv[2] = tv[0] + 0.5 * tv[1]
    dd.ddamg_set_testvectors(h, 0, np.ascontiguousarray(tv), 3)
    with pytest.raises(dd.DdamgError) as e:
        dd.ddamg_rebuild(h, 0)
    assert e.value.code == dd.DDAMG_ERR_SINGULAR


def _check_solution(op, b, x, tol=1e-10):
    r = b - op.apply(x)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_two_level_fp64_workload(dd, precision):
    """The two-level 8^4 workload: true residual <= 1e-10 with the oracle's D; iterations near the oracle's."""
    c = Case(**C1, m0=golden_mass("eps0.3_csw0"))
    U = c.gauge()
    tv = c.random_tv()
    h = c.gpu(precision, U, tv)
    b = np.ascontiguousarray(synth.random_spinors(1, c.dims, 1))
    x = np.zeros_like(b)
    st = dd.ddamg_solve(h, b, x, 1, 1e-10)
    from oracle.wilson import WilsonOp
    op = WilsonOp.build(U, c.m0, c.csw, c.bc_t)
    assert st[0]["converged"]
    assert _check_solution(op, b[0], x[0]) <= 1e-10
    if precision == 0:
        o = c.oracle(U, tv)
        xo, info = o.solve(b[0], tol=1e-10, restart=25)
        assert abs(st[0]["iterations"] - info.iterations) <= max(2, 0.2 * info.iterations)


def test_solve_three_level_and_edge_rhs(dd):
    c = Case(**THREE, n_inv=1, eta_passes=3, max_rhs=3, m0=-0.35, nu=3)
    U = c.gauge()
    h = c.gpu(1, U)
    b = np.ascontiguousarray(synth.random_spinors(3, c.dims, 2))
    b[1] = 0.0                                             # zero right-hand side
    b[2] = synth.point_sources(c.dims, 4)[5]               # point source
    x = np.zeros_like(b)
    st = dd.ddamg_solve(h, b, x, 3, 1e-10)
    from oracle.wilson import WilsonOp
    op = WilsonOp.build(U, c.m0, c.csw, c.bc_t)
    assert st[1]["converged"] and np.all(x[1] == 0)
    for i in (0, 2):
        assert st[i]["converged"] and _check_solution(op, b[i], x[i]) <= 1e-10


@pytest.mark.parametrize("graphs", [1, 0])
def test_batch_invariance(dd, graphs):
    """Each right-hand side gives the same bits alone and inside a batch (fixed reduction partitions)."""
    c = Case(**THREE, n_inv=1, eta_passes=2, max_rhs=4, m0=-0.3)
    h = c.gpu(1)
    dd.ddamg_set_option(h, dd.DDAMG_OPT_GRAPHS, graphs)
    b = np.ascontiguousarray(synth.random_spinors(4, c.dims, 3))
    xb = np.zeros_like(b)
    dd.ddamg_solve(h, b, xb, 4, 1e-10)
    for i in range(4):
        xi = np.zeros_like(b[i:i + 1])
        dd.ddamg_solve(h, np.ascontiguousarray(b[i:i + 1]), xi, 1, 1e-10)
        assert np.array_equal(xi[0], xb[i])


def test_device_pointers_through_torch(dd):
    import torch
    c = Case(**SMALL2)
    h = c.gpu(0)
    f = _fields(2, c.dims, 12, 90)
    ref = np.zeros_like(f)
    dd.ddamg_apply(h, 0, 0, f, ref, 2)
    ft = torch.from_numpy(f).cuda()
    out = torch.zeros_like(ft)
    dd.ddamg_apply(h, 0, 0, ft, out, 2)
    assert np.array_equal(out.cpu().numpy(), ref)


def test_odd_extents_plain_coarsest_gmres_and_solve(dd):
    """Coarsest lattice with odd extents: plain GMRES on D_L, same as the oracle's; full solve to 1e-10."""
    from oracle.krylov import gmres
    c, h, o = _pair(ODD3, max_rhs=2)
    assert o.levels[2].eo is None and o.levels[1].sap.block == (2, 3, 3, 3)
    dims, n, _ = h.level_info(2)
    b = _fields(2, dims, n, 61)
    z = np.zeros_like(b)
    dd.ddamg_coarse_solve(h, 0, b, z, 2)
    for i in range(2):
        zr, info = gmres(o.levels[2].op.apply, b[i], m=50, tol=5e-2, max_cycles=20)
        assert rel(z[i], zr) <= 1e-9
    z32 = np.zeros_like(b)
    dd.ddamg_coarse_solve(h, 1, b, z32, 2)
    for i in range(2):
        assert np.linalg.norm(b[i] - o.levels[2].op.apply(z32[i])) <= 5e-2 * np.linalg.norm(b[i]) * 1.01
    bb = np.ascontiguousarray(synth.random_spinors(1, c.dims, 62))
    x = np.zeros_like(bb)
    st = dd.ddamg_solve(h, bb, x, 1, 1e-10)
    assert st[0]["converged"]
    assert np.linalg.norm(bb[0] - o.levels[0].op.apply(x[0])) <= 1e-10 * np.linalg.norm(bb[0])


@pytest.mark.parametrize("precision", [0, 2])
def test_four_level_solve(dd, precision):
    """Four levels (K-cycles nested twice, plain-GMRES coarsest): true residual <= 1e-10; FP64 K-cycle vs oracle."""
    c = Case(**FOUR, n_inv=1, eta_passes=2, m0=-0.3, nu=2)
    U = c.gauge()
    tv = c.random_tv()
    h = c.gpu(precision, U, tv)
    b = np.ascontiguousarray(synth.random_spinors(1, c.dims, 71))
    x = np.zeros_like(b)
    st = dd.ddamg_solve(h, b, x, 1, 1e-10)
    from oracle.wilson import WilsonOp
    op = WilsonOp.build(U, c.m0, c.csw, c.bc_t)
    assert st[0]["converged"]
    assert np.linalg.norm(b[0] - op.apply(x[0])) <= 1e-10 * np.linalg.norm(b[0])
    if precision == 0:
        o = c.oracle(U, tv)
        z = np.zeros_like(b)
        dd.ddamg_kcycle(h, 0, 0, b, z, 1)
        assert rel(z[0], o.kcycle(0, b[0])) <= 1e-9
