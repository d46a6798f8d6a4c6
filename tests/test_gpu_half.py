"""Parity of the FP16-storage FP32 kernels with the FP64 oracle applied to the same
FP16-rounded operator data (oracle.precision): links and clover term without
scale, P with one scale per aggregate and chirality, coarse blocks with one
scale per site.

Each test builds the hierarchy in FP64 (so that P and the coarse blocks agree
with the oracle's to 1e-12), switches the handle to FP16 storage and compares
one FP32 operation with the oracle on the dequantised data: <= 2e-6 relative,
the FP32 bound.  The quantisation error itself (~1e-4 relative) is far above
that bound, so each test also shows that the FP16 data was the data used.
"""
import numpy as np
import pytest

import synth
from cases import Case, rel, SMALL2, RAGGED2, THREE, C1, golden_mass

pytestmark = pytest.mark.gpu

TOL32 = 2e-6


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1307_6101_gb300 as m
    return m


def _half_pair(dd, spec, **kw):
    c = Case(**{**spec, **kw})
    U = c.gauge()
    tv = c.random_tv()
    h = c.gpu(0, U, tv)
    o = c.oracle(U, tv)
    dd.ddamg_set_option(h, dd.DDAMG_OPT_HALF_STORAGE, 1)
    assert dd.ddamg_get_option(h, dd.DDAMG_OPT_HALF_STORAGE) == 1
    return c, h, o, U


def _fields(n, dims, ndof, seed):
    return np.ascontiguousarray(synth.random_fields(n, dims, ndof, seed))


@pytest.mark.parametrize("spec,csw,bc", [(SMALL2, 1.0, -1), (SMALL2, 0.0, 1), (RAGGED2, 1.3, -1)])
def test_fine_apply_half(dd, spec, csw, bc):
    from oracle.precision import fine_op_half
    c, h, o, U = _half_pair(dd, spec, csw=csw, bc_t=bc)
    f = _fields(3, c.dims, 12, 7)
    ref = fine_op_half(U, c.m0, c.csw, c.bc_t).apply(f)
    out = np.zeros_like(f)
    dd.ddamg_apply(h, 0, 1, f, out, 3)
    assert rel(out, ref) <= TOL32, rel(out, ref)
    assert rel(out, o.levels[0].op.apply(f)) > 1e-5          # FP16 data, not the FP32 copy
    # switching back gives the FP32-storage kernels again
    dd.ddamg_set_option(h, dd.DDAMG_OPT_HALF_STORAGE, 0)
    out32 = np.zeros_like(f)
    dd.ddamg_apply(h, 0, 1, f, out32, 3)
    assert rel(out32, o.levels[0].op.apply(f)) <= TOL32


@pytest.mark.parametrize("spec", [SMALL2, RAGGED2])
def test_fine_sap_half(dd, spec):
    from oracle.precision import fine_op_half
    from oracle.smoother import SAP
    c, h, o, U = _half_pair(dd, spec, mr_steps=4)
    sap = SAP(fine_op_half(U, c.m0, c.csw, c.bc_t), c.sap[0], c.mr_steps)
    b = _fields(2, c.dims, 12, 8)
    z0 = _fields(2, c.dims, 12, 9)
    ref = np.stack([sap.smooth(b[i], z0[i], 1) for i in range(2)])
    z = z0.copy()
    dd.ddamg_smooth(h, 0, 1, b, z, 2, 1)
    assert rel(z, ref) <= TOL32, rel(z, ref)


@pytest.mark.parametrize("spec", [SMALL2, RAGGED2, THREE])
def test_restrict_prolong_half(dd, spec):
    from oracle.transfer import restrict, prolong
    from oracle.precision import interpolation_half
    c, h, o, U = _half_pair(dd, spec)
    for l in range(c.levels - 1):
        dims, n, N = h.level_info(l)
        cdims, nc, _ = h.level_info(l + 1)
        Pq = interpolation_half(o.levels[l].P, c.agg[l])
        f = _fields(2, dims, n, 10 + l)
        g = _fields(2, cdims, nc, 20 + l)
        out = np.zeros_like(g)
        dd.ddamg_restrict(h, l, 1, f, out, 2)
        assert rel(out, restrict(Pq, c.agg[l], f)) <= TOL32
        assert rel(out, restrict(o.levels[l].P, c.agg[l], f)) > 1e-5
        out = np.zeros_like(f)
        dd.ddamg_prolong(h, l, 1, g, out, 2)
        assert rel(out, prolong(Pq, c.agg[l], g)) <= TOL32


@pytest.mark.parametrize("cluster", [1, 0])
@pytest.mark.parametrize("spec", [SMALL2, THREE])
def test_coarse_apply_and_sap_half(dd, spec, cluster):
    from oracle.precision import stencil_half
    from oracle.smoother import SAP
    c, h, o, U = _half_pair(dd, spec)
    dd.ddamg_set_option(h, dd.DDAMG_OPT_SAP_CLUSTER, cluster)
    for l in range(1, c.levels):
        dims, n, _ = h.level_info(l)
        stq = stencil_half(o.levels[l].op)
        f = _fields(3, dims, n, 30 + l)
        out = np.zeros_like(f)
        dd.ddamg_apply(h, l, 1, f, out, 3)
        assert rel(out, stq.apply(f)) <= TOL32, (l, rel(out, stq.apply(f)))
        assert rel(out, o.levels[l].op.apply(f)) > 1e-5
        if l < c.levels - 1:
            sap = SAP(stq, c.sap[l], c.mr_steps)
            b = _fields(2, dims, n, 40 + l)
            z0 = _fields(2, dims, n, 50 + l)
            zref = np.stack([sap.smooth(b[i], z0[i], 1) for i in range(2)])
            z = z0.copy()
            dd.ddamg_smooth(h, l, 1, b, z, 2, 1)
            assert rel(z, zref) <= TOL32, (l, rel(z, zref))


@pytest.mark.parametrize("cluster", [1, 0])
@pytest.mark.parametrize("spec", [SMALL2, THREE])
def test_coarsest_solve_half(dd, spec, cluster):
    """The coarsest odd-even GMRES on FP16 blocks meets its tolerance on the FP16 operator's Schur complement."""
    from oracle.precision import even_odd_half
    c, h, o, U = _half_pair(dd, spec, max_rhs=2)
    dd.ddamg_set_option(h, dd.DDAMG_OPT_COARSEST_CLUSTER, cluster)
    L = c.levels - 1
    dims, n, _ = h.level_info(L)
    eo = even_odd_half(o.levels[L].op)
    b = _fields(2, dims, n, 60)
    z = np.zeros_like(b)
    dd.ddamg_coarse_solve(h, 1, b, z, 2)
    for i in range(2):
        rh = eo.schur_rhs(b[i]) - eo.schur_apply(eo.restrict_even(z[i]))
        assert np.linalg.norm(rh) <= 5e-2 * np.linalg.norm(eo.schur_rhs(b[i])) * 1.01


def _true_residual(U, c, b, x):
    from oracle.wilson import WilsonOp
    op = WilsonOp.build(U, c.m0, c.csw, c.bc_t)
    return np.linalg.norm(b - op.apply(x)) / np.linalg.norm(b)


def test_solve_two_level_half_storage(dd):
    """precision = 2 (FP32 preconditioner on FP16 storage inside FP64 FGMRES): true residual <= 1e-10."""
    c = Case(**C1, m0=golden_mass("eps0.3_csw0"))
    U = c.gauge()
    h = c.gpu(2, U)
    assert dd.ddamg_get_option(h, dd.DDAMG_OPT_HALF_STORAGE) == 1
    b = np.ascontiguousarray(synth.random_spinors(1, c.dims, 1))
    x = np.zeros_like(b)
    st = dd.ddamg_solve(h, b, x, 1, 1e-10)
    assert st[0]["converged"]
    assert _true_residual(U, c, b[0], x[0]) <= 1e-10
    # same solve with FP32 storage: the FP16 rounding may cost iterations, but few
    h32 = c.gpu(1, U)
    x32 = np.zeros_like(b)
    st32 = dd.ddamg_solve(h32, b, x32, 1, 1e-10)
    assert st[0]["iterations"] <= st32[0]["iterations"] + max(3, 0.25 * st32[0]["iterations"])


def test_solve_three_level_half_storage(dd):
    c = Case(**THREE, n_inv=1, eta_passes=3, max_rhs=2, m0=-0.35, nu=3)
    U = c.gauge()
    h = c.gpu(2, U)
    b = np.ascontiguousarray(synth.random_spinors(2, c.dims, 2))
    b[1] = synth.point_sources(c.dims, 4)[3]
    x = np.zeros_like(b)
    st = dd.ddamg_solve(h, b, x, 2, 1e-10)
    for i in range(2):
        assert st[i]["converged"] and _true_residual(U, c, b[i], x[i]) <= 1e-10
