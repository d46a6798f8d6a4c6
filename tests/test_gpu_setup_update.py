"""Setup acceleration: Alg. 4 in batches of test vectors gives the same hierarchy bit for bit as one
vector at a time; a hierarchy updated to a new gauge field (operators rebuilt from the current test
vectors, then Alg. 4 passes) solves the new system to the FP64 true residual, in about the
iterations of a fresh setup."""
import numpy as np
import pytest

import synth
from cases import Case, THREE, SAP4, FOUR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1307_6101_gb300 as m
    return m


def _interp(dd, h, c):
    out = []
    for lvl, n in enumerate(c.n_tv):
        dims, ndof, _ = h.level_info(lvl)
        P = np.zeros((n,) + tuple(dims) + (ndof,), dtype=np.complex128)
        dd.ddamg_get_interpolation(h, lvl, P)
        out.append(P)
    return out


@pytest.mark.parametrize("spec,precision", [(THREE, 0), (THREE, 2), (FOUR, 2)])
def test_batched_alg4_equals_one_vector_at_a_time(dd, spec, precision):
    c = Case(**spec, n_inv=2, eta_passes=2)
    U = c.gauge()
    tv = c.random_tv()
    p1 = c.gpu_params(precision)
    p1.setup_batch = 1
    p4 = c.gpu_params(precision)
    p4.setup_batch = 4
    h1 = dd.ddamg_setup(U, c.dims, c.bc_t, c.m0, c.csw, p1, tv)
    h4 = dd.ddamg_setup(U, c.dims, c.bc_t, c.m0, c.csw, p4, tv)
    for a, b in zip(_interp(dd, h1, c), _interp(dd, h4, c)):
        assert np.array_equal(a, b)
    t1, t4 = dd.ddamg_setup_times(h1), dd.ddamg_setup_times(h4)
    print("\nAlg. 4 K-cycle seconds, one at a time / batched:", t1[0]["kcycle"], t4[0]["kcycle"])
    h1.free()
    h4.free()


def _perturbed(U, delta, seed):
    import synth
    rng = np.random.default_rng(seed)
    W = synth.su3_matrices(U.shape[:-2], delta, rng)
    return np.ascontiguousarray(W @ U)


@pytest.mark.parametrize("precision", [1, 2])
def test_update_gauge(dd, precision):
    from oracle.wilson import WilsonOp
    c = Case(**{**SAP4, "levels": 3, "agg": ((4, 4, 4, 4), (2, 1, 1, 1)), "n_tv": (6, 8),
                "sap": ((4, 4, 4, 4), (1, 1, 2, 2))}, n_inv=2, eta_passes=2, m0=-0.3, max_rhs=2)
    U = c.gauge()
    h = c.gpu(precision, U)
    U2 = _perturbed(U, 0.05, 17)
    b = np.ascontiguousarray(synth.random_spinors(2, c.dims, 3))
    fresh = c.gpu(precision, U2)
    xf = np.zeros_like(b)
    sf = dd.ddamg_solve(fresh, b, xf, 2, 1e-10)
    fresh.free()
    dd.ddamg_update_gauge(h, U2, 1)
    # the fine operator is the new one
    op2 = WilsonOp.build(U2, c.m0, c.csw, c.bc_t)
    f = np.ascontiguousarray(synth.random_spinors(1, c.dims, 9))
    out = np.zeros_like(f)
    dd.ddamg_apply(h, 0, 0, f, out, 1)
    ref = op2.apply(f[0])
    assert np.linalg.norm(out[0] - ref) <= 1e-12 * np.linalg.norm(ref)
    x = np.zeros_like(b)
    su = dd.ddamg_solve(h, b, x, 2, 1e-10)
    for i in range(2):
        assert su[i]["converged"]
        assert np.linalg.norm(b[i] - op2.apply(x[i])) <= 1e-10 * np.linalg.norm(b[i])
        assert su[i]["iterations"] <= sf[i]["iterations"] + max(3, 0.25 * sf[i]["iterations"]), (su, sf)
    # an update without Alg. 4 passes (operators rebuilt only) still solves the new system
    dd.ddamg_update_gauge(h, U, 0)
    op = WilsonOp.build(U, c.m0, c.csw, c.bc_t)
    s0 = dd.ddamg_solve(h, b, x, 2, 1e-10)
    for i in range(2):
        assert s0[i]["converged"] and np.linalg.norm(b[i] - op.apply(x[i])) <= 1e-10 * np.linalg.norm(b[i])
    h.free()
