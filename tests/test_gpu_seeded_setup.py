"""The library draws Alg. 3's random start vectors itself from params.seed (no host fields).

The device generator and synth.philox_fields implement the same counter-based steps, so
(1) with no smoothing and no Alg. 4 the level-0 test vectors and the extra level-1 vectors
after the setup are the generator's fields bit for bit, and (2) a full seeded setup equals,
bit for bit, the setup that is handed those same fields as host arrays.
"""
import numpy as np
import pytest

import synth
from cases import Case, THREE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1307_6101_gb300 as m
    return m


def test_seeded_random_vectors_are_the_generator_fields(dd):
    c = Case(**THREE, n_inv=0, eta_passes=0)
    seed = 0x1234_5678_9ABC
    p = c.gpu_params(0)
    p.seed = seed
    h = dd.ddamg_setup(c.gauge(), c.dims, c.bc_t, c.m0, c.csw, p, None)
    ld = c.level_dims()
    ref = synth.philox_test_vectors(ld, c.n_tv, seed)
    tv0 = np.zeros_like(ref[0])
    dd.ddamg_get_testvectors(h, 0, tv0, c.n_tv[0])
    assert np.array_equal(tv0, ref[0])
    take = c.n_tv[0]
    tv1 = np.zeros((c.n_tv[1],) + ld[1] + (2 * c.n_tv[0],), dtype=np.complex128)
    dd.ddamg_get_testvectors(h, 1, tv1, c.n_tv[1])
    assert np.array_equal(tv1[take:], ref[1])
    h.free()


@pytest.mark.parametrize("precision", [0, 2])
def test_seeded_setup_equals_setup_from_host_fields(dd, precision):
    c = Case(**THREE, n_inv=1, eta_passes=2)
    seed = 77
    p = c.gpu_params(precision)
    p.seed = seed
    U = c.gauge()
    h1 = dd.ddamg_setup(U, c.dims, c.bc_t, c.m0, c.csw, p, None)
    tv = synth.philox_test_vectors(c.level_dims(), c.n_tv, seed)
    h2 = dd.ddamg_setup(U, c.dims, c.bc_t, c.m0, c.csw, c.gpu_params(precision), tv)
    for lvl, n in enumerate(c.n_tv):
        dims, ndof, _ = h1.level_info(lvl)
        P1 = np.zeros((n,) + tuple(dims) + (ndof,), dtype=np.complex128)
        P2 = np.zeros_like(P1)
        dd.ddamg_get_interpolation(h1, lvl, P1)
        dd.ddamg_get_interpolation(h2, lvl, P2)
        assert np.array_equal(P1, P2), lvl
    b = np.ascontiguousarray(synth.random_spinors(1, c.dims, 5))
    x1, x2 = np.zeros_like(b), np.zeros_like(b)
    s1 = dd.ddamg_solve(h1, b, x1, 1, 1e-10)
    s2 = dd.ddamg_solve(h2, b, x2, 1, 1e-10)
    assert s1[0]["converged"] and np.array_equal(x1, x2)
    h1.free()
    h2.free()
