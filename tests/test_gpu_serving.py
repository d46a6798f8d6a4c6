"""Serving (continuous batching over resident hierarchies): every request's result
is the same alone and in a mix of overlapping requests, admission refuses a
hierarchy whose device footprint exceeds the budget, and the footprint estimate
tracks the allocations."""
import threading
import time

import numpy as np
import pytest

import synth
from cases import Case, SMALL2, THREE, BIG3, SAP4

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1307_6101_gb300 as m
    return m


def _true_residual(U, c, b, x):
    from oracle.wilson import WilsonOp
    op = WilsonOp.build(U, c.m0, c.csw, c.bc_t)
    return np.linalg.norm(b - op.apply(x)) / np.linalg.norm(b)


def _requests(c, sizes, seed):
    return [np.ascontiguousarray(synth.random_spinors(n, c.dims, seed + k)) for k, n in enumerate(sizes)]


def test_results_same_alone_and_in_the_mix(dd):
    c = Case(**THREE, n_inv=1, eta_passes=2, max_rhs=3, m0=-0.35, nu=2)
    U = c.gauge()
    h = c.gpu(2, U)
    srv = dd.Server()
    hid = srv.add(h)
    reqs = _requests(c, [2, 1, 3, 1], 40)
    reqs[3][0] = synth.point_sources(c.dims, 4)[2]
    # alone: one request at a time
    alone = []
    for b in reqs:
        x = np.zeros_like(b)
        rid = srv.submit(hid, b, len(b), 1e-10)
        st, t, rc = srv.wait(rid, x, len(b))
        assert rc == dd.DDAMG_OK and all(s["converged"] for s in st)
        alone.append(x)
    # mixed: overlapping submissions, more columns than batch slots (7 > 3)
    ids = []
    for k, b in enumerate(reqs):
        ids.append(srv.submit(hid, b, len(b), 1e-10))
        time.sleep(0.002 * k)
    mixed = []
    for rid, b in zip(ids, reqs):
        x = np.zeros_like(b)
        st, t, rc = srv.wait(rid, x, len(b))
        assert rc == dd.DDAMG_OK
        assert t[1] >= t[2] >= 0 and t[0] >= 0
        mixed.append(x)
    srv.free()
    for b, xa, xm in zip(reqs, alone, mixed):
        assert np.array_equal(xa, xm)
        for i in range(len(b)):
            assert _true_residual(U, c, b[i], xm[i]) <= 1e-10
    # and the same as a plain batched solve on the handle (same restart cycles, same kernels)
    b = reqs[2]
    x = np.zeros_like(b)
    dd.ddamg_solve(h, b, x, len(b), 1e-10)
    assert np.array_equal(x, alone[2])


def test_two_hierarchies_overlap_and_threads_submit(dd):
    c1 = Case(**SMALL2, max_rhs=2)
    c2 = Case(**THREE, n_inv=1, eta_passes=2, max_rhs=2, m0=-0.35, nu=2)
    h1, h2 = c1.gpu(1), c2.gpu(2)
    srv = dd.Server()
    ids = [srv.add(h1), srv.add(h2)]
    cases = [c1, c2]
    out = {}

    def client(k):
        c = cases[k]
        res = []
        for j in range(3):
            b = np.ascontiguousarray(synth.random_spinors(1 + j % 2, c.dims, 70 + 10 * k + j))
            rid = srv.submit(ids[k], b, len(b), 1e-10)
            x = np.zeros_like(b)
            st, t, rc = srv.wait(rid, x, len(b))
            res.append((rc, st))
        out[k] = res

    th = [threading.Thread(target=client, args=(k,)) for k in (0, 1)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    srv.free()
    for k in (0, 1):
        assert len(out[k]) == 3
        for rc, st in out[k]:
            assert rc == dd.DDAMG_OK and all(s["converged"] and s["true_residual"] <= 1e-10 for s in st)


def test_concurrent_hierarchies_give_the_bits_of_solo_solves(dd):
    """Two hierarchies whose worker threads run at the same time on their own streams: every
    request gives the same bits as when its hierarchy serves it alone (reductions of different
    streams use separate scratch)."""
    c1 = Case(**BIG3, n_inv=1, eta_passes=2, max_rhs=3, m0=-0.35, nu=2)
    c2 = Case(**SAP4, n_inv=1, eta_passes=2, max_rhs=3)
    hs = [c1.gpu(2), c2.gpu(2)]
    cs = [c1, c2]
    reqs = [[np.ascontiguousarray(synth.random_spinors(n, c.dims, 90 + 10 * k + j)) for j, n in enumerate((3, 2, 3, 1))]
            for k, c in enumerate(cs)]
    srv = dd.Server()
    try:
        ids = [srv.add(h) for h in hs]
        alone = [[], []]
        for k in (0, 1):
            for b in reqs[k]:
                x = np.zeros_like(b)
                st, t, rc = srv.wait(srv.submit(ids[k], b, len(b), 1e-10), x, len(b))
                assert rc == dd.DDAMG_OK and all(q["converged"] for q in st)
                alone[k].append(x)
        # all requests of both hierarchies at once
        rids = [[srv.submit(ids[k], b, len(b), 1e-10) for b in reqs[k]] for k in (0, 1)]
        for k in (0, 1):
            for rid, b, xa in zip(rids[k], reqs[k], alone[k]):
                x = np.zeros_like(b)
                st, t, rc = srv.wait(rid, x, len(b))
                assert rc == dd.DDAMG_OK
                assert np.array_equal(x, xa)
    finally:
        srv.free()


def test_admission_by_footprint_and_estimate(dd):
    c = Case(**THREE, n_inv=0, eta_passes=1, max_rhs=2, m0=-0.35)
    h = c.gpu(2)
    used = dd.ddamg_device_bytes(h)
    est = dd.ddamg_estimate_bytes(c.dims, c.gpu_params(2))
    assert 0.8 * used <= est <= 1.5 * used, (est, used)
    small = dd.Server(hbm_budget=used // 2)
    with pytest.raises(dd.DdamgError) as e:
        small.add(h)
    assert e.value.code == dd.DDAMG_ERR_ADMISSION
    small.free()
    ok = dd.Server(hbm_budget=used + 1)
    ok.add(h)
    ok.free()
