"""Parity at the full sizes of the workloads, with the inputs, parameters and launch
configuration that bench.py times.

16^3x32, three levels (the benchmark workload): the fine operator on the whole
lattice against the oracle's D (FP64 <= 1e-12; FP32 on FP16 storage <= 2e-6
against the oracle's operator on the same FP16 data), one SAP iteration of the
4^4-block kernel against the oracle's SAP on that operator, and the mixed solve
(CUDA graphs, FP16 storage) to a true relative residual <= 1e-10 measured with
the oracle's D on the whole lattice.

32^3x64, three levels, twelve right-hand sides per batched solve: the twelve
spin-colour point sources at a seeded site, then twelve complex N(0,1) fields.
The oracle evaluates D site by site on a seeded sample of sites
(oracle.wilson.apply_at_sites): the fine operator against the library's on the
sample, and b - D x of every solution on the sample, which must lie below
1e-10 |b| because the whole residual does.  The library's own FP64 true residual
is <= 1e-10 for every column, and a column solved alone equals its batched
result bit for bit.

48^3x96, four levels, one right-hand side, mixed precision: only with
DDAMG_TEST_LARGE=1 and enough memory (about 230 GB on the device, about 130 GB
on the host while the inputs are generated); the solve's residual on sampled
sites by the oracle and the library's FP64 true residual.
"""
import os
import time

import numpy as np
import pytest

import synth
from cases import rel

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-6
TOL = 1e-10


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1307_6101_gb300 as m
    return m


def _params(dd, w, precision, max_rhs):
    return dd.ddamg_default_params(levels=w["levels"], agg=w["agg"], n_tv=w["n_tv"], sap_block=w["sap"],
                                   mr_steps=w["mr_steps"], nu=w["nu"], n_inv=w["n_inv"],
                                   outer_restart=w["outer_restart"], precision=precision, max_rhs=max_rhs,
                                   seed=w["tv_seed"], setup_batch=w.get("setup_batch", 0))


def _sites(dims, n, seed, extra=()):
    rng = np.random.default_rng(seed)
    s = [tuple(int(rng.integers(0, d)) for d in dims) for _ in range(n)]
    # both time boundaries (antiperiodic hops) and the given sites
    s += [(0,) + s[0][1:], (dims[0] - 1,) + s[1][1:]] + [tuple(e) for e in extra]
    return s


def test_benchmark_workload_16c32(dd):
    import bench
    from oracle.wilson import WilsonOp
    from oracle.precision import fine_op_half
    from oracle.smoother import SAP
    w = bench.WORKLOADS["three_level_16c32"]
    U, tv, rhs = bench.inputs(w)
    m0 = bench.mass(w["mass"])
    t0 = time.perf_counter()
    h = dd.ddamg_setup(U, w["dims"], -1, m0, w["csw"], _params(dd, w, 2, w["nrhs"]), tv)
    print(f"\n16^3x32 mixed setup {time.perf_counter() - t0:.1f} s")
    op = WilsonOp.build(U, m0, w["csw"], -1)
    opq = fine_op_half(U, m0, w["csw"], -1)
    f = np.ascontiguousarray(synth.random_spinors(1, w["dims"], 11))
    out = np.zeros_like(f)
    dd.ddamg_apply(h, 0, 0, f, out, 1)
    assert rel(out, op.apply(f)) <= TOL64
    out = np.zeros_like(f)
    dd.ddamg_apply(h, 0, 1, f, out, 1)                     # FP32 arithmetic on the FP16 data
    assert rel(out, opq.apply(f)) <= TOL32, rel(out, opq.apply(f))
    # one SAP iteration (both colours, 4 MR steps per block) of the 4^4-block kernel
    b = np.ascontiguousarray(synth.random_spinors(1, w["dims"], 12))
    z0 = np.ascontiguousarray(synth.random_spinors(1, w["dims"], 13))
    ref = SAP(opq, w["sap"][0], w["mr_steps"]).smooth(b[0], z0[0], 1)
    z = z0.copy()
    dd.ddamg_smooth(h, 0, 1, b, z, 1, 1)
    assert rel(z[0], ref) <= TOL32, rel(z[0], ref)
    # the benchmark's solve: mixed precision, CUDA graphs, true residual with the oracle's D
    x = np.zeros_like(rhs)
    st = dd.ddamg_solve(h, rhs, x, w["nrhs"], TOL)
    h.free()
    for i in range(w["nrhs"]):
        assert st[i]["converged"]
        r = np.linalg.norm(rhs[i] - op.apply(x[i])) / np.linalg.norm(rhs[i])
        assert r <= TOL, r


def test_batched_workload_32c64(dd):
    import bench
    from oracle.wilson import WilsonOp, apply_at_sites
    w = bench.WORKLOADS["batched_32c64"]
    nb = w["nrhs"]
    U, tv, _ = bench.inputs(w, with_rhs=False)
    m0 = bench.mass(w["mass"])
    csw = w["csw"]
    bc = (-1, 1, 1, 1)
    build = lambda Up: WilsonOp.build(Up, m0, csw, 1)   # noqa: E731 (patch operator, periodic)
    t0 = time.perf_counter()
    h = dd.ddamg_setup(U, w["dims"], -1, m0, csw, _params(dd, w, 2, nb), tv)
    print(f"\n32^3x64 mixed setup {time.perf_counter() - t0:.1f} s, device {dd.ddamg_device_bytes(h) / 1e9:.1f} GB")
    del tv
    # fine operator on a sample of sites
    f = np.ascontiguousarray(synth.random_spinors(1, w["dims"], 21))
    out = np.zeros_like(f)
    dd.ddamg_apply(h, 0, 0, f, out, 1)
    sites = _sites(w["dims"], 40, 22)
    ref = apply_at_sites(build, U, f, bc, sites)
    got = np.stack([out[0][s] for s in sites])
    assert rel(got, ref[0]) <= TOL64, rel(got, ref[0])
    # twelve point sources, then twelve N(0,1) fields, each batch in one solve
    pts = synth.point_sources(w["dims"], 23)
    x0 = tuple(int(i) for i in np.argwhere(pts[0].reshape(-1, 12).any(axis=1).reshape(w["dims"]))[0])
    batches = [np.ascontiguousarray(pts), np.ascontiguousarray(synth.random_spinors(nb, w["dims"], 24))]
    del pts
    sites = _sites(w["dims"], 24, 25, extra=[x0])
    for bi, b in enumerate(batches):
        x = np.zeros_like(b)
        t0 = time.perf_counter()
        st = dd.ddamg_solve(h, b, x, nb, TOL)
        print(f"batch {bi}: {nb} RHS in {time.perf_counter() - t0:.2f} s, iterations "
              f"{[s['iterations'] for s in st]}")
        assert all(s["converged"] and s["true_residual"] <= TOL for s in st), st
        dx = apply_at_sites(build, U, x, bc, sites)             # [nb, nsites, 12]
        for i in range(nb):
            rs = np.stack([b[i][s] for s in sites]) - dx[i]
            assert np.linalg.norm(rs) <= TOL * np.linalg.norm(b[i]), (bi, i, np.linalg.norm(rs))
        if bi == 1:
            k = 5
            xa = np.zeros_like(b[k:k + 1])
            dd.ddamg_solve(h, np.ascontiguousarray(b[k:k + 1]), xa, 1, TOL)
            assert np.array_equal(xa[0], x[k])
    h.free()


def _host_available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


@pytest.mark.skipif(os.environ.get("DDAMG_TEST_LARGE") != "1",
                    reason="48^3x96 four levels: about 230 GB of device memory and minutes of setup (opt-in)")
def test_four_level_workload_48c96(dd):
    import torch
    import bench
    from oracle.wilson import WilsonOp, apply_at_sites
    w = bench.WORKLOADS["four_level_48c96"]
    p = _params(dd, w, 2, w["nrhs"])
    need = dd.ddamg_estimate_bytes(w["dims"], p)
    free = torch.cuda.mem_get_info()[0]
    if need > 0.95 * free or _host_available_bytes() < 40e9:
        pytest.skip(f"needs {need / 1e9:.0f} GB of {free / 1e9:.0f} GB free on the device and 40 GB on the host")
    U, tv, rhs = bench.inputs(w)
    m0 = bench.mass(w["mass"])
    t0 = time.perf_counter()
    h = dd.ddamg_setup(U, w["dims"], -1, m0, w["csw"], p, tv)
    print(f"\n48^3x96 four-level mixed setup {time.perf_counter() - t0:.1f} s, device "
          f"{dd.ddamg_device_bytes(h) / 1e9:.1f} GB, phases {dd.ddamg_setup_times(h)[:3]}")
    del tv
    x = np.zeros_like(rhs)
    t0 = time.perf_counter()
    st = dd.ddamg_solve(h, rhs, x, 1, TOL)
    print(f"solve {time.perf_counter() - t0:.2f} s, {st}")
    h.free()
    assert st[0]["converged"] and st[0]["true_residual"] <= TOL, st
    build = lambda Up: WilsonOp.build(Up, m0, w["csw"], 1)   # noqa: E731
    sites = _sites(w["dims"], 24, 31)
    dx = apply_at_sites(build, U, x, (-1, 1, 1, 1), sites)
    rs = np.stack([rhs[0][s] for s in sites]) - dx[0]
    assert np.linalg.norm(rs) <= TOL * np.linalg.norm(rhs[0])
