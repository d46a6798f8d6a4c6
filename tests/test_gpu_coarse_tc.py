"""The tensor-core coarse stencil (FP16 blocks, FP16 hi + lo split of the vectors, FP32 accumulate)
against the oracle's coarse operator on the same dequantised FP16 blocks, for every kernel the
autotuner may choose; bit-identical columns alone and in a batch; the autotuner's choice."""
import numpy as np
import pytest

import synth
from cases import Case, rel, THREE, SAP4

pytestmark = pytest.mark.gpu

TOL32 = 2e-6
# the coarse dof of the three-level workloads at a small size: n = 40 on level 1 and n = 56 on level 2 (the three-level workloads'
# coarse dof); level 2 is 2x1x1x1 (odd extents, so it is applied by the stencil kernel too)
WIDE = dict(dims=(16, 8, 8, 8), levels=3, agg=((4, 4, 4, 4), (2, 2, 2, 2)), n_tv=(20, 28),
            sap=((4, 4, 4, 4), (2, 2, 2, 2)))


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1307_6101_gb300 as m
    return m


def _setup(dd, spec, max_rhs):
    c = Case(**spec, n_inv=0, eta_passes=0, max_rhs=max_rhs)
    U = c.gauge()
    tv = c.random_tv()
    h = c.gpu(0, U, tv)
    dd.ddamg_set_option(h, dd.DDAMG_OPT_HALF_STORAGE, 1)
    return c, h, c.oracle(U, tv)


@pytest.mark.parametrize("spec", [SAP4, THREE, WIDE])
def test_tensor_core_stencil_every_candidate(dd, spec):
    from oracle.precision import stencil_half
    c, h, o = _setup(dd, spec, 20)
    for ks in range(0, 5):
        dd.ddamg_set_option(h, dd.DDAMG_OPT_COARSE_TC, ks)
        for l in range(1, c.levels):
            dims, n, _ = h.level_info(l)
            stq = stencil_half(o.levels[l].op)
            f = np.ascontiguousarray(synth.random_fields(20, dims, n, 70 + l))
            f[3] *= 1e-3                              # columns of very different size in one batch
            f[7] = 0.0
            out = np.zeros_like(f)
            dd.ddamg_apply(h, l, 1, f, out, 20)
            for r in range(20):
                if r == 7:
                    assert not np.any(out[r])
                    continue
                ref = stq.apply(f[r])
                assert rel(out[r], ref) <= TOL32, (ks, l, r, rel(out[r], ref))
            # one column alone gives the same bits as inside the batch
            one = np.zeros_like(f[:1])
            dd.ddamg_apply(h, l, 1, np.ascontiguousarray(f[17:18]), one, 1)
            assert np.array_equal(one[0], out[17]), (ks, l)
    h.free()


def test_autotuner_keeps_the_fastest_candidate(dd):
    c, h, o = _setup(dd, WIDE, 12)
    dd.ddamg_set_option(h, dd.DDAMG_OPT_COARSE_TC, -1)
    for kind, levels in (("coarse", (1, 2)), ("restrict", (0, 1)), ("prolong", (0, 1))):
        for l in levels:
            ms, chosen = dd.ddamg_autotune_times(h, kind, l)
            timed = [k for k in range(5) if ms[k] >= 0]
            assert 0 in timed and 1 in timed, (kind, l, ms)
            assert chosen == min(timed, key=lambda k: ms[k]), (kind, l, ms, chosen)
    assert dd.ddamg_get_option(h, dd.DDAMG_OPT_COARSE_TC) == dd.ddamg_autotune_times(h, "coarse", 1)[1]
    # a solve with the tuned kernels still reaches the FP64 true residual
    b = np.ascontiguousarray(synth.random_spinors(2, c.dims, 3))
    x = np.zeros_like(b)
    st = dd.ddamg_solve(h, b, x, 2, 1e-10)
    assert all(s["converged"] and s["true_residual"] <= 1e-10 for s in st), st
    h.free()


@pytest.mark.parametrize("spec", [SAP4, THREE, WIDE])
def test_batch_transfer_kernels_every_candidate(dd, spec):
    """Restriction on tensor cores (P read once per batch) and the batch prolongation against the
    oracle on the same FP16-rounded P, every candidate; columns alone equal columns in a batch."""
    from oracle.transfer import restrict, prolong
    from oracle.precision import interpolation_half
    c, h, o = _setup(dd, spec, 20)
    for ks in range(0, 5):
        dd.ddamg_set_option(h, dd.DDAMG_OPT_COARSE_TC, ks)
        for l in range(c.levels - 1):
            dims, n, N = h.level_info(l)
            cdims, nc, _ = h.level_info(l + 1)
            Pq = interpolation_half(o.levels[l].P, c.agg[l])
            f = np.ascontiguousarray(synth.random_fields(20, dims, n, 80 + l))
            f[2] *= 1e4
            f[5] = 0.0
            g = np.ascontiguousarray(synth.random_fields(20, cdims, nc, 90 + l))
            out = np.zeros_like(g)
            dd.ddamg_restrict(h, l, 1, f, out, 20)
            back = np.zeros_like(f)
            dd.ddamg_prolong(h, l, 1, g, back, 20)
            for r in range(20):
                if r == 5:
                    assert not np.any(out[r])
                    continue
                ref = restrict(Pq, c.agg[l], f[r])
                assert rel(out[r], ref) <= TOL32, (ks, l, r, rel(out[r], ref))
                refp = prolong(Pq, c.agg[l], g[r])
                assert rel(back[r], refp) <= TOL32, (ks, l, r, rel(back[r], refp))
            one = np.zeros_like(g[:1])
            dd.ddamg_restrict(h, l, 1, np.ascontiguousarray(f[13:14]), one, 1)
            assert np.array_equal(one[0], out[13]), (ks, l)
            onep = np.zeros_like(f[:1])
            dd.ddamg_prolong(h, l, 1, np.ascontiguousarray(g[13:14]), onep, 1)
            assert np.array_equal(onep[0], back[13]), (ks, l)
    h.free()
