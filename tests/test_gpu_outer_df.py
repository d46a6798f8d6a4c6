"""The outer solver's double-FP32 option (DDAMG_OPT_OUTER_DF): the fine operator evaluated in
double-FP32 arithmetic on FP64 vectors against the FP64 oracle (the FP64 bound of 1e-12 per
application; the pairs carry about 48 bits), and mixed solves whose outer FGMRES forms D z_j and
its Gram-Schmidt products that way, held to the FP64 true-residual bound of 1e-10.
"""
import numpy as np
import pytest

import synth
from cases import Case, rel, SMALL2, RAGGED2, BIG3, C1, golden_mass

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1307_6101_gb300 as m
    return m


@pytest.mark.parametrize("spec,csw,bc", [(SMALL2, 1.0, -1), (SMALL2, 0.0, 1), (RAGGED2, 1.3, -1)])
def test_df_operator_matches_oracle(dd, spec, csw, bc):
    from oracle.wilson import WilsonOp
    c = Case(**spec, csw=csw, bc_t=bc)
    U = c.gauge()
    h = c.gpu(0, U)
    op = WilsonOp.build(U, c.m0, c.csw, c.bc_t)
    f = np.ascontiguousarray(synth.random_spinors(3, c.dims, 7))
    for scale in (1.0, 1e-20, 1e20):
        fs = np.ascontiguousarray(f * scale)
        out = np.zeros_like(fs)
        dd.ddamg_apply(h, 0, 2, fs, out, 3)
        ref = np.stack([op.apply(fs[i]) for i in range(3)])
        assert rel(out, ref) <= 1e-12, (scale, rel(out, ref))
        # the FP64 kernel on the same fields, for the record of the gap
        out64 = np.zeros_like(fs)
        dd.ddamg_apply(h, 0, 0, fs, out64, 3)
        assert rel(out64, ref) <= 1e-14


def _true_residual(U, c, b, x):
    from oracle.wilson import WilsonOp
    op = WilsonOp.build(U, c.m0, c.csw, c.bc_t)
    return np.linalg.norm(b - op.apply(x)) / np.linalg.norm(b)


@pytest.mark.parametrize("which", ["two_level", "three_level"])
def test_solve_with_df_outer_meets_fp64_bound(dd, which):
    if which == "two_level":
        c = Case(**C1, m0=golden_mass("eps0.3_csw0"), max_rhs=2)
    else:
        c = Case(**BIG3, n_inv=1, eta_passes=3, max_rhs=2, m0=-0.35, nu=3)
    U = c.gauge()
    h = c.gpu(2, U)
    b = np.ascontiguousarray(synth.random_spinors(2, c.dims, 3))
    its = {}
    for df in (0, 1):
        dd.ddamg_set_option(h, dd.DDAMG_OPT_OUTER_DF, df)
        assert dd.ddamg_get_option(h, dd.DDAMG_OPT_OUTER_DF) == df
        x = np.zeros_like(b)
        st = dd.ddamg_solve(h, b, x, 2, 1e-10)
        for i in range(2):
            assert st[i]["converged"]
            assert _true_residual(U, c, b[i], x[i]) <= 1e-10
        its[df] = [s["iterations"] for s in st]
    for a, b_ in zip(its[0], its[1]):
        assert abs(a - b_) <= 1, its
