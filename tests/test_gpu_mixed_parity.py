"""The mixed-precision path's building blocks against the oracle (the pieces the benchmark's
mixed solve is made of, beyond single operator applications):

* the Galerkin products D_{l+1} = P^+ D_l P that a handle with the FP32 preconditioner forms in
  FP32 from the FP32 copies of D and P (Sec. 3: the preconditioner's setup in single
  precision), against the oracle's FP64 product of the same FP32-rounded operands;
* Alg. 3's smoothing of the random test vectors in FP32 (FP32 and FP16 storage), against the
  oracle's smoothing with the same rounded operator;
* one whole K-cycle (Alg. 2) in FP32 arithmetic on FP16 storage, against the oracle's K-cycle
  on the dequantised operators of every level, with the inner tolerances set below anything
  reachable so that both sides take the same fixed number of Krylov steps.

Bounds (relative 2-norm):
* Galerkin, 1e-5: each stored entry is a sum over an aggregate of up to 256 sites x 6 spin-colour
  products formed in FP32 (tree-ordered partial sums, error ~ log2(1536) u_32 = 7e-7 of the
  summed magnitude), and the hop blocks cancel by up to about ten to one;
* Alg. 3 smoothing, 1e-5: eta_passes = 2 chains 1 + 2 SAP applications per vector, each an
  FP32 result within 2e-6 of its exact value;
* K-cycle, 1e-4: its longest chain of dependent FP32 operator applications is about fifty long
  (two cycles of five inner steps, each through a level-1 cycle of twenty coarsest GMRES steps
  and two SAP applications), each within 2e-6.
"""
import numpy as np
import pytest

import synth
from cases import Case, rel, THREE, SAP4

pytestmark = pytest.mark.gpu

TOL_GALERKIN = 1e-5
TOL_SMOOTH = 1e-5
TOL_KCYCLE = 1e-4


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1307_6101_gb300 as m
    return m


def f32(a):
    a = np.asarray(a)
    return a.astype(np.complex64 if np.iscomplexobj(a) else np.float32).astype(a.dtype)


def fine_op_single(U, m0, csw, bc_t):
    """The Wilson-clover operator on FP32-rounded links and site-diagonal part (the FP32 copies)."""
    from oracle.wilson import WilsonOp, site_diagonal
    return WilsonOp(U=f32(U), diag=f32(site_diagonal(U, m0, csw)), bc=(int(bc_t), 1, 1, 1))


def stencil_single(st):
    from oracle.stencil import Stencil
    return Stencil(diag=f32(st.diag), fwd=f32(st.fwd), bwd=f32(st.bwd))


def _blocks(dd, h, lvl):
    dims, n, _ = h.level_info(lvl)
    V = int(np.prod(dims))
    out = np.zeros((V, 9, n, n), dtype=np.complex128)
    dd.ddamg_get_coarse_operator(h, lvl, out)
    return out


def _oracle_blocks(st):
    """Oracle stencil -> the library's [site lex][k][row][col] block order."""
    dims = st.dims
    V = int(np.prod(dims))
    n = st.ndof
    allb = [st.diag] + [st.fwd[mu] for mu in range(4)] + [st.bwd[mu] for mu in range(4)]
    return np.stack([b.reshape(V, n, n) for b in allb], axis=1)


@pytest.mark.parametrize("spec", [SAP4, THREE])
def test_fp32_galerkin_products(dd, spec):
    from oracle.transfer import build_interpolation, galerkin
    c = Case(**spec, n_inv=0, eta_passes=0)
    U = c.gauge()
    tv = c.random_tv()
    h = c.gpu(1, U, tv)                       # precision 1: Galerkin in FP32 from FP32 copies
    op = fine_op_single(U, c.m0, c.csw, c.bc_t)
    P0 = build_interpolation(tv[0], c.agg[0])
    D1 = galerkin(op, f32(P0), c.agg[0])
    got1 = _blocks(dd, h, 1)
    assert rel(got1, _oracle_blocks(D1)) <= TOL_GALERKIN, rel(got1, _oracle_blocks(D1))
    # the FP64 product of the unrounded operands differs by the FP32 rounding of the inputs
    from oracle.wilson import WilsonOp
    D1x = galerkin(WilsonOp.build(U, c.m0, c.csw, c.bc_t), P0, c.agg[0])
    assert rel(got1, _oracle_blocks(D1x)) > 1e-8
    if c.levels > 2:
        from oracle.transfer import restrict
        take = min(c.n_tv[0], c.n_tv[1])
        tv1 = np.concatenate([restrict(P0, c.agg[0], tv[0][:take]), tv[1][:c.n_tv[1] - take]], axis=0)
        P1 = build_interpolation(tv1, c.agg[1])
        D2 = galerkin(stencil_single(D1), f32(P1), c.agg[1])
        got2 = _blocks(dd, h, 2)
        assert rel(got2, _oracle_blocks(D2)) <= TOL_GALERKIN, rel(got2, _oracle_blocks(D2))
    h.free()


@pytest.mark.parametrize("precision", [1, 2])
def test_fp32_setup_smoothing_alg3(dd, precision):
    from oracle.multigrid import Hierarchy
    from oracle.precision import fine_op_half
    c = Case(**SAP4, n_inv=0, eta_passes=2, mr_steps=4)
    U = c.gauge()
    tv = c.random_tv()
    h = c.gpu(precision, U, tv)
    got = np.zeros_like(tv[0])
    dd.ddamg_get_testvectors(h, 0, got, c.n_tv[0])
    op = fine_op_single(U, c.m0, c.csw, c.bc_t) if precision == 1 else fine_op_half(U, c.m0, c.csw, c.bc_t)
    o = Hierarchy(op, c.oracle_params())
    o.initial_setup_phase(0, [v.copy() if v is not None else None for v in tv])
    ref = o.levels[0].tv
    assert rel(got, ref) <= TOL_SMOOTH, rel(got, ref)
    assert rel(got, tv[0]) > 1e-2                 # the vectors were smoothed
    h.free()


def test_half_storage_kcycle_matches_oracle(dd):
    from oracle.multigrid import Hierarchy
    from oracle.precision import fine_op_half, interpolation_half, stencil_half, even_odd_half
    from oracle.smoother import SAP
    from oracle.lattice import red_black_block
    extra = dict(kcycle_tol=1e-30, coarse_tol=1e-30, coarse_cycles=2, kcycle_len=5, kcycle_cycles=2)
    c = Case(**THREE, n_inv=0, eta_passes=0, nu=2, coarse_restart=10, max_rhs=2, extra=extra)
    U = c.gauge()
    tv = c.random_tv()
    h = c.gpu(0, U, tv)                       # FP64 setup: P and D_l agree with the oracle's to 1e-12
    dd.ddamg_set_option(h, dd.DDAMG_OPT_HALF_STORAGE, 1)
    o = c.oracle(U, tv)
    # the oracle hierarchy on the dequantised FP16 data the FP32 kernels read
    q = Hierarchy(fine_op_half(U, c.m0, c.csw, c.bc_t), c.oracle_params())
    q.levels = [type(lv)(op=lv.op) for lv in o.levels]
    q.levels[0].op = fine_op_half(U, c.m0, c.csw, c.bc_t)
    for l in range(c.levels - 1):
        q.levels[l].P = interpolation_half(o.levels[l].P, c.agg[l])
        if l > 0:
            q.levels[l].op = stencil_half(o.levels[l].op)
        q.levels[l].sap = SAP(q.levels[l].op, red_black_block(q.levels[l].op.dims, c.sap[l]), c.mr_steps)
    q.levels[-1].op = stencil_half(o.levels[-1].op)
    q.levels[-1].eo = even_odd_half(o.levels[-1].op)
    b = np.ascontiguousarray(synth.random_spinors(2, c.dims, 31))
    z = np.zeros_like(b)
    dd.ddamg_kcycle(h, 0, 1, b, z, 2)
    ref = np.stack([q.kcycle(0, b[i]) for i in range(2)])
    assert rel(z, ref) <= TOL_KCYCLE, rel(z, ref)
    # and the FP16 data made a difference: the oracle's FP64-data cycle is further away
    ref64 = np.stack([o.kcycle(0, b[i]) for i in range(2)])
    assert rel(z, ref64) > rel(z, ref)
    h.free()
