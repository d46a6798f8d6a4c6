"""Pins of the FP16 storage rule of oracle.precision: IEEE binary16 rounding,
the per-group error bound, the grouping of the scales, and properties of the
dequantised operators."""
import numpy as np
import pytest

import synth
from oracle.precision import half, scaled_half, fine_op_half, interpolation_half, stencil_half
from oracle.wilson import WilsonOp
from oracle.gamma import GAMMA
from oracle.stencil import Stencil


def test_half_round_to_nearest_even():
    u = 2.0 ** -10                                # binary16 spacing in [1, 2)
    cases = [
        (1.0 + u / 2, 1.0),                       # tie -> even mantissa (1.0)
        (1.0 + 1.5 * u, 1.0 + 2 * u),             # tie -> even mantissa
        (1.0 + u / 2 + 2.0 ** -40, 1.0 + u),      # just above the tie: rounded from the double directly
        (2049.0, 2048.0), (2051.0, 2052.0),       # spacing 2 in [2048, 4096)
        (65504.0, 65504.0),                       # largest finite binary16
        (2.0 ** -24, 2.0 ** -24),                 # smallest subnormal
        (2.0 ** -25, 0.0),                        # tie between 0 and 2^-24 -> 0
        (0.75 * 2.0 ** -24, 2.0 ** -24),
        (-1.0 - 1.5 * u, -1.0 - 2 * u),           # symmetric in sign
    ]
    for x, want in cases:
        assert half(np.array([x]))[0] == want, (x, half(np.array([x]))[0], want)
    z = half(np.array([(1.0 + u / 2) + 1j * (1.0 + 1.5 * u)]))[0]
    assert z == complex(1.0, 1.0 + 2 * u)


def test_scaled_half_error_bound_and_maximum():
    rng = np.random.default_rng(3)
    v = (rng.standard_normal((5, 40)) + 1j * rng.standard_normal((5, 40))) * np.array([1.0, 3.7, 1e-6, 0.2, 9e3])[:, None]
    q = scaled_half(v, axes=(1,))
    for g in range(5):
        m = max(np.abs(v[g].real).max(), np.abs(v[g].imag).max())
        err = np.maximum(np.abs((q[g] - v[g]).real), np.abs((q[g] - v[g]).imag))
        # |x / sigma| <= 1, so the binary16 spacing is <= 2^-10 and the error <= 2^-11 sigma (+ fp32 scale rounding)
        assert err.max() <= 2.0 ** -11 * m * (1 + 2.0 ** -20)
        # the entry of largest modulus is exact up to the FP32 rounding of the scale
        k = np.argmax(np.maximum(np.abs(v[g].real), np.abs(v[g].imag)))
        big = v[g, k].real if abs(v[g, k].real) >= abs(v[g, k].imag) else v[g, k].imag
        qb = q[g, k].real if abs(v[g, k].real) >= abs(v[g, k].imag) else q[g, k].imag
        assert abs(qb - big) <= 2.0 ** -24 * abs(big)
    # a zero group stays zero
    assert np.all(scaled_half(np.zeros((2, 3), complex), axes=(1,)) == 0)


def test_interpolation_half_groups_per_aggregate_and_chirality():
    dims, agg, N, n = (4, 2, 2, 2), (2, 2, 2, 2), 3, 12
    rng = np.random.default_rng(5)
    P = rng.standard_normal((N,) + dims + (n,)) + 1j * rng.standard_normal((N,) + dims + (n,))
    # aggregates along t: 0 and 1; chirality: dofs 0..5 / 6..11; very different magnitudes per group
    mag = {(0, 0): 1.0, (0, 1): 1e-6, (1, 0): 2e-5, (1, 1): 3.0}
    for (a, s), m in mag.items():
        P[:, 2 * a:2 * a + 2, ..., 6 * s:6 * s + 6] *= m
    q = interpolation_half(P, agg)
    for (a, s), m in mag.items():
        blk = P[:, 2 * a:2 * a + 2, ..., 6 * s:6 * s + 6]
        qb = q[:, 2 * a:2 * a + 2, ..., 6 * s:6 * s + 6]
        sig = max(np.abs(blk.real).max(), np.abs(blk.imag).max())
        err = np.maximum(np.abs((qb - blk).real), np.abs((qb - blk).imag)).max()
        # a scale shared with a larger group would push these entries into the binary16 subnormals
        assert err <= 2.0 ** -11 * sig * (1 + 2.0 ** -20), (a, s, err / sig)


def test_stencil_half_groups_per_site():
    rng = np.random.default_rng(6)
    dims, n = (2, 2, 2, 2), 4

    def r(*s):
        return rng.standard_normal(s) + 1j * rng.standard_normal(s)

    st = Stencil(diag=r(*dims, n, n), fwd=r(4, *dims, n, n), bwd=r(4, *dims, n, n))
    scale = np.exp(rng.uniform(-14, 3, size=dims))           # site magnitudes spanning 1e-6 .. 20
    st = Stencil(diag=st.diag * scale[..., None, None], fwd=st.fwd * scale[None, ..., None, None],
                 bwd=st.bwd * scale[None, ..., None, None])
    q = stencil_half(st)
    for idx in np.ndindex(*dims):
        blocks = [st.diag[idx]] + [st.fwd[mu][idx] for mu in range(4)] + [st.bwd[mu][idx] for mu in range(4)]
        qblocks = [q.diag[idx]] + [q.fwd[mu][idx] for mu in range(4)] + [q.bwd[mu][idx] for mu in range(4)]
        sig = max(max(np.abs(b.real).max(), np.abs(b.imag).max()) for b in blocks)
        for b, qb in zip(blocks, qblocks):
            err = np.maximum(np.abs((qb - b).real), np.abs((qb - b).imag)).max()
            assert err <= 2.0 ** -11 * sig * (1 + 2.0 ** -20)


def test_fine_op_half_free_field_is_exact():
    """Unit links and the zero clover term are binary16 numbers: the FP16 operator is the free one."""
    dims = (4, 4, 4, 4)
    m0 = 0.21
    op = fine_op_half(synth.unit_gauge(dims), m0, 1.0, bc_t=1)
    p = np.array([2 * np.pi / 4, 0.0, 2 * np.pi * 3 / 4, 2 * np.pi / 4])
    co = np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")
    u = np.random.default_rng(1).standard_normal(12) + 0j
    psi = np.exp(1j * sum(p[m] * co[m] for m in range(4)))[..., None] * u
    Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
    expect = np.einsum("st,...tc->...sc", Dp, psi.reshape(dims + (4, 3))).reshape(psi.shape)
    assert np.allclose(op.apply(psi), expect, rtol=0, atol=1e-13)


def test_fine_op_half_gamma5_symmetric_and_close():
    dims = (4, 4, 4, 4)
    U = synth.su3_field(dims, 0.4, 2)
    op = fine_op_half(U, -0.3, 1.0)
    ref = WilsonOp.build(U, -0.3, 1.0)
    f = synth.random_fields(2, dims, 12, 4)
    g5 = op.gamma5
    lhs = np.vdot(f[0], g5 * op.apply(g5 * f[1]))
    rhs = np.vdot(op.apply(f[0]), f[1])
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # the stored links are within half a binary16 spacing of the FP64 links (|U_ab| <= 1)
    assert np.abs(op.U - U).max() <= 2.0 ** -11 * np.sqrt(2)
    d = np.linalg.norm(op.apply(f[0]) - ref.apply(f[0])) / np.linalg.norm(ref.apply(f[0]))
    assert 1e-6 < d < 2e-3   # the FP16 operator differs from the FP64 one, by the FP16 rounding


def test_even_odd_half_keeps_fp64_self_inverses():
    from oracle.precision import even_odd_half
    rng = np.random.default_rng(8)
    dims, n = (2, 2, 2, 2), 4

    def r(*s):
        return rng.standard_normal(s) + 1j * rng.standard_normal(s)

    st = Stencil(diag=r(*dims, n, n) + 4 * np.eye(n), fwd=r(4, *dims, n, n), bwd=r(4, *dims, n, n))
    eo = even_odd_half(st)
    assert np.allclose(eo.diag_inv @ st.diag, np.eye(n), atol=1e-13)
    assert not np.allclose(eo.op.diag, st.diag, atol=1e-6)     # the blocks themselves are FP16
