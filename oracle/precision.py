"""FP16 storage of the preconditioner's operator data, dequantised to FP64.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper computes and applies the whole preconditioner in single precision
and keeps the outer FGMRES in double (Sec. 3, opening paragraph); it has no
half-precision storage.  The FP16 storage format of the FP32 preconditioner is
this project's, and this module states it so that the oracle can apply, in
FP64, exactly the operator the FP32 kernels read:

* half(x): x rounded to the nearest IEEE binary16 number, ties to even, the
  real and imaginary parts separately;
* links U_mu(x): half(U), no scale (SU(3) entries have modulus <= 1);
* clover term C(x) (the site-local part of D without the (m0 + 4) shift):
  half(C), no scale; the shift is added back in the arithmetic;
* P_l: one scale per aggregate A and chirality s,
  sigma(A, s) = fp32(max |Re|, |Im| over the N columns restricted to (A, s)),
  stored value sigma * half(x / sigma);
* coarse blocks: one scale per site A over its 9 blocks S(A), F_mu(A), B_mu(A),
  sigma(A) = fp32(max |Re|, |Im|), stored value sigma * half(x / sigma);
* the inverses S(A)^{-1} of the coarsest level's self blocks (odd-even solve)
  are not FP16: they are the inverses of the FP64 blocks, kept in FP32.

A group that is all zero gets sigma = 1.  Dividing by the FP32-rounded scale
makes sigma * half(x / sigma) the exact value the kernels multiply with.
"""
from __future__ import annotations

import numpy as np

from .lattice import to_blocks, from_blocks
from .stencil import Stencil, EvenOdd
from .wilson import WilsonOp, clover_term


def half(x: np.ndarray) -> np.ndarray:
    """Round to the nearest binary16 (ties to even), returned as float64 / complex128."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return half(x.real) + 1j * half(x.imag)
    return x.astype(np.float64).astype(np.float16).astype(np.float64)


def group_scale(v: np.ndarray, axes) -> np.ndarray:
    """fp32(max |Re|, |Im|) over `axes` (keepdims), 1 where the group is zero."""
    m = np.maximum(np.abs(v.real), np.abs(v.imag)).max(axis=axes, keepdims=True)
    s = m.astype(np.float32).astype(np.float64)
    return np.where(m > 0, s, 1.0)


def scaled_half(v: np.ndarray, axes) -> np.ndarray:
    """sigma * half(v / sigma) with one sigma per group (the axes reduced over)."""
    s = group_scale(v, axes)
    return s * half(v / s)


def fine_op_half(U: np.ndarray, m0: float, csw: float, bc_t: int = -1) -> WilsonOp:
    """The Wilson-clover operator on FP16 links and the FP16 clover term."""
    Uq = half(U)
    C = half(clover_term(U, csw))
    diag = C + (m0 + 4.0) * np.eye(12)
    return WilsonOp(U=Uq, diag=diag, bc=(int(bc_t), 1, 1, 1))


def interpolation_half(P: np.ndarray, agg) -> np.ndarray:
    """P[N, T, Z, Y, X, n] with one scale per (aggregate, chirality) over the N columns."""
    n = P.shape[-1]
    h = n // 2
    pb = to_blocks(P, agg)                       # [N, Tb, Zb, Yb, Xb, vol, n]
    out = np.empty_like(pb)
    for s in range(2):
        part = pb[..., s * h:(s + 1) * h]
        # reduce over the columns (axis 0), the sites of the aggregate and the dofs of s
        out[..., s * h:(s + 1) * h] = scaled_half(part, axes=(0, -2, -1))
    return from_blocks(out, agg)


def stencil_half(st: Stencil) -> Stencil:
    """A coarse stencil with one scale per site over its 9 blocks."""
    allb = np.concatenate([st.diag[None], st.fwd, st.bwd], axis=0)   # [9, T, Z, Y, X, n, n]
    q = scaled_half(allb, axes=(0, -2, -1))
    return Stencil(diag=q[0], fwd=q[1:5], bwd=q[5:9])


def even_odd_half(st: Stencil) -> EvenOdd:
    """Odd-even form of the FP16 coarsest operator: FP16 blocks, self inverses of the FP64 blocks."""
    eo = EvenOdd(stencil_half(st))
    eo.diag_inv = np.linalg.inv(st.diag)
    return eo
