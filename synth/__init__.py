"""Seeded synthetic inputs for the Wilson-clover multigrid solver.

This module only draws numbers: gauge links, right-hand sides, random test
vectors and gauge transformations.  It holds none of the solver's arithmetic
(no Dirac operator, no smoother, no transfer operator), so both the CPU
oracle and the CUDA library can be fed from it without sharing method code.

Layouts (all complex128, C-contiguous, so ``.view(np.float64)`` is the C-ABI
layout with interleaved re/im):

* gauge field ``U[t, z, y, x, mu, a, b]`` with ``mu`` = 0..3 = (t, z, y, x);
* fine spinor fields ``psi[n, t, z, y, x, 12]`` with index ``spin*3 + colour``;
* coarse fields ``phi[n, t, z, y, x, dof]``.

The gauge generator follows the recipe of the benchmark configurations: a
complex 3x3 matrix with independent N(0,1) real and imaginary parts, its
Hermitian traceless part H, U = exp(i*eps*H) (through a Hermitian
eigendecomposition), then re-unitarisation (Gram-Schmidt on rows 1 and 2,
row 3 = conj(row1 x row2)) so that det U = 1 to rounding.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "su3_field", "unit_gauge", "su3_matrices", "random_spinors", "random_fields",
    "point_sources", "random_test_vectors", "lattice_volume", "philox4x32_10", "philox_fields",
    "philox_test_vectors",
]


def lattice_volume(dims) -> int:
    T, Z, Y, X = dims
    return int(T) * int(Z) * int(Y) * int(X)


def su3_matrices(shape, eps: float, rng: np.random.Generator) -> np.ndarray:
    """Random SU(3) matrices exp(i*eps*H), re-unitarised; ``shape`` excludes (3, 3)."""
    full = tuple(shape) + (3, 3)
    a = rng.standard_normal(full) + 1j * rng.standard_normal(full)
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1) / 3.0
    h = h - tr[..., None, None] * np.eye(3)
    w, v = np.linalg.eigh(h)
    u = np.einsum("...ik,...k,...jk->...ij", v, np.exp(1j * eps * w), np.conj(v))
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.ascontiguousarray(np.stack([r0, r1, r2], axis=-2))


def su3_field(dims, eps: float, seed: int) -> np.ndarray:
    """Gauge links U[t,z,y,x,mu,3,3] for a T x Z x Y x X lattice."""
    rng = np.random.default_rng(seed)
    return su3_matrices(tuple(dims) + (4,), eps, rng)


def unit_gauge(dims) -> np.ndarray:
    g = np.zeros(tuple(dims) + (4, 3, 3), dtype=np.complex128)
    g[..., 0, 0] = g[..., 1, 1] = g[..., 2, 2] = 1.0
    return g


def random_fields(n: int, dims, ndof: int, seed: int) -> np.ndarray:
    """n complex N(0,1) fields (independent real and imaginary parts) of ndof per site."""
    rng = np.random.default_rng(seed)
    shape = (n,) + tuple(dims) + (ndof,)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_spinors(n: int, dims, seed: int) -> np.ndarray:
    return random_fields(n, dims, 12, seed)


def point_sources(dims, seed: int) -> np.ndarray:
    """12 point sources delta_{x,x0} delta_{spin,s} delta_{colour,c} at a seeded site x0."""
    rng = np.random.default_rng(seed)
    x0 = tuple(int(rng.integers(0, d)) for d in dims)
    out = np.zeros((12,) + tuple(dims) + (12,), dtype=np.complex128)
    for k in range(12):
        out[(k,) + x0 + (k,)] = 1.0
    return out


def random_test_vectors(dims_per_level, n_tv, seed: int):
    """Random start vectors for the setup, one array per level.

    Level 0 gets ``n_tv[0]`` fine spinor fields.  A coarser level l >= 1 gets
    ``max(0, n_tv[l] - n_tv[l-1])`` fields of ``2*n_tv[l-1]`` degrees of freedom
    per site: those fill up the test vectors that restriction from the level
    above does not provide.  ``dims_per_level[l]`` are the lattice dimensions
    of level l.
    """
    out = []
    for lvl, dims in enumerate(dims_per_level[:len(n_tv)]):
        if lvl == 0:
            out.append(random_fields(n_tv[0], dims, 12, seed))
        else:
            extra = max(0, n_tv[lvl] - n_tv[lvl - 1])
            out.append(random_fields(extra, dims, 2 * n_tv[lvl - 1], seed + 7919 * lvl)
                       if extra else None)
    return out


# ---------------------------------------------------------------------------
# Counter-based normal variates: the generator the CUDA library uses to draw the
# setup's random test vectors from a seed (Alg. 3 starts from random vectors).
# Both sides implement it from its published definition so that they draw the
# same bits: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
# as easy as 1, 2, 3", SC 2011) followed by the Box-Muller transform, whose
# logarithm, sine and cosine are evaluated below with IEEE-754 double additions,
# multiplications, divisions and square roots only (no fused multiply-add, no
# library transcendental), each rounded to nearest, in a fixed order that the
# CUDA kernel repeats operation by operation.
#
# Counter and key of the complex entry (field j, lexicographic site x, dof k) on
# level l:  ctr = (x, k, j, l),  key = (seed mod 2^32, seed div 2^32).
# From the four 32-bit outputs r0..r3:
#   u1 = ((r0 + 2^32 r1) >> 11) + 1) * 2^-53   in (0, 1]
#   u2 = ((r2 + 2^32 r3) >> 11)      * 2^-53   in [0, 1)
#   rho = sqrt(-2 ln u1),  entry = rho cos(2 pi u2) + i rho sin(2 pi u2),
# so real and imaginary parts are independent N(0, 1).

PHILOX_M = (0xD2511F53, 0xCD9E8D57)   # multipliers of Philox4x32
PHILOX_W = (0x9E3779B9, 0xBB67AE85)   # Weyl key increments
_MASK32 = np.uint64(0xFFFFFFFF)
LN2 = 0.6931471805599453               # ln 2 rounded to double
HALF_PI = 1.5707963267948966           # pi / 2 rounded to double
LOG_TERMS = 13                         # atanh series terms: s^1 .. s^25
TRIG_TERMS = 13                        # Taylor terms of sin and cos on [0, pi/2)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 arrays (broadcast); returns (r0, r1, r2, r3) as uint64."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK32 for v in (c0, c1, c2, c3)]
    k = [np.asarray(v, dtype=np.uint64) & _MASK32 for v in (k0, k1)]
    m0, m1 = np.uint64(PHILOX_M[0]), np.uint64(PHILOX_M[1])
    for r in range(10):
        if r > 0:
            k = [(k[0] + np.uint64(PHILOX_W[0])) & _MASK32, (k[1] + np.uint64(PHILOX_W[1])) & _MASK32]
        p0 = m0 * c[0]                     # exact: both factors < 2^32
        p1 = m1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
    return tuple(c)


def _ln(u):
    """ln u for u in (0, 1]: u = m 2^e with m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s),
    s = (m - 1)/(m + 1), by its odd power series to s^25 (Horner), plus e ln 2."""
    m, e = np.frexp(u)                     # m in [0.5, 1)
    low = m < 0.7071067811865476
    m = np.where(low, m * 2.0, m)
    e = np.where(low, e - 1, e).astype(np.float64)
    s = (m - 1.0) / (m + 1.0)
    t = s * s
    p = np.full_like(s, 1.0 / (2 * LOG_TERMS - 1))
    for i in range(LOG_TERMS - 2, -1, -1):
        p = p * t + 1.0 / (2 * i + 1)
    return 2.0 * (s * p) + e * LN2


def _trig_coefficients():
    """(-1)^k / (2k+1)! and (-1)^k / (2k)! for k < TRIG_TERMS, by repeated exact-integer divisions."""
    sc, cc = [1.0], [1.0]
    for k in range(1, TRIG_TERMS):
        sc.append(-sc[-1] / float((2 * k) * (2 * k + 1)))
        cc.append(-cc[-1] / float((2 * k - 1) * (2 * k)))
    return sc, cc


def _sincos_2pi(u):
    """(sin 2 pi u, cos 2 pi u) for u in [0, 1): quadrant q = floor(4u), theta = (4u - q) pi/2,
    Taylor series of sin and cos at theta (Horner in theta^2), then the quadrant's symmetry."""
    v = u * 4.0
    q = np.floor(v)
    th = (v - q) * HALF_PI
    t = th * th
    sc, cc = _trig_coefficients()
    ps = np.full_like(th, sc[-1])
    pc = np.full_like(th, cc[-1])
    for k in range(TRIG_TERMS - 2, -1, -1):
        ps = ps * t + sc[k]
        pc = pc * t + cc[k]
    S = th * ps
    C = pc
    q = q.astype(np.int64)
    sin = np.choose(q, [S, C, -S, -C])
    cos = np.choose(q, [C, -S, -C, S])
    return sin, cos


def philox_normal_pairs(x, k, j, level, seed):
    """Complex N(0,1) entries (independent real and imaginary parts) for counters (x, k, j, level)."""
    seed = int(seed)
    r0, r1, r2, r3 = philox4x32_10(x, k, j, level, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    a = ((r0 | (r1 << np.uint64(32))) >> np.uint64(11)) + np.uint64(1)
    b = (r2 | (r3 << np.uint64(32))) >> np.uint64(11)
    u1 = a.astype(np.float64) * 2.0 ** -53      # exact: a <= 2^53
    u2 = b.astype(np.float64) * 2.0 ** -53
    rho = np.sqrt(-2.0 * _ln(u1))
    s, c = _sincos_2pi(u2)
    out = np.empty(rho.shape, dtype=np.complex128)
    out.real = rho * c
    out.imag = rho * s
    return out


def philox_fields(n: int, dims, ndof: int, seed: int, level: int = 0, j0: int = 0) -> np.ndarray:
    """n complex N(0,1) fields [n, T, Z, Y, X, ndof] drawn by the counter-based generator
    (field indices j0 .. j0+n-1 on `level`); the same numbers the CUDA library draws.
    Drawn in slices of at most 2^20 entries, to bound the temporaries."""
    V = lattice_volume(dims)
    out = np.empty((n, V * ndof), dtype=np.complex128)
    lin = np.arange(V * ndof, dtype=np.uint64)
    step = 1 << 20
    for f in range(n):
        for a in range(0, V * ndof, step):
            e = lin[a:a + step]
            x = e // np.uint64(ndof)
            k = e - x * np.uint64(ndof)
            out[f, a:a + step] = philox_normal_pairs(x, k, np.uint64(j0 + f), np.uint64(level), seed)
    return np.ascontiguousarray(out.reshape((n,) + tuple(dims) + (ndof,)))


def philox_test_vectors(dims_per_level, n_tv, seed: int):
    """The random start vectors of the setup as the library draws them from `seed` (same layout
    as random_test_vectors): level 0 fields j = 0..N_0-1, level l >= 1 the extra fields
    j = 0..N_l - N_{l-1} - 1 with 2 N_{l-1} dof per site."""
    out = []
    for lvl, dims in enumerate(dims_per_level[:len(n_tv)]):
        if lvl == 0:
            out.append(philox_fields(n_tv[0], dims, 12, seed, 0))
        else:
            extra = max(0, n_tv[lvl] - n_tv[lvl - 1])
            out.append(philox_fields(extra, dims, 2 * n_tv[lvl - 1], seed, lvl) if extra else None)
    return out
